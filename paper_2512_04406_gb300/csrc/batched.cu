// Thousands of small instances in one persistent launch (manidsdp_batch_*).
//
// Every CTA takes instances from a global counter (dynamic scheduling, so
// instances of uneven size balance across the SMs) and runs the whole of
// Algorithm 1 on each, with the readings of the single-instance path and its
// oracle: RTR with truncated CG on the ALM subproblem (Section 4, Proposition
// 4.2), the multiplier update and certificate (Algorithm 1 steps 4-9), the rank
// update, the sigma rule (5.1), the rank-one rounding, the carried
// negative-curvature direction (Theorem 4.5).  Every decision is taken on the
// device; the host only packs the instances and reads the results.
//
// Sizes: N <= 128 (moment matrices of the order-1 relaxations with n <= 127 and
// of the order-2 ones with n <= 14), factor width p <= 32.  The cost, gradient,
// multiplier and certificate are FP64; the tCG Hessian-vector products are FP32
// (W = Y Up' + Up Y' and Q(W) = W - A*(w) entrywise, T = G Up + sigma Q(W) Y).
// The certificate's eigenpairs (and those of the p x p Gram Y'Y of the rank
// update) come from a parallel two-sided Jacobi method in FP64: n/2 disjoint
// rotations per step in round-robin order, rows then columns, until the
// off-diagonal mass is below 1e-30 of the total.
//
// Per-CTA workspace in global memory (reused across the CTA's instances, L1/L2
// resident at these sizes).  Instance data: the N x N index map, per-class lists
// of the upper-triangle entries (class-sum order fixed, so results are
// deterministic), multiplicities and b.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <vector>

#include "common.cuh"

namespace mds {
namespace {

constexpr int kBMaxN = 128;
constexpr int kBMaxP = 32;

struct BInst {
  int N, m;
  long long off_idx;   // N*N int32 (class of each entry)
  long long off_cptr;  // m+1 int32: entries of class a at cent[cptr[a] .. cptr[a+1])
  long long off_cent;  // upper-triangle entries r*N + c (r <= c), int32
  long long off_cls;   // m doubles: mult, then b (2m)
  long long off_y0;    // element offset of the N x p0 starting factor in Y0
};

struct BParams {
  double sigma0, sigma_min, sigma_max, gamma, kappa1, kappa2, tol;
  double tol_grad_min, tol_grad_max, tol_grad_factor, rank_tol, neg_tol, tcg_floor, tcg_abs;
  double carry_t0, round_eta;
  int p0, p_min, p_max, delta_max, max_outer, max_rtr, max_tcg, carry_halvings;
  int fp64;  // 1: FP64 Hessian-vector products (MANIDSDP_PREC_FP64)
};

struct BOut {  // per instance
  double value, eta_p, eta_d, eta_g, lambda_min;
  int status, p, outer, hessvecs;
};

// Per-CTA workspace offsets (doubles), for Nmax, mmax.
struct BLayout {
  long long XD, G, E, EV, W32, G32;             // N*N (W32, G32 floats in double slots)
  long long Y, Yt, grad, eta, Heta, r, dlt, Hd, Up, U, GY, T;  // N*P
  long long y, yt, w;                            // m
  long long z, zt, ev, tmpN;                     // N
  long long gram, gev, gvec;                     // P*P
  long long total;
};

__host__ __device__ inline BLayout make_layout(int N, int m) {
  BLayout L;
  long long o = 0;
  const long long nn = (long long)N * N, np = (long long)N * kBMaxP, pp = kBMaxP * kBMaxP;
  L.XD = o; o += nn; L.G = o; o += nn; L.E = o; o += nn; L.EV = o; o += nn;
  L.W32 = o; o += (nn + 1) / 2; L.G32 = o; o += (nn + 1) / 2;
  L.Y = o; o += np; L.Yt = o; o += np; L.grad = o; o += np; L.eta = o; o += np;
  L.Heta = o; o += np; L.r = o; o += np; L.dlt = o; o += np; L.Hd = o; o += np;
  L.Up = o; o += np; L.U = o; o += np; L.GY = o; o += np; L.T = o; o += np;
  L.y = o; o += m; L.yt = o; o += m; L.w = o; o += m;
  L.z = o; o += N; L.zt = o; o += N; L.ev = o; o += N; L.tmpN = o; o += N;
  L.gram = o; o += pp; L.gev = o; o += kBMaxP; L.gvec = o; o += pp;
  L.total = o;
  return L;
}

// The device code for each CTA size the tuner chooses from.
namespace bt128 {
constexpr int kBT = 128;
#include "batched_dev.cuh"
}  // namespace bt128
namespace bt256 {
constexpr int kBT = 256;
#include "batched_dev.cuh"
}  // namespace bt256

}  // namespace

// ---- host side --------------------------------------------------------------
namespace {

BParams to_bparams(const manidsdp_params& p) {
  BParams b{};
  b.sigma0 = p.sigma0; b.sigma_min = p.sigma_min; b.sigma_max = p.sigma_max; b.gamma = p.gamma;
  b.kappa1 = p.kappa1; b.kappa2 = p.kappa2; b.tol = p.tol; b.tol_grad_min = p.tol_grad_min;
  b.tol_grad_max = p.tol_grad_max; b.tol_grad_factor = p.tol_grad_factor; b.rank_tol = p.rank_tol;
  b.neg_tol = p.neg_tol; b.tcg_floor = p.tcg_floor; b.tcg_abs = p.tcg_abs; b.carry_t0 = p.carry_t0;
  b.round_eta = p.round_eta; b.p0 = p.p0; b.p_min = p.p_min; b.p_max = p.p_max;
  b.delta_max = p.delta_max; b.max_outer = p.max_outer; b.max_rtr = p.max_rtr;
  b.max_tcg = p.max_tcg; b.carry_halvings = p.carry_halvings;
  b.fp64 = p.precision_mode == MANIDSDP_PREC_FP64 ? 1 : 0;
  return b;
}

size_t align16(size_t x) { return (x + 15) / 16 * 16; }

using KernelFn = void (*)(int, const BInst*, const char*, const double*, BParams, double*, long long,
                          int, int, int*, BOut*, double*, const long long*);

KernelFn kernel_for(int threads) {
  return threads == 128 ? bt128::batched_solve_kernel : bt256::batched_solve_kernel;
}

// Tuned launch shapes, shared by every batch of the process: key (N_max, p_max,
// precision) -> (threads per CTA, CTAs per SM).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tuned;

}  // namespace
}  // namespace mds

struct manidsdp_batch {
  int ninst = 0, nmax = 0, mmax = 0, sms = 1;
  long long y0_len = 0, y_len = 0;
  cudaStream_t s = nullptr;
  manidsdp_params prm{};
  mds::BParams P{};
  char* data = nullptr;        // packed instance data (device)
  mds::BInst* inst = nullptr;  // device
  long long* y_off = nullptr;  // device
  double* y0 = nullptr;        // device, concatenated starting factors
  double* y_out = nullptr;     // device, concatenated multipliers
  mds::BOut* out = nullptr;    // device
  int* next = nullptr;         // device counter
  double* ws = nullptr;        // per-CTA workspaces
  long long ws_stride = 0;
  int ws_ctas = 0;             // CTAs the workspace holds
  int threads = 256, per_sm = 0;
  int occ[2] = {1, 1};         // occupancy limit at 128 and 256 threads
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {

using namespace mds;

void batch_release(manidsdp_batch* b) {
  void* ptrs[] = {b->data, b->inst, b->y_off, b->y0, b->y_out, b->out, b->next, b->ws};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  delete b;
}

int batch_grid(const manidsdp_batch* b) {
  const int occ = b->occ[b->threads == 128 ? 0 : 1];
  const int per_sm = b->per_sm > 0 ? std::min(b->per_sm, occ) : occ;
  return std::max(1, std::min({b->ninst, b->sms * per_sm, b->ws_ctas}));
}

// One launch over the whole batch; device time of the kernel in *ms.
int batch_launch(manidsdp_batch* b, float* ms) {
  MDS_CUDA(cudaMemsetAsync(b->next, 0, sizeof(int), b->s));
  MDS_CUDA(cudaEventRecord(b->e0, b->s));
  count_launches(1);
  kernel_for(b->threads)<<<batch_grid(b), b->threads, 0, b->s>>>(
      b->ninst, b->inst, b->data, b->y0, b->P, b->ws, b->ws_stride, b->nmax, b->mmax, b->next,
      b->out, b->y_out, b->y_off);
  MDS_CUDA(cudaGetLastError());
  MDS_CUDA(cudaEventRecord(b->e1, b->s));
  MDS_CUDA(cudaEventSynchronize(b->e1));
  float t = 0.f;
  MDS_CUDA(cudaEventElapsedTime(&t, b->e0, b->e1));
  if (ms) *ms = t;
  return MANIDSDP_OK;
}

bool batch_params_ok(const manidsdp_params& p) {
  return p.p0 >= 1 && p.p0 <= p.p_max && p.p_max <= kBMaxP && p.p_min >= 1 && p.delta_max >= 0 &&
         p.max_outer >= 0 && p.max_rtr >= 0 && p.max_tcg >= 1 && p.carry_halvings >= 0 &&
         (p.precision_mode == MANIDSDP_PREC_FP64 || p.precision_mode == MANIDSDP_PREC_MIXED) &&
         p.sigma0 > 0.0 && p.sigma_min > 0.0 && p.sigma_max >= p.sigma_min && p.gamma > 1.0 &&
         p.tol > 0.0;
}

int catch_all(const std::function<int()>& f) {
  try {
    return f();
  } catch (const DeviceError&) {
    return MANIDSDP_E_CUDA;
  } catch (const std::bad_alloc&) {
    return MANIDSDP_E_NOMEM;
  } catch (...) {
    return MANIDSDP_E_CUDA;
  }
}

}  // namespace

extern "C" {

int manidsdp_batch_setup(manidsdp_batch** out, int32_t ninst, const int32_t* Ns, const int64_t* ms,
                         const int32_t* idx_cat, const double* b_cat,
                         const manidsdp_params* params, void* stream) {
  if (out == nullptr || ninst < 1 || Ns == nullptr || ms == nullptr || idx_cat == nullptr ||
      b_cat == nullptr)
    return MANIDSDP_E_ARG;
  manidsdp_params prm;
  if (params) {
    prm = *params;
  } else {
    manidsdp_default_params(&prm);
    prm.p_max = kBMaxP;
  }
  if (!batch_params_ok(prm)) return MANIDSDP_E_ARG;
  // validate every instance and pack: index map, per-class upper-entry lists,
  // multiplicities and b, each 16-byte aligned in one buffer
  std::vector<char> host;
  std::vector<BInst> insts(ninst);
  std::vector<long long> y_off(ninst);
  auto put = [&](const void* src, size_t bytes) {
    const size_t off = align16(host.size());
    host.resize(off + bytes);
    std::memcpy(host.data() + off, src, bytes);
    return (long long)off;
  };
  int nmax = 0, mmax = 0;
  long long yo = 0, y0o = 0;
  size_t io = 0, bo = 0;
  for (int i = 0; i < ninst; ++i) {
    const int N = Ns[i];
    const int64_t m = ms[i];
    if (N < 1 || N > kBMaxN || m < 1 || m > int64_t(N) * N) return MANIDSDP_E_ARG;
    const int32_t* idx = idx_cat + io;
    const double* bb = b_cat + bo;
    io += size_t(N) * N;
    bo += size_t(m);
    std::vector<int32_t> cnt(m, 0), cptr(m + 1, 0);
    for (int r = 0; r < N; ++r)
      for (int c = 0; c < N; ++c) {
        const int32_t a = idx[size_t(r) * N + c];
        if (a < 0 || a >= m || a != idx[size_t(c) * N + r]) return MANIDSDP_E_ARG;
        ++cnt[a];
        if (r <= c) ++cptr[a + 1];
      }
    for (int64_t a = 0; a < m; ++a) {
      if (cnt[a] == 0) return MANIDSDP_E_ARG;  // A A* singular (Assumption 2)
      if (!std::isfinite(bb[a])) return MANIDSDP_E_NONFINITE;
      cptr[a + 1] += cptr[a];
    }
    std::vector<int32_t> cent(cptr[m]);
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int r = 0; r < N; ++r)
      for (int c = r; c < N; ++c) cent[fill[idx[size_t(r) * N + c]]++] = r * N + c;
    std::vector<double> cls(2 * m);
    for (int64_t a = 0; a < m; ++a) {
      cls[a] = double(cnt[a]);
      cls[m + a] = bb[a];
    }
    BInst& I = insts[i];
    I.N = N;
    I.m = int(m);
    I.off_idx = put(idx, size_t(N) * N * 4);
    I.off_cptr = put(cptr.data(), cptr.size() * 4);
    I.off_cent = put(cent.data(), cent.size() * 4);
    I.off_cls = put(cls.data(), cls.size() * 8);
    I.off_y0 = y0o;
    y0o += (long long)N * prm.p0;
    y_off[i] = yo;
    yo += m;
    nmax = std::max(nmax, N);
    mmax = std::max(mmax, int(m));
  }
  auto* b = new (std::nothrow) manidsdp_batch();
  if (b == nullptr) return MANIDSDP_E_NOMEM;
  b->ninst = ninst;
  b->nmax = nmax;
  b->mmax = mmax;
  b->y0_len = y0o;
  b->y_len = yo;
  b->s = static_cast<cudaStream_t>(stream);
  b->prm = prm;
  b->P = to_bparams(prm);
  const int st = catch_all([&]() -> int {
    int dev = 0;
    MDS_CUDA(cudaGetDevice(&dev));
    MDS_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    MDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ[0], kernel_for(128), 128, 0));
    MDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ[1], kernel_for(256), 256, 0));
    b->occ[0] = std::max(1, b->occ[0]);
    b->occ[1] = std::max(1, b->occ[1]);
    MDS_CUDA(cudaEventCreate(&b->e0));
    MDS_CUDA(cudaEventCreate(&b->e1));
    MDS_CUDA(cudaMalloc(&b->data, std::max<size_t>(host.size(), 16)));
    MDS_CUDA(cudaMemcpyAsync(b->data, host.data(), host.size(), cudaMemcpyHostToDevice, b->s));
    MDS_CUDA(cudaMalloc(&b->inst, ninst * sizeof(BInst)));
    MDS_CUDA(cudaMemcpyAsync(b->inst, insts.data(), ninst * sizeof(BInst), cudaMemcpyHostToDevice, b->s));
    MDS_CUDA(cudaMalloc(&b->y_off, ninst * sizeof(long long)));
    MDS_CUDA(cudaMemcpyAsync(b->y_off, y_off.data(), ninst * sizeof(long long), cudaMemcpyHostToDevice, b->s));
    MDS_CUDA(cudaMalloc(&b->y0, size_t(b->y0_len) * sizeof(double)));
    MDS_CUDA(cudaMalloc(&b->y_out, size_t(b->y_len) * sizeof(double)));
    MDS_CUDA(cudaMalloc(&b->out, ninst * sizeof(BOut)));
    MDS_CUDA(cudaMalloc(&b->next, sizeof(int)));
    // workspace for the largest grid any launch shape may use
    b->ws_ctas = std::min(ninst, b->sms * std::max(b->occ[0], b->occ[1]));
    b->ws_stride = make_layout(nmax, mmax).total;
    MDS_CUDA(cudaMalloc(&b->ws, size_t(b->ws_ctas) * b->ws_stride * sizeof(double)));
    MDS_CUDA(cudaStreamSynchronize(b->s));
    {  // a launch shape tuned earlier for this key
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tuned.find({nmax, prm.p_max, b->P.fp64});
      if (it != g_tuned.end()) {
        b->threads = it->second.first;
        b->per_sm = it->second.second;
      }
    }
    return MANIDSDP_OK;
  });
  if (st != MANIDSDP_OK) {
    batch_release(b);
    return st;
  }
  *out = b;
  return MANIDSDP_OK;
}

void manidsdp_batch_destroy(manidsdp_batch* b) {
  if (b) batch_release(b);
}

int manidsdp_batch_solve(manidsdp_batch* b, const double* Y0, manidsdp_batch_out* res, double* y,
                         float* ms) {
  if (b == nullptr || Y0 == nullptr) return MANIDSDP_E_ARG;
  static_assert(sizeof(manidsdp_batch_out) == sizeof(BOut), "result layout");
  return catch_all([&]() -> int {
    MDS_CUDA(cudaMemcpyAsync(b->y0, Y0, size_t(b->y0_len) * sizeof(double), cudaMemcpyDefault, b->s));
    float t = 0.f;
    batch_launch(b, &t);
    if (ms) *ms = t;
    std::vector<BOut> o(b->ninst);
    MDS_CUDA(cudaMemcpyAsync(o.data(), b->out, b->ninst * sizeof(BOut), cudaMemcpyDeviceToHost, b->s));
    if (y)
      MDS_CUDA(cudaMemcpyAsync(y, b->y_out, size_t(b->y_len) * sizeof(double), cudaMemcpyDefault, b->s));
    MDS_CUDA(cudaStreamSynchronize(b->s));
    if (res) std::memcpy(res, o.data(), b->ninst * sizeof(BOut));
    bool nonfinite = false, noconv = false;
    for (const BOut& r : o) {
      nonfinite |= r.status == MANIDSDP_E_NONFINITE;
      noconv |= r.status != MANIDSDP_OK;
    }
    return nonfinite ? MANIDSDP_E_NONFINITE : noconv ? MANIDSDP_E_NOCONV : MANIDSDP_OK;
  });
}

int manidsdp_batch_tune(manidsdp_batch* b, const double* Y0, int32_t* threads, int32_t* ctas_per_sm) {
  if (b == nullptr || Y0 == nullptr) return MANIDSDP_E_ARG;
  return catch_all([&]() -> int {
    MDS_CUDA(cudaMemcpyAsync(b->y0, Y0, size_t(b->y0_len) * sizeof(double), cudaMemcpyDefault, b->s));
    float best = INFINITY;
    int bt = b->threads, bs = b->per_sm;
    for (int th : {128, 256}) {
      const int occ = b->occ[th == 128 ? 0 : 1];
      for (int k = 1; k <= occ; k *= 2) {
        const int per = (k * 2 > occ && k < occ) ? occ : k;  // the last step is the limit itself
        b->threads = th;
        b->per_sm = per;
        float t = 0.f;
        batch_launch(b, &t);
        if (t < best) {
          best = t;
          bt = th;
          bs = per;
        }
        if (per == occ) break;
      }
    }
    b->threads = bt;
    b->per_sm = bs;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[{b->nmax, b->prm.p_max, b->P.fp64}] = {bt, bs};
    }
    if (threads) *threads = bt;
    if (ctas_per_sm) *ctas_per_sm = bs;
    return MANIDSDP_OK;
  });
}

int manidsdp_batch_set_launch(manidsdp_batch* b, int32_t threads, int32_t ctas_per_sm) {
  if (b == nullptr || (threads != 128 && threads != 256) || ctas_per_sm < 0) return MANIDSDP_E_ARG;
  b->threads = threads;
  b->per_sm = ctas_per_sm;
  return MANIDSDP_OK;
}

int manidsdp_solve_batched(int32_t ninst, const int32_t* N, const int64_t* m, const int32_t* idx,
                           const double* b, const double* Y0, const manidsdp_params* params,
                           manidsdp_batch_out* res, double* y, void* stream) {
  manidsdp_batch* bt = nullptr;
  const int st = manidsdp_batch_setup(&bt, ninst, N, m, idx, b, params, stream);
  if (st != MANIDSDP_OK) return st;
  const int r = manidsdp_batch_solve(bt, Y0, res, y, nullptr);
  manidsdp_batch_destroy(bt);
  return r;
}

}  // extern "C"

// Thousands of small instances in one persistent launch (manidsdp_batch_*):
// the host side (validation, packing, launch, tuner).
//
// Every CTA takes instances from a global counter, longest first (instances
// sorted by decreasing N, so the long ones do not finish last), and runs the
// whole of Algorithm 1 on each with the readings of the single-instance path and
// its oracle: RTR with truncated CG on the ALM subproblem (Section 4,
// Proposition 4.2), the multiplier update and certificate (Algorithm 1 steps
// 4-9), the rank update, the sigma rule (5.1), the rank-one rounding and the
// carried negative-curvature direction (Theorem 4.5).  Every decision is taken
// on the device; the host packs the instances and reads the results.
//
// Sizes: N <= 128 (moment matrices of the first-order relaxations with
// n <= 127 and of the second-order ones with n <= 14), factor width p <= 32.
// Cost, gradient, multiplier update and certificate are FP64; the tCG
// Hessian-vector products are FP32 from shared memory (MANIDSDP_PREC_MIXED) or
// FP64 (MANIDSDP_PREC_FP64).  The certificate's eigen-information comes from a
// Householder tridiagonalisation, Sturm-count multisection and inverse
// iteration (batched_dev.cuh).
//
// Instance data, packed into one device buffer: the N x N class map (int32 and
// uint16), per-class lists of the upper-triangle entries split into pieces of
// at most kBPiece entries (class sums in a fixed order, so results do not
// depend on the launch shape), multiplicities, b and 1/mult.  Per-CTA
// workspace in global memory, reused across the CTA's instances.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "batched.cuh"

namespace mds {
namespace batch {
namespace {

BParams to_bparams(const manidsdp_params& p) {
  BParams b{};
  b.sigma0 = p.sigma0; b.sigma_min = p.sigma_min; b.sigma_max = p.sigma_max; b.gamma = p.gamma;
  b.kappa1 = p.kappa1; b.kappa2 = p.kappa2; b.tol = p.tol; b.tol_grad_min = p.tol_grad_min;
  b.tol_grad_max = p.tol_grad_max; b.tol_grad_factor = p.tol_grad_factor; b.rank_tol = p.rank_tol;
  b.neg_tol = p.neg_tol; b.tcg_floor = p.tcg_floor; b.tcg_abs = p.tcg_abs; b.carry_t0 = p.carry_t0;
  b.round_eta = p.round_eta; b.sigma_stall = p.sigma_stall; b.p0 = p.p0; b.p_min = p.p_min; b.p_max = p.p_max;
  b.delta_max = p.delta_max; b.max_outer = p.max_outer; b.max_rtr = p.max_rtr;
  b.max_tcg = p.max_tcg; b.carry_halvings = p.carry_halvings;
  b.fp64 = p.precision_mode == MANIDSDP_PREC_FP64 ? 1 : 0;
  b.profile = p.profile ? 1 : 0;
  return b;
}

size_t align16(size_t x) { return (x + 15) / 16 * 16; }

KernelFn kernel_for(int threads) {
  return threads == 128 ? bt128::kernel() : threads == 256 ? bt256::kernel() : bt512::kernel();
}

unsigned smem_bytes(int threads, int N, int m, int np, int P4) {
  return threads == 128   ? bt128::smem_bytes(N, m, np, P4)
         : threads == 256 ? bt256::smem_bytes(N, m, np, P4)
                          : bt512::smem_bytes(N, m, np, P4);
}

constexpr int kShapes[3] = {128, 256, 512};  // threads per CTA the tuner tries
int shape_index(int threads) { return threads == 128 ? 0 : threads == 256 ? 1 : 2;
}

// Tuned launch shapes, shared by every batch of the process: key (N_max, p_max,
// precision) -> (threads per CTA, CTAs per SM).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tuned;

}  // namespace
}  // namespace batch
}  // namespace mds

struct manidsdp_batch {
  int ninst = 0, nmax = 0, mmax = 0, sms = 1;
  long long y0_len = 0, y_len = 0;
  cudaStream_t s = nullptr;
  manidsdp_params prm{};
  mds::batch::BParams P{};
  char* data = nullptr;        // packed instance data (device)
  mds::batch::BInst* inst = nullptr;  // device
  int* order = nullptr;        // device: instances by decreasing size (longest first)
  unsigned smem[3] = {0, 0, 0};  // dynamic shared memory at 128, 256 and 512 threads
  long long* y_off = nullptr;  // device
  double* y0 = nullptr;        // device, concatenated starting factors
  double* y_out = nullptr;     // device, concatenated multipliers
  mds::batch::BOut* out = nullptr;    // device
  int* next = nullptr;         // device counter
  double* ws = nullptr;        // per-CTA workspaces
  long long ws_stride = 0;
  int ws_ctas = 0;             // CTAs the workspace holds
  int threads = 256, per_sm = 0;
  int occ[3] = {1, 1, 1};      // occupancy limit at 128, 256 and 512 threads
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {

using namespace mds;
using namespace mds::batch;

void batch_release(manidsdp_batch* b) {
  void* ptrs[] = {b->data, b->inst, b->order, b->y_off, b->y0, b->y_out, b->out, b->next, b->ws};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  delete b;
}

int batch_grid(const manidsdp_batch* b) {
  const int occ = b->occ[shape_index(b->threads)];
  const int per_sm = b->per_sm > 0 ? std::min(b->per_sm, occ) : occ;
  return std::max(1, std::min({b->ninst, b->sms * per_sm, b->ws_ctas}));
}

// One launch over the whole batch; device time of the kernel in *ms.
int batch_launch(manidsdp_batch* b, float* ms) {
  MDS_CUDA(cudaMemsetAsync(b->next, 0, sizeof(int), b->s));
  MDS_CUDA(cudaEventRecord(b->e0, b->s));
  count_launches(1);
  kernel_for(b->threads)<<<batch_grid(b), b->threads, b->smem[shape_index(b->threads)], b->s>>>(
      b->ninst, b->inst, b->order, b->data, b->y0, b->P, b->ws, b->ws_stride, b->nmax, b->mmax,
      b->next, b->out, b->y_out, b->y_off);
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
         p.tol > 0.0 && p.direct == 0 && p.sigma_stall >= 0.0 && p.sigma_stall < 1.0;
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
  unsigned smem_need[3] = {0, 0, 0};
  const int P4 = (prm.p_max + 3) & ~3;
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
    std::vector<uint32_t> cent(cptr[m]);
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int r = 0; r < N; ++r)
      for (int c = r; c < N; ++c) cent[fill[idx[size_t(r) * N + c]]++] = (uint32_t(r) << 16) | uint32_t(c);
    std::vector<double> cls(3 * m);
    std::vector<float> invmf(m);
    for (int64_t a = 0; a < m; ++a) {
      cls[a] = double(cnt[a]);
      cls[m + a] = bb[a];
      cls[2 * m + a] = 1.0 / double(cnt[a]);
      invmf[a] = float(1.0 / double(cnt[a]));
    }
    BInst& I = insts[i];
    I.N = N;
    I.m = int(m);
    I.off_idx = put(idx, size_t(N) * N * 4);
    {
      std::vector<uint16_t> i16(size_t(N) * N);
      for (size_t t = 0; t < i16.size(); ++t) i16[t] = uint16_t(idx[t]);
      I.off_idx16 = put(i16.data(), i16.size() * 2);
    }
    I.off_cptr = put(cptr.data(), cptr.size() * 4);
    I.off_cent = put(cent.data(), cent.size() * 4);
    I.off_cls = put(cls.data(), cls.size() * 8);
    I.off_invmf = put(invmf.data(), invmf.size() * 4);
    // pieces of at most kBPiece entries, so that no thread sums a long class alone
    std::vector<int32_t> pstart, pcls, cpc(m + 1, 0);
    for (int64_t a = 0; a < m; ++a) {
      cpc[a] = int32_t(pstart.size());
      for (int32_t e = cptr[a]; e < cptr[a + 1]; e += kBPiece) {
        pstart.push_back(e);
        pcls.push_back(int32_t(a));
      }
    }
    cpc[m] = int32_t(pstart.size());
    pstart.push_back(cptr[m]);
    I.np = int(pcls.size());
    I.off_pstart = put(pstart.data(), pstart.size() * 4);
    I.off_pcls = put(pcls.data(), pcls.size() * 4);
    I.off_cpc = put(cpc.data(), cpc.size() * 4);
    I.off_y0 = y0o;
    y0o += (long long)N * prm.p0;
    y_off[i] = yo;
    yo += m;
    nmax = std::max(nmax, N);
    mmax = std::max(mmax, int(m));
    if (prm.precision_mode == MANIDSDP_PREC_MIXED)
      for (int t = 0; t < 3; ++t) smem_need[t] = std::max(smem_need[t], smem_bytes(kShapes[t], N, int(m), I.np, P4));
  }
  // longest first: instances by decreasing N (then decreasing m), ties by number
  std::vector<int> order(ninst);
  for (int i = 0; i < ninst; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return insts[a].N != insts[c].N ? insts[a].N > insts[c].N : insts[a].m > insts[c].m;
  });
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
    int smem_max = 0;
    MDS_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    for (int t = 0; t < 3; ++t) {
      b->smem[t] = smem_need[t];
      if (int(smem_need[t]) > smem_max) throw std::bad_alloc();
      MDS_CUDA(cudaFuncSetAttribute(kernel_for(kShapes[t]), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(smem_need[t])));
    }
    for (int t = 0; t < 3; ++t) {
      MDS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->occ[t], kernel_for(kShapes[t]), kShapes[t],
                                                             b->smem[t]));
      b->occ[t] = std::max(1, b->occ[t]);
    }
    MDS_CUDA(cudaEventCreate(&b->e0));
    MDS_CUDA(cudaEventCreate(&b->e1));
    MDS_CUDA(cudaMalloc(&b->data, std::max<size_t>(host.size(), 16)));
    MDS_CUDA(cudaMemcpyAsync(b->data, host.data(), host.size(), cudaMemcpyHostToDevice, b->s));
    MDS_CUDA(cudaMalloc(&b->inst, ninst * sizeof(BInst)));
    MDS_CUDA(cudaMemcpyAsync(b->inst, insts.data(), ninst * sizeof(BInst), cudaMemcpyHostToDevice, b->s));
    MDS_CUDA(cudaMalloc(&b->order, ninst * sizeof(int)));
    MDS_CUDA(cudaMemcpyAsync(b->order, order.data(), ninst * sizeof(int), cudaMemcpyHostToDevice, b->s));
    MDS_CUDA(cudaMalloc(&b->y_off, ninst * sizeof(long long)));
    MDS_CUDA(cudaMemcpyAsync(b->y_off, y_off.data(), ninst * sizeof(long long), cudaMemcpyHostToDevice, b->s));
    MDS_CUDA(cudaMalloc(&b->y0, size_t(b->y0_len) * sizeof(double)));
    MDS_CUDA(cudaMalloc(&b->y_out, size_t(b->y_len) * sizeof(double)));
    MDS_CUDA(cudaMalloc(&b->out, ninst * sizeof(BOut)));
    MDS_CUDA(cudaMalloc(&b->next, sizeof(int)));
    // workspace for the largest grid any launch shape may use
    b->ws_ctas = std::min(ninst, b->sms * std::max({b->occ[0], b->occ[1], b->occ[2]}));
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
    for (int th : kShapes) {
      const int occ = b->occ[shape_index(th)];
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
  if (b == nullptr || (threads != 128 && threads != 256 && threads != 512) || ctas_per_sm < 0)
    return MANIDSDP_E_ARG;
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

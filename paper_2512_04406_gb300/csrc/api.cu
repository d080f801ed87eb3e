// C ABI of the ManiDSDP hot path: context set-up, subproblem evaluation, the
// Riemannian Hessian-vector product, Lanczos on the certificate, and
// Algorithm 1 (ALM outer loop around Riemannian trust region with truncated CG).
// The host here only sequences kernels and takes the scalar decisions (tCG step
// sizes when the loop is host-driven, trust-region ratio, sigma rule, rank
// update); every vector and matrix operation runs in the kernels: kernels_seg.cu
// and kernels_dense.cu (FP64 form), kernels_df64.cu (df64 evaluation),
// kernels_sddmm.cu, kernels_gemm32.cu and kernels_tcx.cu (FP32 Hessian-vector
// product), kernels_tcg.cu (device-driven truncated CG).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <functional>
#include <new>
#include <stdexcept>

#include "common.cuh"
#include "host_linalg.h"
#include "complex1.h"

using namespace mds;
using namespace mds::hostla;

#include <atomic>
namespace mds {
static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_now() { return g_launches.load(); }
void uncount_launches(long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
}  // namespace mds

namespace {

// splitmix64 (Steele, Lea, Flood 2014): the start vector of Lanczos.
uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

struct manidsdp_ctx {
  mds::ComplexState* cx = nullptr;  // the first-order complex relaxation (setup_ex)
  int N = 0;
  int64_t m = 0;
  int c_kind = 0;
  manidsdp_params prm{};
  cudaStream_t s = nullptr;
  std::vector<void*> allocs;
  // problem data
  int32_t* idx = nullptr;
  double *mult = nullptr, *b = nullptr, *bm = nullptr, *C = nullptr;
  double normb = 0.0, normC = 0.0;
  ClassMap cm;
  // ALM state and N x N work
  double *XD = nullptr, *G = nullptr, *Gt = nullptr;
  float *Gf = nullptr, *Gtf = nullptr;
  // df64 halves of G (mixed mode): Gh doubles as the FP32 G of the Hess-vec
  float *Gh = nullptr, *Gl = nullptr, *Gth = nullptr, *Gtl = nullptr;
  float *Yh = nullptr, *Yl = nullptr;
  // per class; slot[r*N + c] (r <= c): position of entry (r, c) in the inverse map
  double *y = nullptr, *yt = nullptr, *w = nullptr, *piece_buf = nullptr;
  double* y_prev = nullptr;  // direct formulation: y of the previous outer iteration
  int32_t* slot = nullptr;
  float* perm = nullptr;
  double* permd = nullptr;  // class-ordered FP64 values (df64 evaluation)
  double* Sup = nullptr;    // S = Y Y' by upper tiles (df64 evaluation)
  float* wf = nullptr;
  // N x pcap
  int pcap = 0;
  double *Y = nullptr, *Yt = nullptr, *GY = nullptr, *grad = nullptr, *eta = nullptr,
         *Heta = nullptr, *r = nullptr, *delta = nullptr, *Hd = nullptr, *Up = nullptr,
         *Tm = nullptr, *YM = nullptr, *U = nullptr, *tmp = nullptr, *Vn = nullptr;
  float *Yf = nullptr, *Upf = nullptr, *Tmf = nullptr, *YMf = nullptr;
  double *z = nullptr, *zt = nullptr;
  double *M1 = nullptr, *M2 = nullptr;
  float *M1f = nullptr, *M2f = nullptr;
  double *part = nullptr, *out2 = nullptr, *dpart = nullptr;
  void* gws = nullptr;
  size_t gws_bytes = 0;
  void* gws2 = nullptr;  // Gram partials (separate from the GEMM partials they coexist with)
  size_t gws2_bytes = 0;
  // Lanczos
  int kmax = 0;
  double *LV = nullptr, *lh = nullptr, *lw = nullptr, *ls = nullptr;
  double* hp = nullptr;  // pinned host scalars
  // state
  double sigma = 1.0, xdc = 0.0;
  bool yf_valid = false;
  const double* eval_user_Y = nullptr;
  int eval_p = 0;
  bool eval_ok = false;
  double psi = 0.0, r2 = 0.0;
  // state kept for a warm-started (resumed) solve
  bool resume_valid = false;
  int resume_p = 0;
  double resume_rscale = -1.0;
  int resume_outer = 0;
  int* tc_err = nullptr;  // set by a tensor-core kernel whose device-side wait timed out
  // TMA tensor-core engine of the FP32 Hess-vec: its operands as TF32 pairs
  float *Ghi = nullptr, *Glo = nullptr, *QWhi = nullptr, *QWlo = nullptr;  // N x ldg
  float *Yxh = nullptr, *Yxl = nullptr, *Uxh = nullptr, *Uxl = nullptr;    // N x ld(p)
  float *YTh = nullptr, *YTl = nullptr, *UTh = nullptr, *UTl = nullptr;    // p x ldg
  float* Wfull = nullptr;  // W = Y Up' + Up Y' at every entry (N x ldg)
  int tc_pairs = 1;        // 1: TF32 pairs (three products); 0: single TF32 products
  double* lz_prev = nullptr;  // the last certificate's lambda_min Ritz vector (N)
  double* lz_lock = nullptr;  // a vector held out of a Lanczos run (N)
  bool lz_prev_ok = false;
  int2* tiles = nullptr;  // upper-triangle 128 x 128 tile pairs of the SDDMM
  int ntiles = 0;
  bool resume_have_U = false;  // the last iteration augmented Y = [Y, 0] and set U = [0, V]
  int resume_U_cols = 0;
  // counters and phase timers
  int hessvecs = 0, rtr_iters = 0, lanczos_mv = 0, evals = 0, grads = 0;
  double hv_psum = 0.0;
  double ms_hv = 0.0, ms_eval = 0.0, ms_grad = 0.0, ms_lz = 0.0, ms_rank = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // per-stage Hess-vec timing (params.profile == 2, host-driven path)
  cudaEvent_t sev[8] = {};
  double stage_ms[8] = {};
  // device-driven tCG: state, partial sums, capture stream and cached graphs
  void* tcgst = nullptr;
  double *kpart = nullptr, *rpart = nullptr;
  cudaStream_t cs = nullptr;
  // side stream of the FP32 Hess-vec: U'Y and the Y(U'Y) + U(Y'Y) slice run on it
  // while the class sums and the gather GEMM run on the main (or capture) stream
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  struct Graph {
    int p, prec, pairs;
    double sigma;
    const void *Y, *G;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    long long body_launches;
  };
  std::vector<Graph> graphs;
};

namespace {

template <typename T>
T* dalloc(manidsdp_ctx* c, size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) throw std::bad_alloc();
  c->allocs.push_back(p);
  return static_cast<T*>(p);
}

void sync(manidsdp_ctx* c) { MDS_CUDA(cudaStreamSynchronize(c->s)); }

// Phase timing with CUDA events on the context's stream (params.profile).
void tstart(manidsdp_ctx* c) {
  if (c->prm.profile) MDS_CUDA(cudaEventRecord(c->ev0, c->s));
}
void tstop(manidsdp_ctx* c, double* acc) {
  if (!c->prm.profile) return;
  MDS_CUDA(cudaEventRecord(c->ev1, c->s));
  MDS_CUDA(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  MDS_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  *acc += double(ms);
}

// Deterministic dot products of up to three pairs of length n; results on the host.
void dots(manidsdp_ctx* c, size_t n, int k, const double* x0, const double* y0, double* out,
          const double* x1 = nullptr, const double* y1 = nullptr, const double* x2 = nullptr,
          const double* y2 = nullptr) {
  const double* xs[3] = {x0, x1, x2};
  const double* ys[3] = {y0, y1, y2};
  launch_dots(n, k, xs, ys, c->dpart, c->s);
  MDS_CUDA(cudaMemcpyAsync(c->hp, c->dpart + 3 * kRedBlocks, k * sizeof(double),
                           cudaMemcpyDeviceToHost, c->s));
  sync(c);
  for (int i = 0; i < k; ++i) out[i] = c->hp[i];
}

bool mixed(const manidsdp_ctx* c) { return c->prm.precision_mode == MANIDSDP_PREC_MIXED; }
// The FP32 copy of G read by the mixed-precision Hess-vec.
float* g32(manidsdp_ctx* c) { return mixed(c) ? c->Gh : c->Gf; }

// T = G U - sigma A*(w) Y of the FP32 Hessian-vector product as split-K partial
// products in c->gws (tensor cores or FP32 FMA); returns the number of splits.
// The tensor-core engine of the FP32 Hess-vec (kernels_tcx.cu): TMA-fed tcgen05
// SDDMM, Gram products and gather GEMM.
bool use_tcx(const manidsdp_ctx* c) { return c->prm.tensor_cores == 1; }

// Buffers of the tensor-core engine, allocated on first use (outside any capture).
void ensure_tcx(manidsdp_ctx* c) {
  if (c->Ghi != nullptr) return;
  const int N = c->N, ldg = tcx_ld(N), ldp = tcx_ld(c->pcap);
  const size_t nn = size_t(N) * ldg, np = size_t(N) * ldp, pn = size_t(c->pcap) * ldg;
  c->Ghi = dalloc<float>(c, nn);
  c->Glo = dalloc<float>(c, nn);
  c->QWhi = dalloc<float>(c, nn);
  c->QWlo = dalloc<float>(c, nn);
  c->Wfull = dalloc<float>(c, nn);
  float** rows[] = {&c->Yxh, &c->Yxl, &c->Uxh, &c->Uxl};
  for (float** q : rows) *q = dalloc<float>(c, np);
  float** cols[] = {&c->YTh, &c->YTl, &c->UTh, &c->UTl};
  for (float** q : cols) *q = dalloc<float>(c, pn);
  const std::vector<int2> t = tcx_upper_tiles(N);
  c->ntiles = int(t.size());
  c->tiles = dalloc<int2>(c, t.size());
  MDS_CUDA(cudaMemcpyAsync(c->tiles, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice, c->s));
}

// The current point for the tensor-core engine: G (from its FP32 copy) and Y as
// TF32 pairs, Y also transposed.
void tcx_point(manidsdp_ctx* c, const double* Y, int p, cudaStream_t s) {
  ensure_tcx(c);
  const int N = c->N, ldg = tcx_ld(N), ldp = tcx_ld(p);
  launch_tcx_split_matrix(N, g32(c), nullptr, nullptr, 0.f, c->Ghi, c->Glo, ldg, s);
  launch_tcx_split_rows(N, p, Y, c->Yxh, c->Yxl, ldp, c->YTh, c->YTl, ldg, s);
}

// Tensor-core Hess-vec body after the prologue (Up in FP64): Up as TF32 pairs, the
// SDDMM (class sums w and the full W), sigma Q(W) = sigma (W - A*(w)) as pairs and
// the gather GEMM G Up + sigma Q(W) Y.  Returns the number of split-K slices minus
// one: the epilogue adds the last slice where the FMA engine has its separate
// Y(U'Y) + U(Y'Y) slice.
int hessvec_tcx(manidsdp_ctx* c, int p, cudaStream_t s, const std::function<void(int)>& mark) {
  const int N = c->N, ldg = tcx_ld(N), ldp = tcx_ld(p);
  launch_tcx_split_rows(N, p, c->Up, c->Uxh, c->Uxl, ldp, c->UTh, c->UTl, ldg, s);
  if (mark) mark(1);
  launch_tcx_sddmm(N, p, c->Yxh, c->Yxl, c->Uxh, c->Uxl, ldp, c->slot, c->perm, c->Wfull, ldg,
                   c->tiles, c->ntiles, c->tc_err, s, c->tc_pairs);
  if (c->prm.direct)  // direct formulation: no class-mean term
    MDS_CUDA(cudaMemsetAsync(c->wf, 0, size_t(c->m) * sizeof(float), s));
  else
    launch_piece_sums(c->cm, c->perm, c->mult, reinterpret_cast<float*>(c->piece_buf), c->wf, s);
  if (mark) mark(2);
  launch_tcx_split_matrix(N, c->Wfull, c->idx, c->wf, float(c->sigma), c->QWhi, c->QWlo, ldg, s);
  const int S = launch_tcx_gather(N, p, c->Ghi, c->Glo, c->QWhi, c->QWlo, ldg, c->UTh, c->UTl,
                                  c->YTh, c->YTl, ldg, static_cast<float*>(c->gws), c->gws_bytes,
                                  c->tc_err, s, c->tc_pairs);
  if (mark) {
    mark(3);
    mark(4);
  }
  return S - 1;
}

// w = A(Y Up' + Up Y') / mult in FP32 on the FMA engine (tiled SDDMM into the
// class-ordered buffer, per-piece sums).
void class_sums32(manidsdp_ctx* c, int p, cudaStream_t s) {
  if (c->prm.direct) {  // direct formulation: no class-mean term
    MDS_CUDA(cudaMemsetAsync(c->wf, 0, size_t(c->m) * sizeof(float), s));
    return;
  }
  float* pbf = reinterpret_cast<float*>(c->piece_buf);
  launch_sddmm_means(c->cm, c->N, p, c->Yf, c->Upf, c->slot, c->perm, c->mult, pbf, c->wf, s);
}

// T = G U - sigma A*(w) Y of the FP32 Hessian-vector product on the FMA engine as
// split-K partial products in c->gws; returns the number of splits.
int gather_gemm32(manidsdp_ctx* c, int p, cudaStream_t s) {
  return launch_gemm32_partials(c->N, p, g32(c), c->Upf, c->idx, c->wf, float(-c->sigma), c->Yf,
                                c->gws, c->gws_bytes, s);
}

void drop_graphs(manidsdp_ctx* c);

int gather_gemm32_splits(manidsdp_ctx* c, int p) {
  if (use_tcx(c)) return tcx_gather_splits(c->N) - 1;
  return gemm32_splits(c->N, p, c->gws_bytes);
}

// The FP32 Hess-vec after its prologue (Upf, Yf, Y'Y in place) up to the
// split-K partials in c->gws.  FMA engine: class sums and gather GEMM on s; U'Y
// and the Y(U'Y) + U(Y'Y) slice on the side stream when fork is set (joined
// before return), else on s after the GEMM.  Returns the number of GEMM splits.
int hessvec32_body(manidsdp_ctx* c, int p, cudaStream_t s, bool fork) {
  if (use_tcx(c)) return hessvec_tcx(c, p, s, nullptr);
  const int N = c->N;
  const int splits = gather_gemm32_splits(c, p);
  float* ym_out = static_cast<float*>(c->gws) + size_t(splits) * N * p;
  if (fork) {
    MDS_CUDA(cudaEventRecord(c->ev_fork, s));
    MDS_CUDA(cudaStreamWaitEvent(c->s2, c->ev_fork, 0));
    launch_gram2<float>(N, p, c->Upf, nullptr, c->Yf, c->M1f, c->gws2, c->gws2_bytes, c->s2);
    launch_ym32(N, p, c->Yf, c->Upf, c->M1f, float(c->sigma), ym_out, c->s2);
    MDS_CUDA(cudaEventRecord(c->ev_join, c->s2));
  }
  class_sums32(c, p, s);
  if (gather_gemm32(c, p, s) != splits) throw DeviceError{cudaErrorInvalidValue};
  if (fork) {
    MDS_CUDA(cudaStreamWaitEvent(s, c->ev_join, 0));
  } else {
    launch_gram2<float>(N, p, c->Upf, nullptr, c->Yf, c->M1f, c->gws2, c->gws2_bytes, s);
    launch_ym32(N, p, c->Yf, c->Upf, c->M1f, float(c->sigma), ym_out, s);
  }
  return splits;
}

// MANIDSDP_E_TIMEOUT when a tensor-core kernel reported an expired wait (the
// flag is cleared); synchronises the context's stream.
int take_device_error(manidsdp_ctx* c) {
  int e = 0;
  MDS_CUDA(cudaMemcpyAsync(&e, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  MDS_CUDA(cudaStreamSynchronize(c->s));
  if (e == 0) return MANIDSDP_OK;
  MDS_CUDA(cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->s));
  return MANIDSDP_E_TIMEOUT;
}

// Psi, y and G at Y.  FP64 mode: native FP64, G (and Gf = float(G) when given).
// Mixed mode: df64 on the FP32 pipe, G as the float pair (Gh, Gl) and, when
// given, also in FP64.
void evaluate(manidsdp_ctx* c, const double* Y, int p, double* y, double* G, float* Gf,
              double* psi, double* r2, float* Gh = nullptr, float* Gl = nullptr) {
  tstart(c);
  c->evals++;
  if (mixed(c) && Gh != nullptr) {
    launch_split(size_t(c->N) * p, Y, c->Yh, c->Yl, c->s);
    launch_spass_df(c->cm, c->N, p, c->Yh, c->Yl, c->C, c->slot, c->Sup, c->permd, c->mult,
                    c->piece_buf, y, c->s);
    launch_gpass_df(c->N, p, 0, c->Yh, c->Yl, c->idx, c->prm.direct ? c->y_prev : y, c->C,
                    c->sigma, c->XD, G, Gh, Gl,
                    c->part, c->out2, c->s, c->Sup);
  } else {
    launch_class_means<double>(c->cm, c->N, p, 0, Y, nullptr, c->C, c->mult, c->piece_buf, y,
                               c->s);
    launch_gpass(c->N, p, 0, Y, c->idx, c->prm.direct ? c->y_prev : y, c->C, c->sigma, c->XD, G,
                 Gf, c->part, c->out2, c->s);
  }
  MDS_CUDA(cudaMemcpyAsync(c->hp, c->out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  tstop(c, &c->ms_eval);
  sync(c);
  *r2 = c->hp[0];
  *psi = c->hp[1] + c->xdc + 0.5 * c->sigma * c->hp[0];
}

// GY = G Y, z = diag(G S), grad = 2 (GY - Diag(z) Y); returns ||grad||.
double gradient(manidsdp_ctx* c, const double* Y, int p, const double* G,
                const float* Gh = nullptr, const float* Gl = nullptr) {
  const int N = c->N;
  tstart(c);
  c->grads++;
  if (Gh != nullptr) {
    launch_split(size_t(N) * p, Y, c->Yh, c->Yl, c->s);
    launch_gemm_df(N, p, Gh, Gl, c->Yh, c->Yl, c->GY, c->gws, c->gws_bytes, c->s);
  } else {
    launch_gemm<double>(N, p, N, G, N, Y, p, c->GY, p, 1.0, 0.0, nullptr, nullptr, 0.0, nullptr,
                        c->gws, c->gws_bytes, c->s);
  }
  launch_rowdot(N, p, c->GY, Y, c->z, c->s);
  launch_grad_from_gy(N, p, c->GY, c->z, Y, c->grad, c->s);
  tstop(c, &c->ms_grad);
  double gg;
  dots(c, size_t(N) * p, 1, c->grad, c->grad, &gg);
  return std::sqrt(gg);
}

// HU = Hess Psi(Y)[P_Y(U)] using G, Gf and z of the last evaluation at Y:
// prologue (projection, FP32 copies), class means w, split-K gather GEMM
// G U - sigma A*(w) Y, the Gram pair [U'Y; Y'Y], then the row epilogue.
void hessvec(manidsdp_ctx* c, const double* Y, const double* U, int p, double* HU, int prec) {
  const int N = c->N;
  const bool stages = c->prm.profile >= 2;
  auto mark = [&](int i) {
    if (stages) MDS_CUDA(cudaEventRecord(c->sev[i], c->s));
  };
  tstart(c);
  mark(0);
  if (prec == MANIDSDP_PREC_FP64) {
    launch_hv_prep<double>(N, p, Y, U, c->Up, nullptr, nullptr, false, c->s);
    mark(1);
    if (c->prm.direct)  // direct formulation: no class-mean term (sigma I in place of sigma Q)
      MDS_CUDA(cudaMemsetAsync(c->w, 0, size_t(c->m) * sizeof(double), c->s));
    else
      launch_class_means<double>(c->cm, N, p, 1, Y, c->Up, nullptr, c->mult, c->piece_buf, c->w,
                                 c->s);
    mark(2);
    const int splits = launch_gemm_partials<double>(N, p, N, c->G, N, c->Up, p, c->idx, c->w,
                                                    -c->sigma, Y, c->gws, c->gws_bytes, c->s);
    mark(3);
    launch_gram2<double>(N, p, c->Up, Y, Y, c->M1, c->gws2, c->gws2_bytes, c->s);
    mark(4);
    launch_hv_epilogue<double>(N, p, splits, static_cast<const double*>(c->gws), c->M1, Y, c->Up,
                               c->z, c->sigma, HU, c->s);
  } else {
    const bool fresh = !c->yf_valid;
    launch_hv_prep<float>(N, p, Y, U, c->Up, c->Upf, c->Yf, fresh, c->s);
    c->yf_valid = true;
    if (fresh) {  // Y'Y depends on Y only: second p x p slot of M1f
      launch_gram2<float>(N, p, c->Yf, nullptr, c->Yf, c->M1f + size_t(p) * p, c->gws2,
                          c->gws2_bytes, c->s);
      if (use_tcx(c)) tcx_point(c, Y, p, c->s);
    }
    if (!(stages && use_tcx(c))) mark(1);
    int splits;
    if (stages && use_tcx(c)) {  // Gram products in stage 0, the Q(W) Y term in stage 2
      splits = hessvec_tcx(c, p, c->s, mark);
    } else if (stages) {  // serial, with the stage events between the steps
      class_sums32(c, p, c->s);
      mark(2);
      splits = gather_gemm32(c, p, c->s);
      mark(3);
      launch_gram2<float>(N, p, c->Upf, nullptr, c->Yf, c->M1f, c->gws2, c->gws2_bytes, c->s);
      launch_ym32(N, p, c->Yf, c->Upf, c->M1f, float(c->sigma),
                  static_cast<float*>(c->gws) + size_t(splits) * N * p, c->s);
      mark(4);
    } else {
      splits = hessvec32_body(c, p, c->s, true);
    }
    launch_hv_epilogue<float>(N, p, splits, static_cast<const float*>(c->gws), nullptr, Y, c->Up,
                              c->z, c->sigma, HU, c->s);
  }
  mark(5);
  if (stages) {
    MDS_CUDA(cudaEventSynchronize(c->sev[5]));
    for (int i = 0; i < 5; ++i) {
      float ms = 0.f;
      MDS_CUDA(cudaEventElapsedTime(&ms, c->sev[i], c->sev[i + 1]));
      c->stage_ms[i] += ms;
    }
  }
  tstop(c, &c->ms_hv);
  c->hessvecs++;
  c->hv_psum += p;
}

struct LanczosOut {
  std::vector<double> lo;  // smallest Ritz values (ascending), those returned
  double hi = 0.0;
  int steps = 0;
  // the smallest Ritz pair met the residual test (or the Krylov space became
  // invariant): lo[0] is lambda_min to rounding; false after k steps without it,
  // when lo[0] is only an upper bound of lambda_min
  bool converged = false;
  int nvec = 0;  // Ritz vectors written to c->Vn (N x nvec, row-major)
};

// Lanczos with full reorthogonalisation on X = XD - Diag(z) (z on device).
// warm (device N, may be NULL): a previous eigenvector estimate mixed into the
// start vector (start = warm + 0.1 r, r the fixed splitmix64 vector, normalised),
// so that a Krylov space of the slightly changed certificate still holds every
// eigendirection while it starts next to the one sought.
// lock (device N, unit norm, may be NULL): a known eigenvector kept out of the
// Krylov space (it sits in front of the basis, so reorthogonalisation removes
// it), e.g. the exact null vector Yr/sqrt(N) of a rank-one point's certificate;
// the Ritz values are then those of X on its orthogonal complement.
LanczosOut lanczos(manidsdp_ctx* c, const double* z, int kcap, int n_small,
                   bool want_vecs = true, const double* warm = nullptr,
                   const double* lock = nullptr) {
  const int N = c->N;
  double t_lz = 0.0;
  if (c->prm.profile) {
    sync(c);
    t_lz = -1.0;
  }
  const auto wall0 = std::chrono::steady_clock::now();
  int k = std::min(std::min(kcap, c->kmax), N);
  if (k < 1) k = 1;
  std::vector<double> v0(N);
  double nrm = 0.0;
  for (int i = 0; i < N; ++i) {
    const uint64_t u = splitmix64(0x5EEDull + uint64_t(i));
    v0[i] = (double(u >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
    nrm += v0[i] * v0[i];
  }
  nrm = std::sqrt(nrm);
  for (int i = 0; i < N; ++i) v0[i] /= nrm;
  const int off = lock != nullptr ? 1 : 0;
  double* KV = c->LV + size_t(off) * N;  // the Krylov vectors
  if (lock != nullptr)
    MDS_CUDA(cudaMemcpyAsync(c->LV, lock, N * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  MDS_CUDA(cudaMemcpyAsync(KV, v0.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->s));
  if (warm != nullptr) launch_axpby(N, 1.0, warm, 0.1, KV, KV, c->s);
  if (lock != nullptr) {
    double d;
    dots(c, N, 1, c->LV, KV, &d);
    launch_axpby(N, -d, c->LV, 1.0, KV, KV, c->s);
  }
  if (warm != nullptr || lock != nullptr) {
    double nn;
    dots(c, N, 1, KV, KV, &nn);
    launch_axpby(N, 1.0 / std::sqrt(nn), KV, 0.0, nullptr, KV, c->s);
  }
  std::vector<double> al, be;
  int steps = k;
  double res_lo = 0.0;
  bool conv = false;
  for (int j = 0; j < k; ++j) {
    const double* vj = KV + size_t(j) * N;
    launch_gemv_cert(N, c->XD, z, vj, c->lw, c->s);
    c->lanczos_mv++;
    launch_basis_dots(N, off + j + 1, c->LV, c->lw, c->lh, c->s);
    MDS_CUDA(cudaMemcpyAsync(c->hp + 8, c->lh + off + j, sizeof(double), cudaMemcpyDeviceToHost,
                             c->s));
    launch_basis_update(N, off + j + 1, c->LV, c->lh, c->lw, c->s);
    launch_basis_dots(N, off + j + 1, c->LV, c->lw, c->lh, c->s);
    launch_basis_update(N, off + j + 1, c->LV, c->lh, c->lw, c->s);
    double bb;
    dots(c, N, 1, c->lw, c->lw, &bb);  // synchronises; hp[8] now holds alpha_j
    const double alpha = c->hp[8];
    const double beta = std::sqrt(bb);
    al.push_back(alpha);
    if (beta <= 1e-14 * std::max(1.0, std::fabs(alpha)) || j == k - 1) {
      steps = j + 1;
      conv = beta <= 1e-14 * std::max(1.0, std::fabs(alpha)) || j + 1 == N;
      break;
    }
    be.push_back(beta);
    launch_axpby(N, 1.0 / beta, c->lw, 0.0, nullptr, KV + size_t(j + 1) * N, c->s);
    // convergence of the extreme Ritz pairs every 10 steps
    if ((j + 1) % 10 == 0) {
      const int kk = j + 1;
      const double tlo = tridiag_eig(al, be, kk, 0);
      const double thi = tridiag_eig(al, be, kk, kk - 1);
      const auto slo = tridiag_vec(al, be, kk, tlo, {});
      const auto shi = tridiag_vec(al, be, kk, thi, {});
      const double scale = std::max(std::fabs(tlo), std::fabs(thi)) + 1e-300;
      res_lo = beta * std::fabs(slo[kk - 1]);
      const double res_hi = beta * std::fabs(shi[kk - 1]);
      if (res_lo <= 1e-10 * scale && res_hi <= 1e-6 * scale) {
        steps = kk;
        conv = true;
        break;
      }
    }
  }
  LanczosOut out;
  out.steps = steps;
  out.converged = conv;
  const int kk = steps;
  std::vector<double> bt(be.begin(), be.begin() + std::max(0, kk - 1));
  std::vector<double> at(al.begin(), al.begin() + kk);
  out.hi = tridiag_eig(at, bt, kk, kk - 1);
  const int ns = std::min(std::min(n_small, kk), c->pcap);
  std::vector<std::vector<double>> svecs;
  for (int i = 0; i < ns; ++i) {
    const double th = tridiag_eig(at, bt, kk, i);
    out.lo.push_back(th);
    svecs.push_back(tridiag_vec(at, bt, kk, th, svecs));
  }
  // Ritz vectors into Vn (row-major N x ns): column i = sum_j s_i[j] v_j
  std::vector<double> neg(kk);
  for (int i = 0; i < (want_vecs ? ns : 0); ++i) {
    for (int j = 0; j < kk; ++j) neg[j] = -svecs[i][j];
    MDS_CUDA(cudaMemcpyAsync(c->lh, neg.data(), kk * sizeof(double), cudaMemcpyHostToDevice, c->s));
    MDS_CUDA(cudaMemsetAsync(c->lw, 0, N * sizeof(double), c->s));
    launch_basis_update(N, kk, KV, c->lh, c->lw, c->s);
    // sign: first nonzero entry positive
    MDS_CUDA(cudaMemcpyAsync(c->ls, c->lw, N * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
    std::vector<double> hv(N);
    MDS_CUDA(cudaMemcpyAsync(hv.data(), c->lw, N * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    sync(c);
    double sgn = 1.0;
    for (int t = 0; t < N; ++t)
      if (std::fabs(hv[t]) > 1e-14) {
        sgn = hv[t] < 0 ? -1.0 : 1.0;
        break;
      }
    launch_axpby(N, sgn, c->lw, 0.0, nullptr, c->ls, c->s);
    launch_set_cols(N, ns, i, 1, c->ls, c->Vn, c->s);
  }
  out.nvec = want_vecs ? ns : 0;
  sync(c);
  if (t_lz < 0.0)
    c->ms_lz += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
  return out;
}

void default_params(manidsdp_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->sigma0 = 1.0;
  p->sigma_min = 1e-3;
  p->sigma_max = 1e6;
  p->gamma = 2.0;
  p->kappa1 = 0.1;
  p->kappa2 = 10.0;
  p->tol = 1e-8;
  p->tol_grad_min = 1e-11;
  p->tol_grad_max = 1e-2;
  p->tol_grad_factor = 1.0;
  p->rank_tol = 1e-6;
  p->neg_tol = 1e-10;
  p->tcg_floor = 1e-10;
  p->tcg_abs = 0.1;
  p->carry_t0 = 0.0;
  p->round_eta = 1e-2;
  p->tc_lowprec_eta = 0.0;
  p->warm_start = 0;
  p->p0 = 2;
  p->p_min = 2;
  p->p_max = 512;
  p->delta_max = 16;
  p->max_outer = 300;
  p->max_rtr = 15;
  p->max_tcg = 60;
  p->carry_halvings = 30;
  p->lanczos_k = 2000;
  p->precision_mode = MANIDSDP_PREC_FP64;
  p->verbose = 0;
  p->profile = 0;
  p->tcg_device = 1;
  p->tensor_cores = 0;
  p->direct = 0;
  p->sigma_stall = 0.5;
}

// Ranges of the parameters (the switches are 0 or 1).
bool params_ok(const manidsdp_params& p) {
  auto flag = [](int32_t v) { return v == 0 || v == 1; };
  return p.p_max >= 1 && p.p_max <= kMaxP && p.p0 >= 1 && p.p0 <= p.p_max && p.p_min >= 1 &&
         p.delta_max >= 0 && p.lanczos_k >= 1 && p.max_outer >= 0 && p.max_rtr >= 0 &&
         p.max_tcg >= 1 && p.carry_halvings >= 0 &&
         (p.precision_mode == MANIDSDP_PREC_FP64 || p.precision_mode == MANIDSDP_PREC_MIXED) &&
         flag(p.tcg_device) && flag(p.warm_start) && flag(p.tensor_cores) && flag(p.direct) &&
         p.sigma0 > 0.0 && p.sigma_min > 0.0 && p.sigma_max >= p.sigma_min && p.gamma > 1.0 &&
         p.tol > 0.0 && p.tc_lowprec_eta >= 0.0 && p.sigma_stall >= 0.0 && p.sigma_stall < 1.0;
}

struct NonFinite {};

int guard(const std::function<int()>& f) {
  try {
    return f();
  } catch (const NonFinite&) {
    return MANIDSDP_E_NONFINITE;
  } catch (const DeviceError&) {
    return MANIDSDP_E_CUDA;
  } catch (const std::bad_alloc&) {
    return MANIDSDP_E_NOMEM;
  } catch (...) {
    return MANIDSDP_E_CUDA;
  }
}

void release(manidsdp_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  if (c->hp) cudaFreeHost(c->hp);
  c->hp = nullptr;
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  c->ev0 = c->ev1 = nullptr;
  for (auto& e : c->sev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  for (auto& g : c->graphs) {
    cudaGraphExecDestroy(g.exec);
    cudaGraphDestroy(g.graph);
  }
  c->graphs.clear();
  if (c->cs) cudaStreamDestroy(c->cs);
  if (c->s2) cudaStreamDestroy(c->s2);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  c->cs = nullptr;
}

// Reset the ALM state: XD = Xt + D with Xt given (device) or zero; sigma.
void set_state(manidsdp_ctx* c, const double* Xt_dev, double sigma) {
  const size_t NN = size_t(c->N) * c->N;
  if (Xt_dev == nullptr) {
    MDS_CUDA(cudaMemsetAsync(c->G, 0, NN * sizeof(double), c->s));
    launch_xd_from_xt(NN, 0, c->G, c->idx, c->bm, c->XD, c->s);
  } else {
    launch_xd_from_xt(NN, 0, Xt_dev, c->idx, c->bm, c->XD, c->s);
  }
  c->sigma = sigma;
  c->xdc = 0.0;
  if (c->C != nullptr) dots(c, NN, 1, c->XD, c->C, &c->xdc);
  c->eval_ok = false;
  sync(c);
}

}  // namespace

// ============================== C ABI ========================================
extern "C" {

long long manidsdp_launch_count(void) { return mds::g_launches.load(); }

int manidsdp_hessvec_stage_ms(manidsdp_ctx* c, double* ms5, int reset) {
  if (c == nullptr || ms5 == nullptr) return MANIDSDP_E_ARG;
  for (int i = 0; i < 5; ++i) ms5[i] = c->stage_ms[i];
  if (reset)
    for (double& v : c->stage_ms) v = 0.0;
  return MANIDSDP_OK;
}

void manidsdp_default_params(manidsdp_params* params) {
  if (params) default_params(params);
}

const char* manidsdp_strerror(int status) {
  switch (status) {
    case MANIDSDP_OK: return "ok";
    case MANIDSDP_E_ARG: return "invalid argument";
    case MANIDSDP_E_NONFINITE: return "non-finite value";
    case MANIDSDP_E_NOCONV: return "iteration limit reached before the KKT tolerance";
    case MANIDSDP_E_TIMEOUT: return "device-side wait timed out";
    case MANIDSDP_E_CUDA: return "CUDA runtime error";
    case MANIDSDP_E_NOMEM: return "device allocation failed";
    case MANIDSDP_E_TOOLARGE: return "input exceeds the fixed-size scratch of a no-alloc entry point";
    default: return "unknown status";
  }
}

int manidsdp_setup(manidsdp_ctx** ctx_out, int32_t N, int64_t m, const int32_t* idx,
                   const double* b, int32_t c_kind, const double* c_dense,
                   const manidsdp_params* params, void* stream) {
  if (ctx_out == nullptr || idx == nullptr || b == nullptr || N < 1 || N > kMaxN || m < 1 ||
      m > int64_t(N) * N || (c_kind != MANIDSDP_C_ZERO && c_kind != MANIDSDP_C_DENSE) ||
      (c_kind == MANIDSDP_C_DENSE && c_dense == nullptr))
    return MANIDSDP_E_ARG;
  manidsdp_params prm;
  if (params)
    prm = *params;
  else
    default_params(&prm);
  if (!params_ok(prm)) return MANIDSDP_E_ARG;
  // validate the index map and build the per-class inverse map on the host
  const size_t NN = size_t(N) * N;
  std::vector<int32_t> count(m, 0);
  for (int r = 0; r < N; ++r)
    for (int c2 = 0; c2 < N; ++c2) {
      const int32_t a = idx[size_t(r) * N + c2];
      if (a < 0 || a >= m || a != idx[size_t(c2) * N + r]) return MANIDSDP_E_ARG;
      count[a]++;
    }
  for (int64_t a = 0; a < m; ++a)
    if (count[a] == 0) return MANIDSDP_E_ARG;  // A A* singular (Assumption 2)
  std::vector<double> mult(m);
  for (int64_t a = 0; a < m; ++a) mult[a] = double(count[a]);
  std::vector<int32_t> ucount(m + 1, 0);
  for (int r = 0; r < N; ++r)
    for (int c2 = r; c2 < N; ++c2) ucount[idx[size_t(r) * N + c2] + 1]++;
  for (int64_t a = 0; a < m; ++a) ucount[a + 1] += ucount[a];
  const int32_t n_ent = ucount[m];
  std::vector<uint32_t> ent(n_ent);
  std::vector<int32_t> slot(NN, 0);
  {
    std::vector<int32_t> pos(ucount.begin(), ucount.end() - 1);
    for (int r = 0; r < N; ++r)
      for (int c2 = r; c2 < N; ++c2) {
        const int32_t at = pos[idx[size_t(r) * N + c2]]++;
        ent[at] = (uint32_t(r) << 16) | uint32_t(c2);
        slot[size_t(r) * N + c2] = at;
      }
  }
  std::vector<int32_t> pstart, pclass, mclass, mrange;
  for (int64_t a = 0; a < m; ++a) {
    const int32_t e0 = ucount[a], e1 = ucount[a + 1];
    const int np = (e1 - e0 + kPieceLen - 1) / kPieceLen;
    if (np > 1) {
      mclass.push_back(int32_t(a));
      mrange.push_back(int32_t(pstart.size()));
      mrange.push_back(int32_t(pstart.size()) + np);
    }
    for (int t = 0; t < np; ++t) {
      pstart.push_back(e0 + t * kPieceLen);
      pclass.push_back(np > 1 ? -1 : int32_t(a));
    }
  }
  pstart.push_back(n_ent);

  manidsdp_ctx* c = new (std::nothrow) manidsdp_ctx();
  if (c == nullptr) return MANIDSDP_E_NOMEM;
  int st = guard([&]() -> int {
    c->N = N;
    c->m = m;
    c->c_kind = c_kind;
    c->prm = prm;
    c->s = static_cast<cudaStream_t>(stream);
    MDS_CUDA(cudaMallocHost(&c->hp, 64 * sizeof(double)));
    MDS_CUDA(cudaEventCreate(&c->ev0));
    MDS_CUDA(cudaEventCreate(&c->ev1));
    for (auto& e : c->sev) MDS_CUDA(cudaEventCreate(&e));
    MDS_CUDA(cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking));
    MDS_CUDA(cudaStreamCreateWithFlags(&c->s2, cudaStreamNonBlocking));
    MDS_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    MDS_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    c->idx = dalloc<int32_t>(c, NN);
    MDS_CUDA(cudaMemcpyAsync(c->idx, idx, NN * sizeof(int32_t), cudaMemcpyHostToDevice, c->s));
    c->tc_err = dalloc<int>(c, 1);
    MDS_CUDA(cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->s));
    c->mult = dalloc<double>(c, m);
    MDS_CUDA(cudaMemcpyAsync(c->mult, mult.data(), m * sizeof(double), cudaMemcpyHostToDevice, c->s));
    c->b = dalloc<double>(c, m);
    MDS_CUDA(cudaMemcpyAsync(c->b, b, m * sizeof(double), cudaMemcpyDefault, c->s));
    std::vector<double> hb(m), hbm(m);
    MDS_CUDA(cudaMemcpyAsync(hb.data(), c->b, m * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    sync(c);
    double nb = 0.0;
    for (int64_t a = 0; a < m; ++a) {
      hbm[a] = hb[a] / mult[a];
      nb += hb[a] * hb[a];
    }
    c->normb = std::sqrt(nb);
    c->bm = dalloc<double>(c, m);
    MDS_CUDA(cudaMemcpyAsync(c->bm, hbm.data(), m * sizeof(double), cudaMemcpyHostToDevice, c->s));
    if (c_kind == MANIDSDP_C_DENSE) {
      c->C = dalloc<double>(c, NN);
      MDS_CUDA(cudaMemcpyAsync(c->C, c_dense, NN * sizeof(double), cudaMemcpyDefault, c->s));
    }
    // inverse map
    c->cm.n_entries = n_ent;
    c->cm.n_pieces = int32_t(pclass.size());
    c->cm.n_multi = int32_t(mclass.size());
    c->cm.ent = dalloc<uint32_t>(c, n_ent);
    c->cm.piece_start = dalloc<int32_t>(c, pstart.size());
    c->cm.piece_class = dalloc<int32_t>(c, pclass.size());
    c->cm.multi_class = dalloc<int32_t>(c, mclass.size());
    c->cm.multi_range = dalloc<int32_t>(c, mrange.size());
    MDS_CUDA(cudaMemcpyAsync(c->cm.ent, ent.data(), n_ent * sizeof(uint32_t), cudaMemcpyHostToDevice, c->s));
    MDS_CUDA(cudaMemcpyAsync(c->cm.piece_start, pstart.data(), pstart.size() * 4, cudaMemcpyHostToDevice, c->s));
    MDS_CUDA(cudaMemcpyAsync(c->cm.piece_class, pclass.data(), pclass.size() * 4, cudaMemcpyHostToDevice, c->s));
    if (!mclass.empty()) {
      MDS_CUDA(cudaMemcpyAsync(c->cm.multi_class, mclass.data(), mclass.size() * 4, cudaMemcpyHostToDevice, c->s));
      MDS_CUDA(cudaMemcpyAsync(c->cm.multi_range, mrange.data(), mrange.size() * 4, cudaMemcpyHostToDevice, c->s));
    }
    // N x N work
    c->XD = dalloc<double>(c, NN);
    c->G = dalloc<double>(c, NN);
    c->Gt = dalloc<double>(c, NN);
    c->Gf = dalloc<float>(c, NN);
    c->Gtf = dalloc<float>(c, NN);
    if (prm.precision_mode == MANIDSDP_PREC_MIXED) {
      c->Gh = dalloc<float>(c, NN);
      c->Gl = dalloc<float>(c, NN);
      c->Gth = dalloc<float>(c, NN);
      c->Gtl = dalloc<float>(c, NN);
    }
    // per class
    c->y = dalloc<double>(c, m);
    c->yt = dalloc<double>(c, m);
    c->w = dalloc<double>(c, m);
    c->wf = dalloc<float>(c, m);
    c->y_prev = dalloc<double>(c, m);
    MDS_CUDA(cudaMemsetAsync(c->y_prev, 0, m * sizeof(double), c->s));
    c->piece_buf = dalloc<double>(c, pclass.size());
    c->slot = dalloc<int32_t>(c, NN);
    MDS_CUDA(cudaMemcpyAsync(c->slot, slot.data(), NN * sizeof(int32_t), cudaMemcpyHostToDevice, c->s));
    c->perm = dalloc<float>(c, n_ent);
    if (prm.precision_mode == MANIDSDP_PREC_MIXED) {
      c->permd = dalloc<double>(c, n_ent);
      c->Sup = dalloc<double>(c, NN);
    }
    // N x pcap
    c->pcap = prm.p_max;
    const size_t np = size_t(N) * c->pcap;
    double** dbufs[] = {&c->Y, &c->Yt, &c->GY, &c->grad, &c->eta, &c->Heta, &c->r, &c->delta,
                        &c->Hd, &c->Up, &c->Tm, &c->YM, &c->U, &c->tmp, &c->Vn};
    for (double** pp : dbufs) *pp = dalloc<double>(c, np);
    float** fbufs[] = {&c->Yf, &c->Upf, &c->Tmf, &c->YMf, &c->Yh, &c->Yl};
    for (float** pp : fbufs) *pp = dalloc<float>(c, np);
    c->z = dalloc<double>(c, N);
    c->zt = dalloc<double>(c, N);
    const size_t pp2 = size_t(2) * c->pcap * c->pcap;  // [U'Y; Y'Y]
    c->M1 = dalloc<double>(c, pp2);
    c->M2 = dalloc<double>(c, pp2);
    c->M1f = dalloc<float>(c, pp2);
    c->M2f = dalloc<float>(c, pp2);
    c->part = dalloc<double>(c, gpass_partials(N));
    c->out2 = dalloc<double>(c, 2);
    c->dpart = dalloc<double>(c, 3 * kRedBlocks + 3);
    c->gws_bytes = std::max((np + size_t(2) * 304 * 4096) * sizeof(double),
                            size_t(tcx_gather_splits(N) + 1) * np * sizeof(float));
    c->gws = dalloc<double>(c, c->gws_bytes / sizeof(double));
    c->gws2_bytes = size_t(1) << 21;
    c->gws2 = dalloc<double>(c, c->gws2_bytes / sizeof(double));
    c->tcgst = dalloc<double>(c, (tcg_state_bytes() + 7) / 8);
    c->kpart = dalloc<double>(c, tcg_epilogue_blocks(N));
    c->rpart = dalloc<double>(c, tcg_update_blocks());
    if (c->C != nullptr) {
      double cc;
      dots(c, NN, 1, c->C, c->C, &cc);
      c->normC = std::sqrt(cc);
    }
    c->kmax = std::min(std::max(prm.lanczos_k, 1), N);
    c->LV = dalloc<double>(c, size_t(c->kmax + 2) * N);  // + a locked vector
    c->lh = dalloc<double>(c, c->kmax + 2);
    c->lw = dalloc<double>(c, N);
    c->lz_prev = dalloc<double>(c, N);
    c->lz_lock = dalloc<double>(c, N);
    c->ls = dalloc<double>(c, N);
    set_state(c, nullptr, prm.sigma0);
    return MANIDSDP_OK;
  });
  if (st != MANIDSDP_OK) {
    release(c);
    delete c;
    return st;
  }
  *ctx_out = c;
  return MANIDSDP_OK;
}

void manidsdp_destroy(manidsdp_ctx* ctx) {
  if (ctx == nullptr) return;
  cudaStreamSynchronize(ctx->s);
  if (ctx->cx) complex_destroy(ctx->cx);
  release(ctx);
  delete ctx;
}

int manidsdp_setup_ex(manidsdp_ctx** ctx_out, const manidsdp_problem* pr,
                      const manidsdp_params* params, void* stream) {
  if (ctx_out == nullptr || pr == nullptr) return MANIDSDP_E_ARG;
  manidsdp_params prm;
  if (params)
    prm = *params;
  else
    default_params(&prm);
  if (!params_ok(prm)) return MANIDSDP_E_ARG;
  if (pr->is_complex) {
    if (pr->N < 1 || 2 * int64_t(pr->N) > kMaxN || pr->q_re == nullptr || prm.direct)
      return MANIDSDP_E_ARG;
    auto* c = new (std::nothrow) manidsdp_ctx();
    if (c == nullptr) return MANIDSDP_E_NOMEM;
    c->N = pr->N;
    c->prm = prm;
    c->s = static_cast<cudaStream_t>(stream);
    const int st = complex_setup(&c->cx, pr->N, pr->q_re, pr->q_im, prm, c->s);
    if (st != MANIDSDP_OK) {
      delete c;
      return st;
    }
    *ctx_out = c;
    return MANIDSDP_OK;
  }
  const int N = pr->N;
  if (N < 1 || N > kMaxN || pr->idx == nullptr ||
      (pr->idx_layout != MANIDSDP_IDX_FULL && pr->idx_layout != MANIDSDP_IDX_PACKED_UPPER))
    return MANIDSDP_E_ARG;
  const size_t NN = size_t(N) * N;
  std::vector<int32_t> full;
  const int32_t* idx = pr->idx;
  if (pr->idx_layout == MANIDSDP_IDX_PACKED_UPPER) {  // mirror the upper triangle
    full.resize(NN);
    size_t e = 0;
    for (int r = 0; r < N; ++r)
      for (int g = r; g < N; ++g, ++e) full[size_t(r) * N + g] = full[size_t(g) * N + r] = idx[e];
    idx = full.data();
  }
  std::vector<double> cd;
  const double* cdense = pr->c_dense;
  int32_t kind = pr->c_kind;
  if (kind == MANIDSDP_C_CSR) {  // expand to the dense operand; must be symmetric
    if (pr->c_rowptr == nullptr || pr->c_rowptr[0] != 0) return MANIDSDP_E_ARG;
    cd.assign(NN, 0.0);
    for (int r = 0; r < N; ++r) {
      if (pr->c_rowptr[r + 1] < pr->c_rowptr[r]) return MANIDSDP_E_ARG;
      for (int64_t e = pr->c_rowptr[r]; e < pr->c_rowptr[r + 1]; ++e) {
        const int32_t g = pr->c_col[e];
        if (g < 0 || g >= N || cd[size_t(r) * N + g] != 0.0) return MANIDSDP_E_ARG;
        cd[size_t(r) * N + g] = pr->c_val[e];
      }
    }
    for (int r = 0; r < N; ++r)
      for (int g = r + 1; g < N; ++g)
        if (cd[size_t(r) * N + g] != cd[size_t(g) * N + r]) return MANIDSDP_E_ARG;
    cdense = cd.data();
    kind = MANIDSDP_C_DENSE;
  }
  return manidsdp_setup(ctx_out, N, pr->m, idx, pr->b, kind, cdense, &prm, stream);
}

int manidsdp_set_params(manidsdp_ctx* c, const manidsdp_params* prm) {
  if (c != nullptr && prm != nullptr && c->cx != nullptr) {
    if (!params_ok(*prm) || prm->precision_mode < 0) return MANIDSDP_E_ARG;
    const int st = complex_set_params(c->cx, *prm);
    if (st == MANIDSDP_OK) c->prm = *prm;
    return st;
  }
  if (c == nullptr || prm == nullptr || !params_ok(*prm) || prm->p_max != c->prm.p_max ||
      prm->precision_mode != c->prm.precision_mode)
    return MANIDSDP_E_ARG;
  const bool engine_changed =
      prm->tensor_cores != c->prm.tensor_cores || prm->direct != c->prm.direct;
  c->prm = *prm;
  c->kmax = std::min(std::max(c->prm.lanczos_k, 1), std::min(c->kmax, c->N));
  if (engine_changed) drop_graphs(c);  // cached tCG graphs hold the old gather GEMM
  return MANIDSDP_OK;
}

int manidsdp_set_direct_y(manidsdp_ctx* c, const double* y) {
  if (c == nullptr || c->cx != nullptr || y == nullptr) return MANIDSDP_E_ARG;
  return guard([&]() -> int {
    MDS_CUDA(cudaMemcpyAsync(c->y_prev, y, size_t(c->m) * sizeof(double), cudaMemcpyDefault, c->s));
    c->eval_ok = false;
    sync(c);
    return MANIDSDP_OK;
  });
}

int manidsdp_set_state(manidsdp_ctx* c, const double* Xt, double sigma) {
  if (c != nullptr && c->cx != nullptr) return MANIDSDP_E_ARG;  // no multiplier (R = 0)
  if (c == nullptr || !(sigma > 0.0)) return MANIDSDP_E_ARG;
  return guard([&]() -> int {
    if (Xt != nullptr) {
      const size_t NN = size_t(c->N) * c->N;
      MDS_CUDA(cudaMemcpyAsync(c->Gt, Xt, NN * sizeof(double), cudaMemcpyDefault, c->s));
      set_state(c, c->Gt, sigma);
    } else {
      set_state(c, nullptr, sigma);
    }
    return MANIDSDP_OK;
  });
}

int manidsdp_get_multiplier(manidsdp_ctx* c, double* Xt) {
  if (c != nullptr && c->cx != nullptr) return MANIDSDP_E_ARG;  // no multiplier (R = 0)
  if (c == nullptr || Xt == nullptr) return MANIDSDP_E_ARG;
  return guard([&]() -> int {
    const size_t NN = size_t(c->N) * c->N;
    launch_xd_from_xt(NN, 1, c->XD, c->idx, c->bm, c->Gt, c->s);
    MDS_CUDA(cudaMemcpyAsync(Xt, c->Gt, NN * sizeof(double), cudaMemcpyDefault, c->s));
    c->eval_ok = false;
    sync(c);
    return MANIDSDP_OK;
  });
}

int manidsdp_get_dual_matrix(manidsdp_ctx* c, double* XD) {
  if (c != nullptr && c->cx != nullptr) return MANIDSDP_E_ARG;  // no multiplier (R = 0)
  if (c == nullptr || XD == nullptr) return MANIDSDP_E_ARG;
  return guard([&]() -> int {
    const size_t NN = size_t(c->N) * c->N;
    MDS_CUDA(cudaMemcpyAsync(XD, c->XD, NN * sizeof(double), cudaMemcpyDefault, c->s));
    sync(c);
    return MANIDSDP_OK;
  });
}

int manidsdp_subproblem_eval(manidsdp_ctx* c, const double* Y, int32_t p, double* psi,
                             double* rgrad, double* z, double* y, double* rnorm) {
  if (c != nullptr && c->cx != nullptr) {
    if (Y == nullptr || y != nullptr) return MANIDSDP_E_ARG;
    if (rnorm) *rnorm = 0.0;
    return complex_eval(c->cx, Y, p, psi, rgrad, z);
  }
  if (c == nullptr || Y == nullptr || p < 1 || p > c->pcap) return MANIDSDP_E_ARG;
  return guard([&]() -> int {
    const size_t np = size_t(c->N) * p;
    MDS_CUDA(cudaMemcpyAsync(c->Y, Y, np * sizeof(double), cudaMemcpyDefault, c->s));
    double ps, r2;
    if (mixed(c)) {
      evaluate(c, c->Y, p, c->y, c->G, nullptr, &ps, &r2, c->Gh, c->Gl);
      gradient(c, c->Y, p, c->G, c->Gh, c->Gl);
    } else {
      evaluate(c, c->Y, p, c->y, c->G, c->Gf, &ps, &r2);
      gradient(c, c->Y, p, c->G);
    }
    c->yf_valid = false;
    c->eval_ok = true;
    c->eval_user_Y = Y;
    c->eval_p = p;
    if (psi) *psi = ps;
    if (rnorm) *rnorm = std::sqrt(r2);
    if (rgrad) MDS_CUDA(cudaMemcpyAsync(rgrad, c->grad, np * sizeof(double), cudaMemcpyDefault, c->s));
    if (z) MDS_CUDA(cudaMemcpyAsync(z, c->z, c->N * sizeof(double), cudaMemcpyDefault, c->s));
    if (y) MDS_CUDA(cudaMemcpyAsync(y, c->y, c->m * sizeof(double), cudaMemcpyDefault, c->s));
    sync(c);
    return MANIDSDP_OK;
  });
}

int manidsdp_hessvec(manidsdp_ctx* c, const double* Y, const double* U, int32_t p, double* HU,
                     int32_t precision) {
  if (c != nullptr && c->cx != nullptr) {
    if (Y == nullptr || U == nullptr || HU == nullptr) return MANIDSDP_E_ARG;
    return complex_hessvec(c->cx, Y, U, p, HU, precision);
  }
  if (c == nullptr || Y == nullptr || U == nullptr || HU == nullptr || p < 1 || p > c->pcap ||
      (precision != MANIDSDP_PREC_FP64 && precision != MANIDSDP_PREC_MIXED))
    return MANIDSDP_E_ARG;
  if (!c->eval_ok || c->eval_user_Y != Y || c->eval_p != p) return MANIDSDP_E_ARG;
  return guard([&]() -> int {
    const size_t np = size_t(c->N) * p;
    MDS_CUDA(cudaMemcpyAsync(c->delta, U, np * sizeof(double), cudaMemcpyDefault, c->s));
    hessvec(c, c->Y, c->delta, p, c->Hd, precision);
    MDS_CUDA(cudaMemcpyAsync(HU, c->Hd, np * sizeof(double), cudaMemcpyDefault, c->s));
    sync(c);
    return take_device_error(c);
  });
}

int manidsdp_lanczos(manidsdp_ctx* c, const double* Y, int32_t p, int32_t which, int32_t k,
                     double* lambda, double* v, int32_t* steps) {
  if (c != nullptr && c->cx != nullptr) {
    if (Y == nullptr || lambda == nullptr || (which != MANIDSDP_EIG_MIN && which != MANIDSDP_EIG_MAX))
      return MANIDSDP_E_ARG;
    return complex_lanczos(c->cx, Y, p, which, k, lambda, which == MANIDSDP_EIG_MIN ? v : nullptr,
                           steps);
  }
  if (c == nullptr || Y == nullptr || p < 1 || p > c->pcap || lambda == nullptr ||
      (which != MANIDSDP_EIG_MIN && which != MANIDSDP_EIG_MAX))
    return MANIDSDP_E_ARG;
  return guard([&]() -> int {
    const int N = c->N;
    const size_t np = size_t(N) * p;
    MDS_CUDA(cudaMemcpyAsync(c->tmp, Y, np * sizeof(double), cudaMemcpyDefault, c->s));
    launch_gemm<double>(N, p, N, c->XD, N, c->tmp, p, c->GY, p, 1.0, 0.0, nullptr, nullptr, 0.0,
                        nullptr, c->gws, c->gws_bytes, c->s);
    launch_rowdot(N, p, c->GY, c->tmp, c->zt, c->s);
    LanczosOut lo = lanczos(c, c->zt, k > 0 ? k : c->prm.lanczos_k, 1);
    if (which == MANIDSDP_EIG_MIN) {
      *lambda = lo.lo[0];
      if (v) MDS_CUDA(cudaMemcpyAsync(v, c->Vn, N * sizeof(double), cudaMemcpyDefault, c->s));
    } else {
      *lambda = lo.hi;
      if (v) return MANIDSDP_E_ARG;  // only the smallest pair carries a vector
    }
    if (steps) *steps = lo.steps;
    c->eval_ok = false;
    sync(c);
    return MANIDSDP_OK;
  });
}

}  // extern "C"

// ============================== Algorithm 1 ==================================
namespace {

struct TcgOut {
  int iters;
  bool boundary;
};

// Truncated CG on the trust-region model at c->Y (gradient in c->grad).
TcgOut tcg(manidsdp_ctx* c, int p, double Delta, double tol_grad) {
  const int N = c->N;
  const size_t n = size_t(N) * p;
  const manidsdp_params& P = c->prm;
  MDS_CUDA(cudaMemsetAsync(c->eta, 0, n * sizeof(double), c->s));
  MDS_CUDA(cudaMemsetAsync(c->Heta, 0, n * sizeof(double), c->s));
  MDS_CUDA(cudaMemcpyAsync(c->r, c->grad, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  launch_axpby(n, -1.0, c->grad, 0.0, nullptr, c->delta, c->s);
  double rr;
  dots(c, n, 1, c->r, c->r, &rr);
  const double r0 = std::sqrt(rr);
  double ee = 0.0, ed = 0.0, dd = rr;
  const double target = std::max(r0 * std::max(std::min(std::pow(r0, 1.0), 0.1), P.tcg_floor),
                                 P.tcg_abs * tol_grad);
  for (int j = 1; j <= P.max_tcg; ++j) {
    hessvec(c, c->Y, c->delta, p, c->Hd, P.precision_mode);
    double kap;
    dots(c, n, 1, c->delta, c->Hd, &kap);
    const double alpha = kap != 0.0 ? rr / kap : INFINITY;
    const double ee_new = ee + 2.0 * alpha * ed + alpha * alpha * dd;
    if (kap <= 0.0 || ee_new >= Delta * Delta) {
      const double tau = (-ed + std::sqrt(ed * ed + dd * (Delta * Delta - ee))) / dd;
      launch_axpby(n, tau, c->delta, 1.0, c->eta, c->eta, c->s);
      launch_axpby(n, tau, c->Hd, 1.0, c->Heta, c->Heta, c->s);
      return {j, true};
    }
    launch_axpby(n, alpha, c->delta, 1.0, c->eta, c->eta, c->s);
    launch_axpby(n, alpha, c->Hd, 1.0, c->Heta, c->Heta, c->s);
    launch_axpby(n, alpha, c->Hd, 1.0, c->r, c->r, c->s);
    ee = ee_new;
    double rr_new;
    dots(c, n, 1, c->r, c->r, &rr_new);
    if (std::sqrt(rr_new) <= target) return {j, false};
    const double beta = rr_new / rr;
    rr = rr_new;
    launch_axpby(n, -1.0, c->r, beta, c->delta, c->delta, c->s);
    ed = beta * (ed + alpha * dd);
    dd = rr + beta * beta * dd;
  }
  return {P.max_tcg, false};
}

void drop_graphs(manidsdp_ctx* c) {
  for (auto& g : c->graphs) {
    cudaGraphExecDestroy(g.exec);
    cudaGraphDestroy(g.graph);
  }
  c->graphs.clear();
}

// Build the WHILE-node graph of one tCG run at the current (p, sigma, Y, G).
manidsdp_ctx::Graph& tcg_graph_for(manidsdp_ctx* c, int p, int prec) {
  const void* Gkey = prec == MANIDSDP_PREC_MIXED ? static_cast<const void*>(g32(c))
                                                 : static_cast<const void*>(c->G);
  for (auto& g : c->graphs)
    if (g.p == p && g.prec == prec && g.sigma == c->sigma && g.Y == c->Y && g.G == Gkey &&
        g.pairs == c->tc_pairs)
      return g;
  if (c->graphs.size() >= 4) drop_graphs(c);
  const int N = c->N;
  const size_t n = size_t(N) * p;
  manidsdp_ctx::Graph G{};
  G.p = p;
  G.prec = prec;
  G.sigma = c->sigma;
  G.Y = c->Y;
  G.G = Gkey;
  G.pairs = c->tc_pairs;
  MDS_CUDA(cudaGraphCreate(&G.graph, 0));
  cudaGraphConditionalHandle h;
  MDS_CUDA(cudaGraphConditionalHandleCreate(&h, G.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  MDS_CUDA(cudaGraphAddNode(&node, G.graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const long long l0 = launches_now();
  MDS_CUDA(cudaStreamBeginCaptureToGraph(c->cs, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
  cudaStream_t s = c->cs;
  const int neb = tcg_epilogue_blocks(N);
  if (prec == MANIDSDP_PREC_FP64) {
    launch_tcg_prep<double>(N, p, c->tcgst, c->Y, c->r, c->delta, c->Up, nullptr, s);
    if (c->prm.direct)  // direct formulation: no class-mean term
      MDS_CUDA(cudaMemsetAsync(c->w, 0, size_t(c->m) * sizeof(double), s));
    else
      launch_class_means<double>(c->cm, N, p, 1, c->Y, c->Up, nullptr, c->mult, c->piece_buf,
                                 c->w, s);
    const int splits = launch_gemm_partials<double>(N, p, N, c->G, N, c->Up, p, c->idx, c->w,
                                                    -c->sigma, c->Y, c->gws, c->gws_bytes, s);
    launch_gram2<double>(N, p, c->Up, c->Y, c->Y, c->M1, c->gws2, c->gws2_bytes, s);
    launch_tcg_epilogue<double>(N, p, splits, static_cast<const double*>(c->gws), c->M1, c->Y,
                                c->Up, c->z, c->sigma, c->delta, c->Hd, c->kpart, s);
  } else {
    launch_tcg_prep<float>(N, p, c->tcgst, c->Y, c->r, c->delta, c->Up, c->Upf, s);
    const int splits = hessvec32_body(c, p, s, true);
    launch_tcg_epilogue<float>(N, p, splits, static_cast<const float*>(c->gws), nullptr, c->Y,
                               c->Up, c->z, c->sigma, c->delta, c->Hd, c->kpart, s);
  }
  launch_tcg_alpha(neb, c->kpart, c->tcgst, s);
  launch_tcg_update(n, c->tcgst, c->delta, c->Hd, c->eta, c->Heta, c->r, c->rpart, s);
  launch_tcg_beta(tcg_update_blocks(), c->rpart, c->tcgst, h, s);
  MDS_CUDA(cudaStreamEndCapture(c->cs, &body));
  G.body_launches = launches_now() - l0;
  uncount_launches(G.body_launches);  // counted per executed iteration instead
  MDS_CUDA(cudaGraphInstantiate(&G.exec, G.graph, 0));
  c->graphs.push_back(G);
  return c->graphs.back();
}

// tCG as one graph launch; eta, Heta hold the step and H eta on return.
TcgOut tcg_device(manidsdp_ctx* c, int p, double Delta, double tol_grad) {
  const int N = c->N;
  const size_t n = size_t(N) * p;
  const manidsdp_params& P = c->prm;
  const int prec = P.precision_mode;
  if (prec == MANIDSDP_PREC_MIXED && !c->yf_valid) {
    launch_to_float(n, c->Y, c->Yf, c->s);
    launch_gram2<float>(N, p, c->Yf, nullptr, c->Yf, c->M1f + size_t(p) * p, c->gws2,
                        c->gws2_bytes, c->s);
    if (use_tcx(c)) tcx_point(c, c->Y, p, c->s);
    c->yf_valid = true;
  }
  MDS_CUDA(cudaMemsetAsync(c->eta, 0, n * sizeof(double), c->s));
  MDS_CUDA(cudaMemsetAsync(c->Heta, 0, n * sizeof(double), c->s));
  MDS_CUDA(cudaMemsetAsync(c->delta, 0, n * sizeof(double), c->s));
  MDS_CUDA(cudaMemcpyAsync(c->r, c->grad, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  const double* gg[1] = {c->grad};
  launch_dots(n, 1, gg, gg, c->dpart, c->s);
  launch_tcg_init(c->tcgst, c->dpart + 3 * kRedBlocks, Delta, P.tcg_floor, P.tcg_abs * tol_grad,
                  P.max_tcg, c->s);
  auto& G = tcg_graph_for(c, p, prec);
  tstart(c);
  MDS_CUDA(cudaGraphLaunch(G.exec, c->s));
  tstop(c, &c->ms_hv);
  int flag = 0, iters = 0;
  tcg_read_state(c->tcgst, &flag, &iters, c->hp + 16, c->s);
  count_launches(G.body_launches * iters);
  c->hessvecs += iters;
  c->hv_psum += double(p) * iters;
  return {iters, flag == 2 || flag == 3};
}

struct RtrOut {
  int iters;
  double gnorm;
  int rejected = 0, boundary = 0;
  double delta_end = 0.0;
};

// Riemannian trust region on Psi_k from c->Y; leaves y, G, z, grad at the final Y.
RtrOut rtr(manidsdp_ctx* c, int p, double tol_grad) {
  const int N = c->N;
  const size_t n = size_t(N) * p;
  const manidsdp_params& P = c->prm;
  const double Delta_bar = M_PI * std::sqrt(double(N));
  double Delta = Delta_bar / 8.0;
  double fx, r2;
  const bool mx = mixed(c);
  evaluate(c, c->Y, p, c->y, mx ? nullptr : c->G, nullptr, &fx, &r2, mx ? c->Gh : nullptr,
           mx ? c->Gl : nullptr);
  c->yf_valid = false;
  double gn = gradient(c, c->Y, p, c->G, mx ? c->Gh : nullptr, mx ? c->Gl : nullptr);
  int it = 0, nrej = 0, nbound = 0;
  for (; it < P.max_rtr; ++it) {
    if (gn <= tol_grad) break;
    TcgOut t = P.tcg_device ? tcg_device(c, p, Delta, tol_grad) : tcg(c, p, Delta, tol_grad);
    double d2[2];
    dots(c, n, 2, c->grad, c->eta, d2, c->eta, c->Heta);
    const double model_dec = -(d2[0] + 0.5 * d2[1]);
    launch_retract(N, p, c->Y, c->eta, 1.0, c->Yt, c->s);
    double f_new, r2n;
    evaluate(c, c->Yt, p, c->yt, mx ? nullptr : c->Gt, nullptr, &f_new, &r2n,
             mx ? c->Gth : nullptr, mx ? c->Gtl : nullptr);
    const double reg = std::max(1.0, std::fabs(fx)) * 1e3 * 2.220446049250313e-16;
    const double rho = (model_dec + reg > 0.0) ? (fx - f_new + reg) / (model_dec + reg) : -INFINITY;
    if (!std::isfinite(f_new)) throw NonFinite{};
    if (rho < 0.25)
      Delta /= 4.0;
    else if (rho > 0.75 && t.boundary)
      Delta = std::min(2.0 * Delta, Delta_bar);
    if (t.boundary) ++nbound;
    if (!(rho > 0.1)) ++nrej;
    if (rho > 0.1) {
      std::swap(c->Y, c->Yt);
      std::swap(c->G, c->Gt);
      std::swap(c->Gf, c->Gtf);
      std::swap(c->Gh, c->Gth);
      std::swap(c->Gl, c->Gtl);
      std::swap(c->y, c->yt);
      fx = f_new;
      c->yf_valid = false;
      gn = gradient(c, c->Y, p, c->G, mx ? c->Gh : nullptr, mx ? c->Gl : nullptr);
    }
  }
  c->rtr_iters += it;
  c->psi = fx;
  RtrOut out{it, gn};
  out.rejected = nrej;
  out.boundary = nbound;
  out.delta_end = Delta;
  return out;
}

// Row-major N x p_old -> N x p_new in place through c->tmp (zero-padded columns).
void relayout(manidsdp_ctx* c, double* buf, int p_old, int p_new) {
  launch_pad_cols(c->N, p_old, p_new, buf, c->tmp, c->s);
  MDS_CUDA(cudaMemcpyAsync(buf, c->tmp, size_t(c->N) * p_new * sizeof(double),
                           cudaMemcpyDeviceToDevice, c->s));
}

}  // namespace

extern "C" int manidsdp_solve(manidsdp_ctx* c, const double* Y0, int32_t p0, double* Y_out,
                              int32_t* p_out, double* y_out, double* z_out, double* Xt_out,
                              manidsdp_report* report) {
  if (c != nullptr && c->cx != nullptr) {
    if (y_out != nullptr || Xt_out != nullptr) return MANIDSDP_E_ARG;
    return complex_solve(c->cx, Y0, p0, Y_out, p_out, z_out, report);
  }
  if (c == nullptr || Y0 == nullptr || p0 < 1 || p0 > c->pcap) return MANIDSDP_E_ARG;
  int status = MANIDSDP_E_NOCONV;
  manidsdp_report rep{};
  int gst = guard([&]() -> int {
    const int N = c->N;
    const manidsdp_params& P = c->prm;
    const auto t_solve0 = std::chrono::steady_clock::now();
    c->hessvecs = c->rtr_iters = c->lanczos_mv = c->evals = c->grads = 0;
    c->hv_psum = c->ms_hv = c->ms_eval = c->ms_grad = c->ms_lz = c->ms_rank = 0.0;
    const bool resume = P.warm_start && c->resume_valid;
    if (!resume) c->lz_prev_ok = false;
    int p = p0;
    double rscale = -1.0;
    double sigma = P.sigma0;
    if (resume) {  // continue from the context's factor, multiplier and penalty
      p = c->resume_p;
      rscale = c->resume_rscale;
      sigma = c->sigma;
      c->eval_ok = false;
    } else {
      set_state(c, nullptr, P.sigma0);
      c->resume_outer = 0;
      MDS_CUDA(cudaMemcpyAsync(c->tmp, Y0, size_t(N) * p * sizeof(double), cudaMemcpyDefault, c->s));
      launch_retract(N, p, c->tmp, c->tmp, 0.0, c->Y, c->s);
      if (P.direct) {  // the direct formulation's first frozen y: y(S0 + C)
        double f0, r20;
        const bool mx = mixed(c);
        evaluate(c, c->Y, p, c->y, mx ? nullptr : c->G, nullptr, &f0, &r20, mx ? c->Gh : nullptr,
                 mx ? c->Gl : nullptr);
        MDS_CUDA(cudaMemcpyAsync(c->y_prev, c->y, size_t(c->m) * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->s));
        c->eval_ok = false;
      }
    }
    bool have_U = resume && c->resume_have_U;
    int U_cols = have_U ? c->resume_U_cols : 0;
    double eta_prev = INFINITY;
    for (int k = 0; k < P.max_outer; ++k) {
      c->sigma = sigma;
      // precision schedule: single TF32 products while eta_max is above tc_lowprec_eta
      c->tc_pairs = (P.tc_lowprec_eta > 0.0 && eta_prev > P.tc_lowprec_eta) ? 0 : 1;
      // step 3a: the carried direction U = [0, V]
      if (have_U) {
        double f0, r2;
        const bool mx = mixed(c);
        evaluate(c, c->Y, p, c->y, mx ? nullptr : c->G, nullptr, &f0, &r2, mx ? c->Gh : nullptr,
                 mx ? c->Gl : nullptr);
        c->yf_valid = false;
        gradient(c, c->Y, p, c->G, mx ? c->Gh : nullptr, mx ? c->Gl : nullptr);
        hessvec(c, c->Y, c->U, p, c->Hd, P.precision_mode);
        double curv;
        dots(c, size_t(N) * p, 1, c->U, c->Hd, &curv);
        bool moved = false;
        if (curv < 0.0) {
          double t = P.carry_t0 > 0.0 ? P.carry_t0 : std::sqrt(double(N));
          for (int i = 0; i < P.carry_halvings; ++i) {
            launch_retract(N, p, c->Y, c->U, t, c->Yt, c->s);
            double ft, r2t;
            evaluate(c, c->Yt, p, c->yt, mx ? nullptr : c->Gt, nullptr, &ft, &r2t,
                     mx ? c->Gth : nullptr, mx ? c->Gtl : nullptr);
            if (ft <= f0 - 1e-4 * 0.5 * t * t * std::fabs(curv)) {
              std::swap(c->Y, c->Yt);
              moved = true;
              break;
            }
            t *= 0.5;
          }
        }
        if (!moved) {
          launch_pad_cols(N, p, p - U_cols, c->Y, c->tmp, c->s);  // keep the first p-U_cols columns
          p -= U_cols;
          MDS_CUDA(cudaMemcpyAsync(c->Y, c->tmp, size_t(N) * p * sizeof(double),
                                   cudaMemcpyDeviceToDevice, c->s));
        }
        have_U = false;
      }
      // step 3b: RTR on Psi_k
      const double tol_k = rscale < 0.0 ? P.tol_grad_max
                                        : std::max(P.tol_grad_min,
                                                   std::min(P.tol_grad_max, P.tol_grad_factor * rscale));
      RtrOut ro = rtr(c, p, tol_k);
      // steps 4-8: y at the final Y is in c->y; Xt <- Xt - sigma R
      if (mixed(c)) {
        launch_split(size_t(N) * p, c->Y, c->Yh, c->Yl, c->s);
        launch_gpass_df(N, p, 1, c->Yh, c->Yl, c->idx, c->y, c->C, sigma, c->XD, nullptr, nullptr,
                        nullptr, c->part, c->out2, c->s);
      } else {
        launch_gpass(N, p, 1, c->Y, c->idx, c->y, c->C, sigma, c->XD, nullptr, nullptr, c->part,
                     c->out2, c->s);
      }
      if (P.direct)  // the next subproblem's frozen y (direct formulation's y-update)
        MDS_CUDA(cudaMemcpyAsync(c->y_prev, c->y, size_t(c->m) * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->s));
      MDS_CUDA(cudaMemcpyAsync(c->hp, c->out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
      sync(c);
      const double rnorm = std::sqrt(c->hp[0]);
      const double sum_z = c->hp[1];
      if (c->C != nullptr) dots(c, size_t(N) * N, 1, c->XD, c->C, &c->xdc);
      launch_gemm<double>(N, p, N, c->XD, N, c->Y, p, c->GY, p, 1.0, 0.0, nullptr, nullptr, 0.0,
                          nullptr, c->gws, c->gws_bytes, c->s);
      launch_rowdot(N, p, c->GY, c->Y, c->z, c->s);
      // step 9: extreme eigenpairs of X
      // the carried negative-curvature directions need converged Ritz vectors,
      // so the full Krylov cap; warm-started from the previous certificate's vector
      const int nsmall = std::max(1, P.delta_max);
      LanczosOut lo = lanczos(c, c->z, P.lanczos_k, nsmall, true,
                              c->lz_prev_ok ? c->lz_prev : nullptr);
      double by;
      dots(c, c->m, 1, c->b, c->y, &by);
      rep.eta_p = rnorm / (1.0 + c->normC);
      rep.pobj = sum_z + c->xdc;
      rep.value = by;
      rep.eta_g = std::fabs(rep.pobj - by) / (1.0 + std::fabs(rep.pobj) + std::fabs(by));
      if (lo.nvec > 0) {  // warm start of the next certificate check
        launch_pad_cols(N, lo.nvec, 1, c->Vn, c->lz_prev, c->s);
        c->lz_prev_ok = true;
      }
      rep.eta_d = std::max(0.0, -lo.lo[0]) / (1.0 + std::fabs(lo.hi));
      rep.lambda_min = lo.lo[0];
      rep.lambda_max = lo.hi;
      rep.sigma = sigma;
      rep.outer = k + 1;
      rep.p = p;
      const double eta = std::max(rep.eta_p, std::max(rep.eta_d, rep.eta_g));
      eta_prev = eta;
      if (P.verbose)
        std::fprintf(stderr,
                     "[manidsdp] k=%d p=%d sigma=%.3g rtr=%d(rej %d, bnd %d, D %.2e) gnorm=%.3e "
                     "tol=%.2e eta=(%.2e %.2e %.2e) lmin=%.3e V=%.12f hv=%d lz=%d t=%.3fs\n",
                     k, p, sigma, ro.iters, ro.rejected, ro.boundary, ro.delta_end, ro.gnorm, tol_k,
                     rep.eta_p, rep.eta_d, rep.eta_g, lo.lo[0], by, c->hessvecs, lo.steps,
                     std::chrono::duration<double>(std::chrono::steady_clock::now() - t_solve0)
                         .count());
      if (!std::isfinite(eta)) {
        status = MANIDSDP_E_NONFINITE;
        break;
      }
      // the stop needs lambda_min itself, not an upper bound of it
      if (eta <= P.tol && lo.converged) {
        status = MANIDSDP_OK;
        break;
      }
      // step 10 (first half): drop numerically null directions of Y
      {
        launch_gram<double>(N, p, p, c->Y, c->Y, c->M2, c->gws, c->gws_bytes, c->s);
        std::vector<double> A(size_t(p) * p);
        MDS_CUDA(cudaMemcpyAsync(A.data(), c->M2, A.size() * sizeof(double), cudaMemcpyDeviceToHost, c->s));
        sync(c);
        const auto th0 = std::chrono::steady_clock::now();
        const SymTridiag T = sym_tridiag(A, p);
        const double wmax = tridiag_eig(T.d, T.e, p, p - 1);
        // rank-one rounding: Yr = sign(Y w), w the top eigenvector of Y'Y; accept when
        // Yr Yr' is consistent with the classes (R = 0) and its certificate is PSD
        if (eta <= P.round_eta) {
          std::vector<double> wtop = tridiag_vec(T.d, T.e, p, wmax, {});
          tridiag_backtransform(T, wtop);
          MDS_CUDA(cudaMemcpyAsync(c->M1, wtop.data(), p * sizeof(double), cudaMemcpyHostToDevice, c->s));
          launch_gemm<double>(N, 1, p, c->Y, p, c->M1, 1, c->GY, 1, 1.0, 0.0, nullptr, nullptr,
                              0.0, nullptr, c->gws, c->gws_bytes, c->s);
          launch_sign(N, c->GY, c->Yt, c->s);
          double fr, r2r;
          const bool mx = mixed(c);
          evaluate(c, c->Yt, 1, c->yt, mx ? nullptr : c->Gt, nullptr, &fr, &r2r,
                   mx ? c->Gth : nullptr, mx ? c->Gtl : nullptr);
          if (r2r == 0.0) {
            launch_gemm<double>(N, 1, N, c->XD, N, c->Yt, 1, c->GY, 1, 1.0, 0.0, nullptr, nullptr,
                                0.0, nullptr, c->gws, c->gws_bytes, c->s);
            launch_rowdot(N, 1, c->GY, c->Yt, c->zt, c->s);
            // Yr / sqrt(N) is an exact null vector of X_r (X_r Yr = 0 entrywise
            // since Yr_i^2 = 1): lock it, so that Lanczos resolves the rest of
            // the spectrum instead of a cluster at zero
            launch_axpby(N, 1.0 / std::sqrt(double(N)), c->Yt, 0.0, nullptr, c->lz_lock, c->s);
            LanczosOut lr = lanczos(c, c->zt, P.lanczos_k, 1, false,
                                    c->lz_prev_ok ? c->lz_prev : nullptr, c->lz_lock);
            double byr;
            dots(c, c->m, 1, c->b, c->yt, &byr);
            const double ed = std::max(0.0, -lr.lo[0]) / (1.0 + std::fabs(lr.hi));
            // with R = 0 the evaluated Psi is <Xt + D, S_r + C> = sum(z_r) + <C, Xt + D>
            const double po = fr;
            const double eg = std::fabs(po - byr) / (1.0 + std::fabs(po) + std::fabs(byr));
            if (std::max(ed, eg) <= P.tol && lr.converged) {
              MDS_CUDA(cudaMemcpyAsync(c->Y, c->Yt, N * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
              MDS_CUDA(cudaMemcpyAsync(c->y, c->yt, c->m * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
              MDS_CUDA(cudaMemcpyAsync(c->z, c->zt, N * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
              p = 1;
              rep.eta_p = 0.0;
              rep.eta_d = ed;
              rep.eta_g = eg;
              rep.pobj = po;
              rep.value = byr;
              rep.lambda_min = lr.lo[0];
              rep.lambda_max = lr.hi;
              rep.p = 1;
              if (P.verbose)
                std::fprintf(stderr, "[manidsdp] k=%d rank-one rounding accepted: eta=(0 %.2e %.2e) V=%.12f\n",
                             k, ed, eg, byr);
              status = MANIDSDP_OK;
              break;
            }
          }
        }
        // keep the eigendirections of Y'Y above rank_tol * lambda_max, at least p_min
        const int nlow = sturm_below(T.d, T.e, p, P.rank_tol * wmax);
        const int r = std::max(p - nlow, std::min(P.p_min, p));
        if (r < p) {
          std::vector<std::vector<double>> vecs;  // eigenvectors of T, descending
          for (int i = p - 1; i >= p - r; --i)
            vecs.push_back(tridiag_vec(T.d, T.e, p, tridiag_eig(T.d, T.e, p, i), vecs));
          std::vector<double> W(size_t(p) * r);  // row-major p x r, columns ascending
          for (int j = 0; j < r; ++j) {
            std::vector<double> x = vecs[r - 1 - j];
            tridiag_backtransform(T, x);
            for (int i = 0; i < p; ++i) W[size_t(i) * r + j] = x[i];
          }
          MDS_CUDA(cudaMemcpyAsync(c->M1, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, c->s));
          launch_gemm<double>(N, r, p, c->Y, p, c->M1, r, c->tmp, r, 1.0, 0.0, nullptr, nullptr,
                              0.0, nullptr, c->gws, c->gws_bytes, c->s);
          launch_retract(N, r, c->tmp, c->tmp, 0.0, c->Y, c->s);
          p = r;
        }
        c->ms_rank += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th0).count();
      }
      // step 11: sigma rule (5.1)
      const double lhs = rnorm / (1.0 + c->normb);
      const double lhs_prev = rscale;
      rscale = lhs;
      if (lhs < P.kappa1 * ro.gnorm)
        sigma = std::max(sigma / P.gamma, P.sigma_min);
      else if (lhs > P.kappa2 * ro.gnorm)
        sigma = std::min(P.gamma * sigma, P.sigma_max);
      else if (P.sigma_stall > 0.0 && lhs_prev > 0.0 && ro.gnorm <= tol_k &&
               lhs > P.sigma_stall * lhs_prev)  // stalled primal residual (params.sigma_stall)
        sigma = std::min(P.gamma * sigma, P.sigma_max);
      // steps 9-10 (second half): negative curvature -> U = [0, V], Y = [Y, 0]
      const double thr = -P.neg_tol * (1.0 + std::fabs(lo.hi));
      int nneg = 0;
      while (nneg < int(lo.lo.size()) && lo.lo[nneg] < thr) ++nneg;
      const int delta = std::min(std::min(nneg, P.delta_max), P.p_max - p);
      if (delta > 0) {
        relayout(c, c->Y, p, p + delta);
        MDS_CUDA(cudaMemsetAsync(c->U, 0, size_t(N) * (p + delta) * sizeof(double), c->s));
        // Vn is N x nvec row-major; take its first delta columns
        launch_pad_cols(N, lo.nvec, delta, c->Vn, c->Tm, c->s);
        launch_set_cols(N, p + delta, p, delta, c->Tm, c->U, c->s);
        p += delta;
        have_U = true;
        U_cols = delta;
      }
    }
    c->sigma = sigma;
    c->tc_pairs = 1;
    c->resume_valid = true;
    c->resume_p = p;  // columns of c->Y now (after rank drop and augmentation)
    c->resume_rscale = rscale;
    c->resume_outer += rep.outer;
    c->resume_have_U = have_U;
    c->resume_U_cols = U_cols;
    rep.rtr_iters = c->rtr_iters;
    rep.hessvecs = c->hessvecs;
    rep.lanczos_matvecs = c->lanczos_mv;
    rep.evals = c->evals;
    rep.grads = c->grads;
    rep.hessvec_p_sum = c->hv_psum;
    rep.ms_hessvec = c->ms_hv;
    rep.ms_eval = c->ms_eval;
    rep.ms_grad = c->ms_grad;
    rep.ms_lanczos = c->ms_lz;
    rep.ms_rank = c->ms_rank;
    rep.status = status;
    if (Y_out) MDS_CUDA(cudaMemcpyAsync(Y_out, c->Y, size_t(N) * rep.p * sizeof(double), cudaMemcpyDefault, c->s));
    if (p_out) *p_out = rep.p;
    if (y_out) MDS_CUDA(cudaMemcpyAsync(y_out, c->y, c->m * sizeof(double), cudaMemcpyDefault, c->s));
    if (z_out) MDS_CUDA(cudaMemcpyAsync(z_out, c->z, N * sizeof(double), cudaMemcpyDefault, c->s));
    if (Xt_out) {
      launch_xd_from_xt(size_t(N) * N, 1, c->XD, c->idx, c->bm, c->Gt, c->s);
      MDS_CUDA(cudaMemcpyAsync(Xt_out, c->Gt, size_t(N) * N * sizeof(double), cudaMemcpyDefault, c->s));
    }
    sync(c);
    c->eval_ok = false;
    return take_device_error(c);
  });
  if (report) *report = rep;
  if (gst != MANIDSDP_OK) return gst;
  return status;
}

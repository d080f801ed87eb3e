// The first-order complex relaxation (UCQP: min z^H Q z, |z_i| = 1) on one GPU.
//
// Factor: Y = A + iB held as the real n x 2p array [A | B]; G Y = Q Y is the real
// GEMM  Qre [A | B] + Qim [-B | A]  (K = 2n).  The mixed form runs the tCG
// Hessian-vector products  Hess[U] = P_Y(2 Q Up) - 2 Diag(mu) Up  (Up = P_Y(U);
// the Q(W) term of Proposition 4.2 vanishes: every entry is its own class) on the
// tensor cores as the two-segment TF32-pair GEMM [Qre | Qim] [Up ; Up J]; the
// cost, gradient, multipliers mu and certificate stay FP64.  lambda_min of the
// Hermitian certificate X = Q - Diag(mu) comes from Lanczos with full FP64
// reorthogonalisation on its real embedding [[Xre, -Xim], [Xim, Xre]] (2n x 2n,
// each eigenvalue twice; an eigenvector [a; b] is the complex vector a + ib).
// Rank adaptation follows Theorem 4.5: while lambda_min < -neg_tol (1 +
// |lambda_max|) one column is appended and the factor moves along [0, v] by
// backtracking with the second-order Armijo test.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "complex1.h"
#include "host_linalg.h"

namespace mds {

using namespace hostla;

struct ComplexState {
  int n = 0, pcap = 0, kmax = 0;
  cudaStream_t s = nullptr;
  manidsdp_params prm{};
  std::vector<void*> allocs;
  double* hp = nullptr;  // pinned host scalars
  double *Qre = nullptr, *Qim = nullptr, *XB = nullptr;
  float *Qh = nullptr, *Ql = nullptr, *QIh = nullptr, *QIl = nullptr;  // TF32 pairs (ld ldg)
  // n x 2 pcap (FP64)
  double *Y = nullptr, *Yt = nullptr, *G = nullptr, *grad = nullptr, *eta = nullptr,
         *Heta = nullptr, *r = nullptr, *delta = nullptr, *Hd = nullptr, *Up = nullptr,
         *U = nullptr, *tmp = nullptr, *rot = nullptr, *Tm = nullptr;
  float *Upf = nullptr, *Yf = nullptr;
  float *UTh = nullptr, *UTl = nullptr, *UJh = nullptr, *UJl = nullptr;  // 2 pcap x ldg
  double *z = nullptr, *z2 = nullptr, *ones = nullptr, *dpart = nullptr;
  void* gws = nullptr;
  size_t gws_bytes = 0;
  int* tc_err = nullptr;
  double *LV = nullptr, *lw = nullptr, *lh = nullptr, *vmin = nullptr;
  int hessvecs = 0, rtr_iters = 0, lz_mv = 0, evals = 0;
  double ms_hv = 0.0;
};

namespace {

template <typename T>
T* calloc_dev(ComplexState* c, size_t n) {
  void* p = nullptr;
  if (n == 0) n = 1;
  if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) throw std::bad_alloc();
  c->allocs.push_back(p);
  return static_cast<T*>(p);
}

void csync(ComplexState* c) { MDS_CUDA(cudaStreamSynchronize(c->s)); }

// Deterministic dot products of up to two pairs of length n; host results.
void cdots(ComplexState* c, size_t n, int k, const double* x0, const double* y0, double* out,
           const double* x1 = nullptr, const double* y1 = nullptr) {
  const double* xs[3] = {x0, x1, nullptr};
  const double* ys[3] = {y0, y1, nullptr};
  launch_dots(n, k, xs, ys, c->dpart, c->s);
  MDS_CUDA(cudaMemcpyAsync(c->hp, c->dpart + 3 * kRedBlocks, k * sizeof(double),
                           cudaMemcpyDeviceToHost, c->s));
  csync(c);
  for (int i = 0; i < k; ++i) out[i] = c->hp[i];
}

// out = Y J = [-B | A] for Y = [A | B] (n x 2p); conj = 1 gives [B | -A] (unused).
__global__ void cplx_rot_kernel(int n, int p, const double* __restrict__ Y, double* __restrict__ out) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t tot = size_t(n) * 2 * p;
  if (i >= tot) return;
  const int row = int(i / (2 * p)), col = int(i % (2 * p));
  const double* y = Y + size_t(row) * 2 * p;
  out[i] = col < p ? -y[p + col] : y[col - p];
}
void launch_rot(int n, int p, const double* Y, double* out, cudaStream_t s) {
  const size_t tot = size_t(n) * 2 * p;
  count_launches(1);
  cplx_rot_kernel<<<unsigned((tot + 255) / 256), 256, 0, s>>>(n, p, Y, out);
  MDS_CUDA(cudaGetLastError());
}

// [A | B] (n x 2p) -> [A, a | B, b] (n x 2(p+1)); a, b (n) may be NULL for zeros.
__global__ void cplx_grow_kernel(int n, int p, const double* __restrict__ Y,
                                 const double* __restrict__ a, const double* __restrict__ b,
                                 double* __restrict__ out) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int q = p + 1;
  const size_t tot = size_t(n) * 2 * q;
  if (i >= tot) return;
  const int row = int(i / (2 * q)), col = int(i % (2 * q));
  const double* y = Y + size_t(row) * 2 * p;
  double v;
  if (col < p)
    v = y[col];
  else if (col == p)
    v = a ? a[row] : 0.0;
  else if (col < 2 * q - 1)
    v = y[p + (col - q)];
  else
    v = b ? b[row] : 0.0;
  out[i] = v;
}
void launch_grow(int n, int p, const double* Y, const double* a, const double* b, double* out,
                 cudaStream_t s) {
  const size_t tot = size_t(n) * 2 * (p + 1);
  count_launches(1);
  cplx_grow_kernel<<<unsigned((tot + 255) / 256), 256, 0, s>>>(n, p, Y, a, b, out);
  MDS_CUDA(cudaGetLastError());
}

// XB = [[Qre, -Qim], [Qim, Qre]] (2n x 2n): the real embedding of Q.
__global__ void cplx_embed_kernel(int n, const double* __restrict__ qre,
                                  const double* __restrict__ qim, double* __restrict__ XB) {
  const size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t n2 = size_t(2) * n;
  if (i >= n2 * n2) return;
  const int r = int(i / n2), c = int(i % n2);
  const int rr = r % n, cc = c % n;
  const size_t e = size_t(rr) * n + cc;
  const bool top = r < n, left = c < n;
  XB[i] = (top == left) ? qre[e] : (top ? -qim[e] : qim[e]);
}

// z2 = [mu; mu]
void dup2(ComplexState* c, const double* z) {
  MDS_CUDA(cudaMemcpyAsync(c->z2, z, c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  MDS_CUDA(cudaMemcpyAsync(c->z2 + c->n, z, c->n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
}

// G = Q Y = Qre Y + Qim (Y J) in FP64; returns f = <Y, G>.
double qy(ComplexState* c, const double* Y, int p, double* G) {
  const int n = c->n, w = 2 * p;
  launch_rot(n, p, Y, c->rot, c->s);
  launch_gemm<double>(n, w, n, c->Qre, n, Y, w, G, w, 1.0, 0.0, nullptr, nullptr, 0.0, nullptr,
                      c->gws, c->gws_bytes, c->s);
  launch_gemm<double>(n, w, n, c->Qim, n, c->rot, w, G, w, 1.0, 1.0, nullptr, nullptr, 0.0,
                      nullptr, c->gws, c->gws_bytes, c->s);
  double f;
  cdots(c, size_t(n) * w, 1, Y, G, &f);
  c->evals++;
  return f;
}

// At Y: G = Q Y, mu = rowdot(G, Y), grad = 2 (G - Diag(mu) Y); returns f and ||grad||.
void point(ComplexState* c, const double* Y, int p, double* f, double* gn) {
  const int n = c->n;
  *f = qy(c, Y, p, c->G);
  launch_rowdot(n, 2 * p, c->G, Y, c->z, c->s);
  launch_grad_from_gy(n, 2 * p, c->G, c->z, Y, c->grad, c->s);
  double gg;
  cdots(c, size_t(n) * 2 * p, 1, c->grad, c->grad, &gg);
  *gn = std::sqrt(gg);
}

// HU = P_Y(2 Q Up) - 2 Diag(mu) Up, Up = P_Y(U), mu = c->z of the last point().
void hessvec(ComplexState* c, const double* Y, const double* U, int p, double* HU, int prec) {
  const int n = c->n, w = 2 * p;
  c->hessvecs++;
  if (prec == MANIDSDP_PREC_MIXED) {
    launch_hv_prep<float>(n, w, Y, U, c->Up, c->Upf, c->Yf, false, c->s);
    launch_rot(n, p, c->Up, c->rot, c->s);
    const int ldg = tcx_ld(n);
    launch_tcx_split_rows(n, w, c->Up, nullptr, nullptr, 0, c->UTh, c->UTl, ldg, c->s);
    launch_tcx_split_rows(n, w, c->rot, nullptr, nullptr, 0, c->UJh, c->UJl, ldg, c->s);
    const int S = launch_tcx_gather(n, w, c->Qh, c->Ql, c->QIh, c->QIl, ldg, c->UTh, c->UTl,
                                    c->UJh, c->UJl, ldg, static_cast<float*>(c->gws),
                                    c->gws_bytes, c->tc_err, c->s);
    launch_hv_epilogue<float>(n, w, S - 1, static_cast<const float*>(c->gws), nullptr, Y, c->Up,
                              c->z, 0.0, HU, c->s);
  } else {
    launch_hv_prep<double>(n, w, Y, U, c->Up, nullptr, nullptr, false, c->s);
    launch_rot(n, p, c->Up, c->rot, c->s);
    launch_gemm<double>(n, w, n, c->Qre, n, c->Up, w, c->Tm, w, 1.0, 0.0, nullptr, nullptr, 0.0,
                        nullptr, c->gws, c->gws_bytes, c->s);
    launch_gemm<double>(n, w, n, c->Qim, n, c->rot, w, c->Tm, w, 1.0, 1.0, nullptr, nullptr, 0.0,
                        nullptr, c->gws, c->gws_bytes, c->s);
    launch_hv_epilogue<double>(n, w, 0, c->Tm, nullptr, Y, c->Up, c->z, 0.0, HU, c->s);
  }
}


struct CLanczos {
  double lo = 0.0, hi = 0.0;
  int steps = 0;
  bool converged = false;
};

// Lanczos with full FP64 reorthogonalisation on the real embedding XB - Diag(z2)
// (2n x 2n); the unit Ritz vector of the smallest Ritz value into c->vmin (2n),
// first entry above 1e-14 in magnitude positive.  Same stopping rule as the
// real certificate check: every 10 steps, smallest pair's residual <= 1e-10 and
// largest's <= 1e-6 of the larger extreme Ritz value.
CLanczos clanczos(ComplexState* c, int kcap, bool want_vec) {
  const int N = 2 * c->n;
  int k = std::min(std::min(kcap, c->kmax), N);
  if (k < 1) k = 1;
  std::vector<double> v0(N);
  double nrm = 0.0;
  for (int i = 0; i < N; ++i) {
    uint64_t x = 0x5EEDull + uint64_t(i) + 0x9E3779B97F4A7C15ull;  // splitmix64
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    v0[i] = (double(x >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
    nrm += v0[i] * v0[i];
  }
  nrm = std::sqrt(nrm);
  for (int i = 0; i < N; ++i) v0[i] /= nrm;
  MDS_CUDA(cudaMemcpyAsync(c->LV, v0.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->s));
  std::vector<double> al, be;
  int steps = k;
  bool conv = false;
  for (int j = 0; j < k; ++j) {
    const double* vj = c->LV + size_t(j) * N;
    launch_gemv_cert(N, c->XB, c->z2, vj, c->lw, c->s);
    c->lz_mv++;
    launch_basis_dots(N, j + 1, c->LV, c->lw, c->lh, c->s);
    MDS_CUDA(cudaMemcpyAsync(c->hp + 8, c->lh + j, sizeof(double), cudaMemcpyDeviceToHost, c->s));
    launch_basis_update(N, j + 1, c->LV, c->lh, c->lw, c->s);
    launch_basis_dots(N, j + 1, c->LV, c->lw, c->lh, c->s);
    launch_basis_update(N, j + 1, c->LV, c->lh, c->lw, c->s);
    double bb;
    cdots(c, N, 1, c->lw, c->lw, &bb);  // synchronises; hp[8] holds alpha_j
    const double alpha = c->hp[8];
    const double beta = std::sqrt(bb);
    al.push_back(alpha);
    if (beta <= 1e-14 * std::max(1.0, std::fabs(alpha)) || j == k - 1) {
      steps = j + 1;
      conv = beta <= 1e-14 * std::max(1.0, std::fabs(alpha)) || j + 1 == N;
      break;
    }
    be.push_back(beta);
    launch_axpby(N, 1.0 / beta, c->lw, 0.0, nullptr, c->LV + size_t(j + 1) * N, c->s);
    if ((j + 1) % 10 == 0) {
      const int kk = j + 1;
      const double tlo = tridiag_eig(al, be, kk, 0), thi = tridiag_eig(al, be, kk, kk - 1);
      const auto slo = tridiag_vec(al, be, kk, tlo, {});
      const auto shi = tridiag_vec(al, be, kk, thi, {});
      const double scale = std::max(std::fabs(tlo), std::fabs(thi)) + 1e-300;
      if (beta * std::fabs(slo[kk - 1]) <= 1e-10 * scale &&
          beta * std::fabs(shi[kk - 1]) <= 1e-6 * scale) {
        steps = kk;
        conv = true;
        break;
      }
    }
  }
  CLanczos out;
  out.steps = steps;
  out.converged = conv;
  std::vector<double> bt(be.begin(), be.begin() + std::max(0, steps - 1));
  std::vector<double> at(al.begin(), al.begin() + steps);
  out.lo = tridiag_eig(at, bt, steps, 0);
  out.hi = tridiag_eig(at, bt, steps, steps - 1);
  if (want_vec) {
    std::vector<double> sv = tridiag_vec(at, bt, steps, out.lo, {});
    MDS_CUDA(cudaMemcpyAsync(c->lh, sv.data(), steps * sizeof(double), cudaMemcpyHostToDevice, c->s));
    MDS_CUDA(cudaMemsetAsync(c->vmin, 0, N * sizeof(double), c->s));
    // basis_update subtracts: vmin = -sum_j (-s_j) v_j
    for (auto& x : sv) x = -x;
    MDS_CUDA(cudaMemcpyAsync(c->lh, sv.data(), steps * sizeof(double), cudaMemcpyHostToDevice, c->s));
    launch_basis_update(N, steps, c->LV, c->lh, c->vmin, c->s);
    std::vector<double> hv(N);
    MDS_CUDA(cudaMemcpyAsync(hv.data(), c->vmin, N * sizeof(double), cudaMemcpyDeviceToHost, c->s));
    csync(c);
    double sgn = 1.0;
    for (int t = 0; t < N; ++t)
      if (std::fabs(hv[t]) > 1e-14) {
        sgn = hv[t] < 0 ? -1.0 : 1.0;
        break;
      }
    if (sgn < 0) launch_axpby(N, -1.0, c->vmin, 0.0, nullptr, c->vmin, c->s);
  }
  csync(c);
  return out;
}

// Truncated CG (Steihaug-Toint) on the model at c->Y (gradient c->grad); the
// same stopping rules as the real path's host loop.
int ctcg(ComplexState* c, int p, double Delta, int max_tcg, bool* boundary) {
  const size_t n = size_t(c->n) * 2 * p;
  const int prec = c->prm.precision_mode;
  MDS_CUDA(cudaMemsetAsync(c->eta, 0, n * sizeof(double), c->s));
  MDS_CUDA(cudaMemsetAsync(c->Heta, 0, n * sizeof(double), c->s));
  MDS_CUDA(cudaMemcpyAsync(c->r, c->grad, n * sizeof(double), cudaMemcpyDeviceToDevice, c->s));
  launch_axpby(n, -1.0, c->grad, 0.0, nullptr, c->delta, c->s);
  double rr;
  cdots(c, n, 1, c->r, c->r, &rr);
  const double r0 = std::sqrt(rr);
  double ee = 0.0, ed = 0.0, dd = rr;
  const double target = r0 * std::max(std::min(r0, 0.1), c->prm.tcg_floor);
  *boundary = false;
  for (int j = 1; j <= max_tcg; ++j) {
    hessvec(c, c->Y, c->delta, p, c->Hd, prec);
    double kap;
    cdots(c, n, 1, c->delta, c->Hd, &kap);
    const double alpha = kap != 0.0 ? rr / kap : INFINITY;
    const double ee_new = ee + 2.0 * alpha * ed + alpha * alpha * dd;
    if (kap <= 0.0 || ee_new >= Delta * Delta) {
      const double tau = (-ed + std::sqrt(ed * ed + dd * (Delta * Delta - ee))) / dd;
      launch_axpby(n, tau, c->delta, 1.0, c->eta, c->eta, c->s);
      launch_axpby(n, tau, c->Hd, 1.0, c->Heta, c->Heta, c->s);
      *boundary = true;
      return j;
    }
    launch_axpby(n, alpha, c->delta, 1.0, c->eta, c->eta, c->s);
    launch_axpby(n, alpha, c->Hd, 1.0, c->Heta, c->Heta, c->s);
    launch_axpby(n, alpha, c->Hd, 1.0, c->r, c->r, c->s);
    ee = ee_new;
    double rr_new;
    cdots(c, n, 1, c->r, c->r, &rr_new);
    if (std::sqrt(rr_new) <= target) return j;
    const double beta = rr_new / rr;
    rr = rr_new;
    launch_axpby(n, -1.0, c->r, beta, c->delta, c->delta, c->s);
    ed = beta * (ed + alpha * dd);
    dd = rr + beta * beta * dd;
  }
  return max_tcg;
}

// Riemannian trust region from c->Y to ||grad|| <= tol_grad; leaves G, z, grad at
// the final point.  Returns the cost.
double crtr(ComplexState* c, int p, double tol_grad, int max_rtr, int max_tcg, double* gn_out) {
  const int n = c->n;
  const size_t np = size_t(n) * 2 * p;
  const double Delta_bar = M_PI * std::sqrt(double(n));
  double Delta = Delta_bar / 8.0;
  double fx, gn;
  point(c, c->Y, p, &fx, &gn);
  for (int it = 0; it < max_rtr && gn > tol_grad; ++it) {
    bool bnd = false;
    ctcg(c, p, Delta, max_tcg, &bnd);
    double d2[2];
    cdots(c, np, 2, c->grad, c->eta, d2, c->eta, c->Heta);
    const double model_dec = -(d2[0] + 0.5 * d2[1]);
    launch_retract(n, 2 * p, c->Y, c->eta, 1.0, c->Yt, c->s);
    const double f_new = qy(c, c->Yt, p, c->tmp);
    if (!std::isfinite(f_new)) throw DeviceError{cudaErrorUnknown};
    const double reg = std::max(1.0, std::fabs(fx)) * 1e3 * 2.220446049250313e-16;
    const double rho = (model_dec + reg > 0.0) ? (fx - f_new + reg) / (model_dec + reg) : -INFINITY;
    if (rho < 0.25)
      Delta /= 4.0;
    else if (rho > 0.75 && bnd)
      Delta = std::min(2.0 * Delta, Delta_bar);
    c->rtr_iters++;
    if (rho > 0.1) {
      std::swap(c->Y, c->Yt);
      point(c, c->Y, p, &fx, &gn);
    }
  }
  *gn_out = gn;
  return fx;
}

int cguard(const std::function<int()>& f) {
  try {
    return f();
  } catch (const DeviceError&) {
    return MANIDSDP_E_CUDA;
  } catch (const std::bad_alloc&) {
    return MANIDSDP_E_NOMEM;
  }
}

}  // namespace

int complex_setup(ComplexState** out, int n, const double* qre, const double* qim,
                  const manidsdp_params& prm, cudaStream_t s) {
  auto* c = new ComplexState();
  const int st = cguard([&]() -> int {
    c->n = n;
    c->s = s;
    c->prm = prm;
    c->pcap = std::min(prm.p_max, kMaxP / 2);
    MDS_CUDA(cudaMallocHost(&c->hp, 32 * sizeof(double)));
    const size_t nn = size_t(n) * n;
    c->Qre = calloc_dev<double>(c, nn);
    c->Qim = calloc_dev<double>(c, nn);
    MDS_CUDA(cudaMemcpyAsync(c->Qre, qre, nn * sizeof(double), cudaMemcpyDefault, s));
    if (qim != nullptr)
      MDS_CUDA(cudaMemcpyAsync(c->Qim, qim, nn * sizeof(double), cudaMemcpyDefault, s));
    else
      MDS_CUDA(cudaMemsetAsync(c->Qim, 0, nn * sizeof(double), s));
    const size_t n2 = size_t(2) * n;
    c->XB = calloc_dev<double>(c, n2 * n2);
    count_launches(1);
    cplx_embed_kernel<<<unsigned((n2 * n2 + 255) / 256), 256, 0, s>>>(n, c->Qre, c->Qim, c->XB);
    MDS_CUDA(cudaGetLastError());
    // FP32 copies, then TF32 pairs for the tensor-core Hess-vec
    const int ldg = tcx_ld(n);
    float* f32 = calloc_dev<float>(c, nn);
    float** pr[] = {&c->Qh, &c->Ql, &c->QIh, &c->QIl};
    for (float** q : pr) *q = calloc_dev<float>(c, size_t(n) * ldg);
    launch_to_float(nn, c->Qre, f32, s);
    launch_tcx_split_matrix(n, f32, nullptr, nullptr, 0.f, c->Qh, c->Ql, ldg, s);
    launch_to_float(nn, c->Qim, f32, s);
    launch_tcx_split_matrix(n, f32, nullptr, nullptr, 0.f, c->QIh, c->QIl, ldg, s);
    const size_t np = size_t(n) * 2 * c->pcap;
    double** d[] = {&c->Y, &c->Yt, &c->G, &c->grad, &c->eta, &c->Heta, &c->r, &c->delta,
                    &c->Hd, &c->Up, &c->U, &c->tmp, &c->rot, &c->Tm};
    for (double** q : d) *q = calloc_dev<double>(c, np);
    c->Upf = calloc_dev<float>(c, np);
    c->Yf = calloc_dev<float>(c, np);
    const size_t pn = size_t(2 * c->pcap) * ldg;
    float** tp[] = {&c->UTh, &c->UTl, &c->UJh, &c->UJl};
    for (float** q : tp) *q = calloc_dev<float>(c, pn);
    c->z = calloc_dev<double>(c, n);
    c->z2 = calloc_dev<double>(c, n2);
    c->ones = calloc_dev<double>(c, n);
    {
      std::vector<double> one_h(n, 1.0);
      MDS_CUDA(cudaMemcpyAsync(c->ones, one_h.data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
      csync(c);
    }
    c->dpart = calloc_dev<double>(c, 3 * kRedBlocks + 3);
    c->gws_bytes = std::max((np + size_t(2) * 304 * 4096) * sizeof(double),
                            size_t(tcx_gather_splits(n) + 1) * np * sizeof(float));
    c->gws = calloc_dev<double>(c, c->gws_bytes / sizeof(double));
    c->tc_err = calloc_dev<int>(c, 1);
    MDS_CUDA(cudaMemsetAsync(c->tc_err, 0, sizeof(int), s));
    c->kmax = std::min(std::max(prm.lanczos_k, 1), int(n2));
    c->LV = calloc_dev<double>(c, size_t(c->kmax + 1) * n2);
    c->lh = calloc_dev<double>(c, c->kmax + 1);
    c->lw = calloc_dev<double>(c, n2);
    c->vmin = calloc_dev<double>(c, n2);
    csync(c);
    return MANIDSDP_OK;
  });
  if (st != MANIDSDP_OK) {
    complex_destroy(c);
    return st;
  }
  *out = c;
  return MANIDSDP_OK;
}

void complex_destroy(ComplexState* c) {
  if (c == nullptr) return;
  for (void* p : c->allocs) cudaFree(p);
  if (c->hp) cudaFreeHost(c->hp);
  delete c;
}

int complex_set_params(ComplexState* c, const manidsdp_params& prm) {
  if (prm.p_max != c->prm.p_max) return MANIDSDP_E_ARG;
  c->prm = prm;
  c->kmax = std::min(std::min(std::max(prm.lanczos_k, 1), c->kmax), 2 * c->n);
  return MANIDSDP_OK;
}

int complex_eval(ComplexState* c, const double* Y, int p, double* psi, double* rgrad, double* z) {
  if (p < 1 || p > c->pcap) return MANIDSDP_E_ARG;
  return cguard([&]() -> int {
    const size_t np = size_t(c->n) * 2 * p;
    MDS_CUDA(cudaMemcpyAsync(c->Y, Y, np * sizeof(double), cudaMemcpyDefault, c->s));
    double f, gn;
    point(c, c->Y, p, &f, &gn);
    if (psi) *psi = f;
    if (rgrad) MDS_CUDA(cudaMemcpyAsync(rgrad, c->grad, np * sizeof(double), cudaMemcpyDefault, c->s));
    if (z) MDS_CUDA(cudaMemcpyAsync(z, c->z, c->n * sizeof(double), cudaMemcpyDefault, c->s));
    csync(c);
    return MANIDSDP_OK;
  });
}

int complex_hessvec(ComplexState* c, const double* Y, const double* U, int p, double* HU,
                    int precision) {
  if (p < 1 || p > c->pcap) return MANIDSDP_E_ARG;
  return cguard([&]() -> int {
    const size_t np = size_t(c->n) * 2 * p;
    MDS_CUDA(cudaMemcpyAsync(c->Yt, Y, np * sizeof(double), cudaMemcpyDefault, c->s));
    MDS_CUDA(cudaMemcpyAsync(c->U, U, np * sizeof(double), cudaMemcpyDefault, c->s));
    double f, gn;
    point(c, c->Yt, p, &f, &gn);  // mu at Y
    hessvec(c, c->Yt, c->U, p, c->Hd, precision);
    MDS_CUDA(cudaMemcpyAsync(HU, c->Hd, np * sizeof(double), cudaMemcpyDefault, c->s));
    int e = 0;
    MDS_CUDA(cudaMemcpyAsync(&e, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    csync(c);
    return e ? MANIDSDP_E_TIMEOUT : MANIDSDP_OK;
  });
}

int complex_lanczos(ComplexState* c, const double* Y, int p, int which, int k, double* lambda,
                    double* v, int* steps) {
  if (p < 1 || p > c->pcap) return MANIDSDP_E_ARG;
  return cguard([&]() -> int {
    const size_t np = size_t(c->n) * 2 * p;
    MDS_CUDA(cudaMemcpyAsync(c->Yt, Y, np * sizeof(double), cudaMemcpyDefault, c->s));
    double f, gn;
    point(c, c->Yt, p, &f, &gn);
    dup2(c, c->z);
    CLanczos lz = clanczos(c, k > 0 ? k : c->prm.lanczos_k, v != nullptr);
    *lambda = which == MANIDSDP_EIG_MIN ? lz.lo : lz.hi;
    if (v) MDS_CUDA(cudaMemcpyAsync(v, c->vmin, 2 * c->n * sizeof(double), cudaMemcpyDefault, c->s));
    if (steps) *steps = lz.steps;
    csync(c);
    return MANIDSDP_OK;
  });
}

// The rank-adaptive trust region of the complex relaxation (the real path's
// Algorithm 1 with R = 0: no multiplier or sigma updates): RTR to
// ||grad|| <= tol_grad_min (at most 500 iterations, tCG at most 1000 products);
// then the certificate; if lambda_min < -neg_tol (1 + |lambda_max|) and p < p_max,
// one column is appended along [0, v] with backtracking from t = sqrt(n).  Stops at
// max(eta_d, eta_g) <= tol on a converged Lanczos run.
int complex_solve(ComplexState* c, const double* Y0, int p0, double* Y_out, int* p_out,
                  double* z_out, manidsdp_report* report) {
  if (Y0 == nullptr || p0 < 1 || p0 > c->pcap) return MANIDSDP_E_ARG;
  int status = MANIDSDP_E_NOCONV;
  manidsdp_report rep{};
  const int gst = cguard([&]() -> int {
    const manidsdp_params& P = c->prm;
    const int n = c->n;
    c->hessvecs = c->rtr_iters = c->lz_mv = c->evals = 0;
    int p = p0;
    MDS_CUDA(cudaMemcpyAsync(c->tmp, Y0, size_t(n) * 2 * p * sizeof(double), cudaMemcpyDefault, c->s));
    launch_retract(n, 2 * p, c->tmp, c->tmp, 0.0, c->Y, c->s);
    for (int k = 0; k < P.max_outer; ++k) {
      double gn;
      const double f = crtr(c, p, P.tol_grad_min, 500, 1000, &gn);
      double smu;  // sum(mu): the dual objective
      cdots(c, n, 1, c->z, c->ones, &smu);
      dup2(c, c->z);
      CLanczos lz = clanczos(c, P.lanczos_k, true);
      rep.eta_p = 0.0;
      rep.eta_d = std::max(0.0, -lz.lo) / (1.0 + std::fabs(lz.hi));
      rep.eta_g = std::fabs(f - smu) / (1.0 + std::fabs(f) + std::fabs(smu));
      rep.value = f;
      rep.pobj = smu;
      rep.lambda_min = lz.lo;
      rep.lambda_max = lz.hi;
      rep.outer = k + 1;
      rep.p = p;
      if (P.verbose)
        std::fprintf(stderr, "[manidsdp-c] k=%d p=%d f=%.12f gnorm=%.2e eta=(%.2e %.2e) lmin=%.3e lz=%d%s\n",
                     k, p, f, gn, rep.eta_d, rep.eta_g, lz.lo, lz.steps, lz.converged ? "" : " (unconverged)");
      if (std::max(rep.eta_d, rep.eta_g) <= P.tol && lz.converged) {
        status = MANIDSDP_OK;
        break;
      }
      if (lz.lo >= -P.neg_tol * (1.0 + std::fabs(lz.hi)) || p >= c->pcap) continue;
      // append a column along [0, v]: v = a + ib from the embedding's eigenvector [a; b]
      launch_grow(n, p, c->Y, nullptr, nullptr, c->tmp, c->s);
      MDS_CUDA(cudaMemsetAsync(c->rot, 0, size_t(n) * 2 * p * sizeof(double), c->s));
      launch_grow(n, p, c->rot, c->vmin, c->vmin + n, c->U, c->s);  // U = [0, v]
      std::swap(c->Y, c->tmp);
      ++p;
      double f0, g0;
      point(c, c->Y, p, &f0, &g0);
      const double curv = 2.0 * lz.lo;  // 2 v^H X v with |v| = 1
      double t = std::sqrt(double(n));
      for (int i = 0; i < 40; ++i) {
        launch_retract(n, 2 * p, c->Y, c->U, t, c->Yt, c->s);
        const double ft = qy(c, c->Yt, p, c->tmp);
        if (ft <= f0 - 1e-4 * 0.5 * t * t * std::fabs(curv)) {
          std::swap(c->Y, c->Yt);
          break;
        }
        t *= 0.5;
      }
    }
    rep.hessvecs = c->hessvecs;
    rep.rtr_iters = c->rtr_iters;
    rep.lanczos_matvecs = c->lz_mv;
    rep.evals = c->evals;
    rep.status = status;
    if (Y_out) MDS_CUDA(cudaMemcpyAsync(Y_out, c->Y, size_t(n) * 2 * rep.p * sizeof(double), cudaMemcpyDefault, c->s));
    if (p_out) *p_out = rep.p;
    if (z_out) MDS_CUDA(cudaMemcpyAsync(z_out, c->z, n * sizeof(double), cudaMemcpyDefault, c->s));
    int e = 0;
    MDS_CUDA(cudaMemcpyAsync(&e, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    csync(c);
    return e ? MANIDSDP_E_TIMEOUT : MANIDSDP_OK;
  });
  if (report) *report = rep;
  if (gst != MANIDSDP_OK) return gst;
  return status;
}

}  // namespace mds

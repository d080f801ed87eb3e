// Extreme eigenpair of a caller-held dense symmetric matrix without any device
// allocation: manidsdp_lanczos_dense_noalloc.  The paper has no counterpart.
//
// It runs Lanczos with full FP64 reorthogonalisation on X - Diag(d), with the
// iteration, stopping rules and kernels of manidsdp_lanczos, but on a matrix the
// caller passes in and with the Krylov basis in one static device array instead
// of a context's workspace.  Nothing here calls cudaMalloc, cudaFree or a library
// that allocates, and the host side keeps its tridiagonal data in fixed arrays.
//
// Scratch state: nothing in the array has to be zero at entry.  Every region
// is written before it is read; the zero diagonal used when d is NULL and the
// accumulator of the Ritz vector are cleared by each call.  All calls on one
// device share the array, so two calls in flight at once on that device (from
// two streams or two host threads) overwrite each other's basis.
#include <cmath>
#include <cstring>

#include "common.cuh"

using namespace mds;

namespace {

// Limits of the static scratch: N <= 16384, k <= 256 Lanczos steps, and the
// Krylov basis k x N FP64 within 4 MiB (k * N <= 524288).
constexpr int kNaMaxN = 16384;
constexpr int kNaMaxK = 256;
constexpr size_t kNaBasis = size_t(1) << 19;
// basis | w (N) | zero diagonal (N) | Ritz vector (N) | h (k + 1) | pad
constexpr size_t kNaDoubles = kNaBasis + 3 * size_t(kNaMaxN) + kNaMaxK + 64;

static __device__ __align__(256) double g_na_scratch[kNaDoubles];

// Device address of the scratch in the current device's context.  In host code
// g_na_scratch names a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress on every call: after a cudaDeviceReset, or when the
// primary context is destroyed and created again, the module is loaded anew and
// the array may sit elsewhere, so a cached address could point at freed or
// foreign memory.  The lookup allocates nothing; the first one on a device loads
// the library's module there.
int na_scratch(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return MANIDSDP_E_CUDA;
  }
  *out = static_cast<double*>(p);
  return MANIDSDP_OK;
}

// The Lanczos start vector: entry i is splitmix64(0x5EED + i) mapped to
// [-1, 1) (Steele, Lea, Flood 2014); normalised afterwards.
__device__ __forceinline__ unsigned long long na_splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void na_start_kernel(int N, double* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned long long u = na_splitmix64(0x5EEDull + (unsigned long long)i);
  v[i] = (double(u >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}
// v /= sqrt(*nn)
__global__ void na_normalise_kernel(int N, const double* __restrict__ nn, double* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) v[i] /= sqrt(nn[0]);
}
// out = sign * w, sign making the first entry with |w_i| > 1e-14 positive.
__global__ void __launch_bounds__(256) na_sign_kernel(int N, const double* __restrict__ w,
                                                      double* __restrict__ out) {
  __shared__ int first[256];
  int f = N;
  for (int i = threadIdx.x; i < N; i += 256)
    if (fabs(w[i]) > 1e-14) {
      f = i;
      break;
    }
  first[threadIdx.x] = f;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) first[threadIdx.x] = min(first[threadIdx.x], first[threadIdx.x + st]);
    __syncthreads();
  }
  const double sgn = (first[0] < N && w[first[0]] < 0.0) ? -1.0 : 1.0;
  for (int i = threadIdx.x; i < N; i += 256) out[i] = sgn * w[i];
}

// ---- symmetric tridiagonal T (diagonal a[0..k-1], off-diagonal b[0..k-2]) ----
int na_sturm_below(const double* a, const double* b, int k, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < k; ++i) {
    const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0) ++cnt;
  }
  return cnt;
}
// i-th smallest eigenvalue (0-based): bisection on Sturm counts inside the
// Gershgorin interval.
double na_tridiag_eig(const double* a, const double* b, int k, int i) {
  double lo = a[0], hi = a[0];
  for (int j = 0; j < k; ++j) {
    const double r = (j > 0 ? std::fabs(b[j - 1]) : 0.0) + (j < k - 1 ? std::fabs(b[j]) : 0.0);
    lo = std::fmin(lo, a[j] - r);
    hi = std::fmax(hi, a[j] + r);
  }
  const double scale = std::fmax(std::fabs(lo), std::fabs(hi)) + 1e-300;
  for (int it = 0; it < 200 && hi - lo > 1e-17 * scale; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (na_sturm_below(a, b, k, mid) > i)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}
// Unit eigenvector x of T for the eigenvalue theta: four steps of inverse
// iteration, T - theta I factored as L U without pivoting (tiny pivots lifted).
void na_tridiag_vec(const double* a, const double* b, int k, double theta, double* x) {
  double l[kNaMaxK], d[kNaMaxK];
  double tn = 0.0;
  for (int j = 0; j < k; ++j)
    tn = std::fmax(tn, std::fabs(a[j]) + (j < k - 1 ? std::fabs(b[j]) : 0.0));
  const double tiny = 1e-14 * (tn + 1e-300);
  for (int j = 0; j < k; ++j) x[j] = 1.0 + 0.01 * ((j * 7919) % 101);
  for (int it = 0; it < 4; ++it) {
    d[0] = a[0] - theta;
    if (std::fabs(d[0]) < tiny) d[0] = tiny;
    for (int j = 1; j < k; ++j) {
      l[j] = b[j - 1] / d[j - 1];
      d[j] = (a[j] - theta) - l[j] * b[j - 1];
      if (std::fabs(d[j]) < tiny) d[j] = tiny;
    }
    for (int j = 1; j < k; ++j) x[j] -= l[j] * x[j - 1];
    x[k - 1] /= d[k - 1];
    for (int j = k - 2; j >= 0; --j) x[j] = (x[j] - b[j] * x[j + 1]) / d[j];
    double nrm = 0.0;
    for (int j = 0; j < k; ++j) nrm += x[j] * x[j];
    nrm = std::sqrt(nrm);
    for (int j = 0; j < k; ++j) x[j] /= nrm;
  }
}

// True when the current device can read p: its own device memory, managed
// memory, or registered host memory (pageable host memory is rejected).
bool na_device_readable(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged ||
         (a.type == cudaMemoryTypeHost && a.devicePointer != nullptr);
}

// One device double to the host (the copy into pageable host memory returns
// once it has landed; the synchronisation makes that explicit).
void na_read(const double* src, double* dst, cudaStream_t s) {
  MDS_CUDA(cudaMemcpyAsync(dst, src, sizeof(double), cudaMemcpyDeviceToHost, s));
  MDS_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

extern "C" {

int manidsdp_lanczos_dense_noalloc(int32_t N, const double* X, const double* d, int32_t which,
                                   int32_t k, double* lambda, double* v, int32_t* steps_out,
                                   void* stream) {
  if (N < 1 || X == nullptr || lambda == nullptr ||
      (which != MANIDSDP_EIG_MIN && which != MANIDSDP_EIG_MAX))
    return MANIDSDP_E_ARG;
  if (k <= 0) k = N < 64 ? N : 64;
  if (k > N) k = N;
  if (N > kNaMaxN || k > kNaMaxK || size_t(k) * size_t(N) > kNaBasis) return MANIDSDP_E_TOOLARGE;
  if (!na_device_readable(X) || (d != nullptr && !na_device_readable(d))) return MANIDSDP_E_ARG;
  double* scratch = nullptr;
  const int st = na_scratch(&scratch);
  if (st != MANIDSDP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    double* V = scratch;                    // k x N Krylov basis
    double* w = V + kNaBasis;               // N
    double* zero = w + kNaMaxN;             // N, the diagonal when d is NULL
    double* ritz = zero + kNaMaxN;          // N, the returned vector
    double* h = ritz + kNaMaxN;             // k + 1
    const double* dg = d;
    if (dg == nullptr) {
      MDS_CUDA(cudaMemsetAsync(zero, 0, size_t(N) * sizeof(double), s));
      dg = zero;
    }
    count_launches(1);
    na_start_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, V);
    MDS_CUDA(cudaGetLastError());
    launch_basis_dots(N, 1, V, V, h + kNaMaxK, s);
    count_launches(1);
    na_normalise_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, h + kNaMaxK, V);
    MDS_CUDA(cudaGetLastError());

    double al[kNaMaxK], be[kNaMaxK];
    int n_al = 0;
    int steps = k;
    for (int j = 0; j < k; ++j) {
      const double* vj = V + size_t(j) * N;
      launch_gemv_cert(N, X, dg, vj, w, s);
      launch_basis_dots(N, j + 1, V, w, h, s);
      double alpha;
      na_read(h + j, &alpha, s);
      launch_basis_update(N, j + 1, V, h, w, s);
      launch_basis_dots(N, j + 1, V, w, h, s);
      launch_basis_update(N, j + 1, V, h, w, s);
      launch_basis_dots(N, 1, w, w, h + kNaMaxK, s);
      double bb;
      na_read(h + kNaMaxK, &bb, s);
      if (!std::isfinite(alpha) || !std::isfinite(bb)) return MANIDSDP_E_NONFINITE;
      const double beta = std::sqrt(bb);
      al[n_al++] = alpha;
      if (beta <= 1e-14 * std::fmax(1.0, std::fabs(alpha)) || j == k - 1) {
        steps = j + 1;
        break;
      }
      be[j] = beta;
      launch_axpby(N, 1.0 / beta, w, 0.0, nullptr, V + size_t(j + 1) * N, s);
      if ((j + 1) % 10 == 0) {  // the extreme Ritz pairs' residuals every 10 steps
        const int kk = j + 1;
        double sv[kNaMaxK];
        const double tlo = na_tridiag_eig(al, be, kk, 0);
        const double thi = na_tridiag_eig(al, be, kk, kk - 1);
        const double scale = std::fmax(std::fabs(tlo), std::fabs(thi)) + 1e-300;
        na_tridiag_vec(al, be, kk, tlo, sv);
        const double res_lo = beta * std::fabs(sv[kk - 1]);
        na_tridiag_vec(al, be, kk, thi, sv);
        const double res_hi = beta * std::fabs(sv[kk - 1]);
        // the requested end of the spectrum to 1e-10, the other (a scale) to 1e-6
        const double tol_lo = which == MANIDSDP_EIG_MIN ? 1e-10 : 1e-6;
        const double tol_hi = which == MANIDSDP_EIG_MIN ? 1e-6 : 1e-10;
        if (res_lo <= tol_lo * scale && res_hi <= tol_hi * scale) {
          steps = kk;
          break;
        }
      }
    }
    const int kk = steps;
    const double theta = na_tridiag_eig(al, be, kk, which == MANIDSDP_EIG_MIN ? 0 : kk - 1);
    if (v != nullptr) {
      double sv[kNaMaxK];
      na_tridiag_vec(al, be, kk, theta, sv);
      for (int j = 0; j < kk; ++j) sv[j] = -sv[j];
      MDS_CUDA(cudaMemcpyAsync(h, sv, size_t(kk) * sizeof(double), cudaMemcpyHostToDevice, s));
      MDS_CUDA(cudaMemsetAsync(w, 0, size_t(N) * sizeof(double), s));
      launch_basis_update(N, kk, V, h, w, s);  // w = sum_j s_j v_j
      count_launches(1);
      na_sign_kernel<<<1, 256, 0, s>>>(N, w, ritz);
      MDS_CUDA(cudaGetLastError());
      MDS_CUDA(cudaMemcpyAsync(v, ritz, size_t(N) * sizeof(double), cudaMemcpyDefault, s));
    }
    MDS_CUDA(cudaStreamSynchronize(s));
    *lambda = theta;
    if (steps_out) *steps_out = steps;
    return MANIDSDP_OK;
  } catch (const DeviceError&) {
    return MANIDSDP_E_CUDA;
  }
}

}  // extern "C"

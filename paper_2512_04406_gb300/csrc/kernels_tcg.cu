// Truncated CG (Steihaug-Toint; the textbook RTR inner solver of Section 4) run
// entirely on the device: the step-size, boundary, negative-curvature and
// residual tests are evaluated by single-block kernels that also set the
// condition of a CUDA-graph WHILE node, so one graph launch runs the whole tCG.
//
// One iteration (graph body):
//   prep      delta = -r + beta delta;  Up = P_Y(delta)            (Lemma 4.1)
//   means     w = (AA*)^{-1} A(Y Up' + Up Y')                       (Section 3)
//   gemm      T = G Up - sigma A*(w) Y  (split-K partials)
//   gram2     [Up'Y; Y'Y]
//   epilogue  Hd = Hess[Up] (Eq. (4.7)) and partials of <delta, Hd>
//   alpha     kappa, alpha, boundary / negative-curvature decision
//   update    eta += step delta; Heta += step Hd; r += alpha Hd; partials of <r, r>
//   beta      convergence test, beta, recurrences for <eta,eta>, <eta,delta>,
//             <delta,delta>; sets the WHILE condition
#include "common.cuh"

namespace mds {

// tCG scalars in device memory.
struct TcgState {
  double rr, ee, ed, dd;      // <r,r>, <eta,eta>, <eta,delta>, <delta,delta>
  double delta2, target;      // trust radius squared, residual target
  double alpha, beta, step, ee_new;
  int flag;                   // 0 running, 1 converged, 2 boundary, 3 negative curvature, 4 max
  int iters, max_iters, pad;
};

__global__ void tcg_init_kernel(TcgState* st, const double* __restrict__ rr0, double delta,
                                double target_rel_floor, double abs_target, int max_iters) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double rr = rr0[0];
  const double r0 = sqrt(rr);
  double rel = fmin(r0, 0.1);  // min(||r0||^theta, kappa) with theta = 1, kappa = 0.1
  rel = fmax(rel, target_rel_floor);
  st->rr = rr;
  st->ee = 0.0;
  st->ed = 0.0;
  st->dd = rr;
  st->delta2 = delta * delta;
  st->target = fmax(r0 * rel, abs_target);
  st->alpha = st->beta = st->step = st->ee_new = 0.0;
  st->flag = 0;
  st->iters = 0;
  st->max_iters = max_iters;
}

// delta = -r + beta delta, Up = P_Y(delta), UpT = T(Up); one warp per row.
template <typename T>
__global__ void tcg_prep_kernel(int N, int p, const TcgState* __restrict__ st,
                                const double* __restrict__ Y, const double* __restrict__ r,
                                double* __restrict__ delta, double* __restrict__ Up,
                                T* __restrict__ UpT) {
  const int lane = threadIdx.x % 32;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (row >= N) return;
  const double beta = st->beta;
  const size_t o = size_t(row) * p;
  double d = 0.0;
  for (int c = lane; c < p; c += 32) {
    const double dl = fma(beta, delta[o + c], -r[o + c]);
    delta[o + c] = dl;
    d = fma(dl, Y[o + c], d);
  }
  for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
  for (int c = lane; c < p; c += 32) {
    const double up = fma(-d, Y[o + c], delta[o + c]);
    Up[o + c] = up;
    if (UpT != nullptr) UpT[o + c] = T(up);
  }
}

// Hessian epilogue (as hv_epilogue_kernel) plus per-block partials of <delta, Hd>.
// M == nullptr: the slice `splits` of part already holds sigma (Y M1 + Up M2), so
// Ht = 2 * (sum of splits + 1 slices).
template <typename T>
__global__ void __launch_bounds__(256) tcg_epilogue_kernel(
    int N, int p, int splits, const T* __restrict__ part, const T* __restrict__ M,
    const double* __restrict__ Y, const double* __restrict__ Up, const double* __restrict__ z,
    double sigma, const double* __restrict__ delta, double* __restrict__ Hd,
    double* __restrict__ kpart) {
  __shared__ double red[8];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  double kap = 0.0;
  if (row < N) {
    const size_t o = size_t(row) * p;
    const size_t np = size_t(N) * p;
    const T* M1 = M;
    const T* M2 = M + size_t(p) * p;
    constexpr int MAXC = 16;  // columns per lane held in registers (p <= 512)
    double ht[MAXC];
    double d = 0.0;
#pragma unroll
    for (int t = 0; t < MAXC; ++t) {
      const int c = lane + 32 * t;
      ht[t] = 0.0;
      if (c < p) {
        T tv = T(0);
        for (int zz = 0; zz < splits; ++zz) tv += part[zz * np + o + c];
        if (M == nullptr) {
          ht[t] = 2.0 * (double(tv) + double(part[size_t(splits) * np + o + c]));
        } else {
          T ym = T(0);
          for (int k = 0; k < p; ++k) {
            ym = fma(T(Y[o + k]), M1[size_t(k) * p + c], ym);
            ym = fma(T(Up[o + k]), M2[size_t(k) * p + c], ym);
          }
          ht[t] = 2.0 * double(tv) + 2.0 * sigma * double(ym);
        }
        d = fma(ht[t], Y[o + c], d);
      }
    }
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    const double zz2 = 2.0 * z[row];
#pragma unroll
    for (int t = 0; t < MAXC; ++t) {
      const int c = lane + 32 * t;
      if (c < p) {
        const double h = ht[t] - d * Y[o + c] - zz2 * Up[o + c];
        Hd[o + c] = h;
        kap = fma(h, delta[o + c], kap);
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) kap += __shfl_xor_sync(0xffffffffu, kap, off);
  if (lane == 0) red[warp] = kap;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    kpart[blockIdx.x] = s;
  }
}

// kappa = sum of the partials; alpha; boundary / negative-curvature step.
__global__ void __launch_bounds__(256) tcg_alpha_kernel(int nparts, const double* __restrict__ kpart,
                                                        TcgState* st) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) s += kpart[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double kap = red[0];
  const double alpha = kap != 0.0 ? st->rr / kap : INFINITY;
  const double ee_new = st->ee + 2.0 * alpha * st->ed + alpha * alpha * st->dd;
  st->alpha = alpha;
  st->ee_new = ee_new;
  if (kap <= 0.0 || ee_new >= st->delta2) {
    const double ed = st->ed, dd = st->dd, ee = st->ee;
    st->step = (-ed + sqrt(ed * ed + dd * (st->delta2 - ee))) / dd;
    st->flag = kap <= 0.0 ? 3 : 2;
  } else {
    st->step = alpha;
  }
}

// eta += step delta; Heta += step Hd; r += alpha Hd (interior step); partials of <r, r>.
__global__ void __launch_bounds__(256) tcg_update_kernel(size_t n, const TcgState* __restrict__ st,
                                                         const double* __restrict__ delta,
                                                         const double* __restrict__ Hd,
                                                         double* __restrict__ eta,
                                                         double* __restrict__ Heta,
                                                         double* __restrict__ r,
                                                         double* __restrict__ rpart) {
  __shared__ double red[256];
  const double step = st->step;
  const bool interior = st->flag == 0;
  const double alpha = st->alpha;
  double acc = 0.0;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const double h = Hd[i];
    eta[i] = fma(step, delta[i], eta[i]);
    Heta[i] = fma(step, h, Heta[i]);
    if (interior) {
      const double rv = fma(alpha, h, r[i]);
      r[i] = rv;
      acc = fma(rv, rv, acc);
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) rpart[blockIdx.x] = red[0];
}

// Residual test, beta and the recurrences; sets the WHILE condition.
__global__ void __launch_bounds__(256) tcg_beta_kernel(int nparts, const double* __restrict__ rpart,
                                                       TcgState* st,
                                                       cudaGraphConditionalHandle handle) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 256) s += rpart[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  st->iters += 1;
  unsigned int go = 0;
  if (st->flag == 0) {
    const double rr_new = red[0];
    if (sqrt(rr_new) <= st->target) {
      st->flag = 1;
    } else if (st->iters >= st->max_iters) {
      st->flag = 4;
    } else {
      const double beta = rr_new / st->rr;
      const double alpha = st->alpha;
      st->ee = st->ee_new;
      st->ed = beta * (st->ed + alpha * st->dd);
      st->rr = rr_new;
      st->dd = rr_new + beta * beta * st->dd;
      st->beta = beta;
      go = 1;
    }
  }
  cudaGraphSetConditional(handle, go);
}

// ---- launchers --------------------------------------------------------------------
size_t tcg_state_bytes() { return sizeof(TcgState); }

void launch_tcg_init(void* st, const double* rr0, double delta, double floor_rel, double abs_target,
                     int max_iters, cudaStream_t s) {
  count_launches(1);
  tcg_init_kernel<<<1, 32, 0, s>>>(static_cast<TcgState*>(st), rr0, delta, floor_rel, abs_target,
                                   max_iters);
  MDS_CUDA(cudaGetLastError());
}

int tcg_epilogue_blocks(int N) { return (N * 32 + 255) / 256; }
int tcg_update_blocks() { return kRedBlocks; }

template <typename T>
void launch_tcg_prep(int N, int p, const void* st, const double* Y, const double* r, double* delta,
                     double* Up, T* UpT, cudaStream_t s) {
  count_launches(1);
  tcg_prep_kernel<T><<<(N * 32 + 255) / 256, 256, 0, s>>>(
      N, p, static_cast<const TcgState*>(st), Y, r, delta, Up, UpT);
  MDS_CUDA(cudaGetLastError());
}
template void launch_tcg_prep<double>(int, int, const void*, const double*, const double*, double*,
                                      double*, double*, cudaStream_t);
template void launch_tcg_prep<float>(int, int, const void*, const double*, const double*, double*,
                                     double*, float*, cudaStream_t);

template <typename T>
void launch_tcg_epilogue(int N, int p, int splits, const T* part, const T* M, const double* Y,
                         const double* Up, const double* z, double sigma, const double* delta,
                         double* Hd, double* kpart, cudaStream_t s) {
  count_launches(1);
  tcg_epilogue_kernel<T><<<tcg_epilogue_blocks(N), 256, 0, s>>>(N, p, splits, part, M, Y, Up, z,
                                                                sigma, delta, Hd, kpart);
  MDS_CUDA(cudaGetLastError());
}
template void launch_tcg_epilogue<double>(int, int, int, const double*, const double*,
                                          const double*, const double*, const double*, double,
                                          const double*, double*, double*, cudaStream_t);
template void launch_tcg_epilogue<float>(int, int, int, const float*, const float*, const double*,
                                         const double*, const double*, double, const double*,
                                         double*, double*, cudaStream_t);

void launch_tcg_alpha(int nparts, const double* kpart, void* st, cudaStream_t s) {
  count_launches(1);
  tcg_alpha_kernel<<<1, 256, 0, s>>>(nparts, kpart, static_cast<TcgState*>(st));
  MDS_CUDA(cudaGetLastError());
}

void launch_tcg_update(size_t n, const void* st, const double* delta, const double* Hd,
                       double* eta, double* Heta, double* r, double* rpart, cudaStream_t s) {
  count_launches(1);
  tcg_update_kernel<<<kRedBlocks, 256, 0, s>>>(n, static_cast<const TcgState*>(st), delta, Hd, eta,
                                               Heta, r, rpart);
  MDS_CUDA(cudaGetLastError());
}

void launch_tcg_beta(int nparts, const double* rpart, void* st, cudaGraphConditionalHandle h,
                     cudaStream_t s) {
  count_launches(1);
  tcg_beta_kernel<<<1, 256, 0, s>>>(nparts, rpart, static_cast<TcgState*>(st), h);
  MDS_CUDA(cudaGetLastError());
}

// flag, iters of the state (host copy through a pinned buffer)
void tcg_read_state(const void* st, int* flag, int* iters, void* pinned, cudaStream_t s) {
  MDS_CUDA(cudaMemcpyAsync(pinned, st, sizeof(TcgState), cudaMemcpyDeviceToHost, s));
  MDS_CUDA(cudaStreamSynchronize(s));
  const TcgState* h = static_cast<const TcgState*>(pinned);
  *flag = h->flag;
  *iters = h->iters;
}

}  // namespace mds

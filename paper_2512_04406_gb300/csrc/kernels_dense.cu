// Dense and row-local kernels of the subproblem (Section 4):
//   G Y and G U (Proposition 4.2) as a tiled split-K GEMM that can also add the
//   moment matrix A*(w) applied to a second operand (the Q(W) Y term of the
//   Hessian), Gram matrices Y'Y and U'Y, the row-local Hessian epilogue
//   (Eq. (4.7)), the tangent projector (Lemma 4.1), the row-normalising
//   retraction, deterministic reductions, and the Lanczos helpers for the
//   certificate X = Xt + D - Diag(z) (Algorithm 1, step 9).
#include <algorithm>

#include "common.cuh"

namespace mds {

// ---- GEMM ------------------------------------------------------------------
// Block tile BM x BN, thread tile TM x TN, K chunk BK; grid.z splits K.  With
// GATHER the A operand gets a second part gscale * w[idx[r, k]] paired with B2.
template <typename T, int BM, int BN, int TM, int TN, bool GATHER>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) gemm_kernel(
    int M, int ncol, int K, int kchunk, const T* __restrict__ A, int lda, const T* __restrict__ B,
    int ldb, const int32_t* __restrict__ idx, const T* __restrict__ w, T gscale,
    const T* __restrict__ B2, T* __restrict__ out_part) {
  constexpr int BK = 16;
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];
  __shared__ T Ws[GATHER ? BK : 1][GATHER ? BM + 1 : 1];
  __shared__ T B2s[GATHER ? BK : 1][GATHER ? BN : 1];
  const int tx = threadIdx.x % (BN / TN), ty = threadIdx.x / (BN / TN);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  for (int k0 = kb; k0 < ke; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += NT) {
      const int r = t / BK, kk = t % BK;
      const int gr = m0 + r, gk = k0 + kk;
      const bool ok = gr < M && gk < ke;
      As[kk][r] = ok ? A[size_t(gr) * lda + gk] : T(0);
      if (GATHER) Ws[kk][r] = ok ? gscale * w[idx[size_t(gr) * K + gk]] : T(0);
    }
    for (int t = threadIdx.x; t < BK * BN; t += NT) {
      const int kk = t / BN, c = t % BN;
      const int gk = k0 + kk, gc = n0 + c;
      const bool ok = gk < ke && gc < ncol;
      Bs[kk][c] = ok ? B[size_t(gk) * ldb + gc] : T(0);
      if (GATHER) B2s[kk][c] = ok ? B2[size_t(gk) * ldb + gc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      if (GATHER) {
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = Ws[kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bb[j] = B2s[kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  T* op = out_part + size_t(blockIdx.z) * M * ncol;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = m0 + ty * TM + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = n0 + tx * TN + j;
      if (c < ncol) op[size_t(r) * ncol + c] = acc[i][j];
    }
  }
}

// out = alpha * sum_z part[z] + beta * out, in ascending z.
template <typename T>
__global__ void splitk_reduce_kernel(int M, int ncol, int splits, const T* __restrict__ part,
                                     T* __restrict__ out, int ldc, T alpha, T beta) {
  const size_t n = size_t(M) * ncol;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    T s = T(0);
    for (int z = 0; z < splits; ++z) s += part[size_t(z) * n + i];
    const int r = int(i / ncol), c = int(i % ncol);
    T* o = out + size_t(r) * ldc + c;
    *o = (beta == T(0)) ? alpha * s : fma(alpha, s, beta * *o);
  }
}

template <typename T, int BM, int BN, int TM, int TN>
static int gemm_cfg(int M, int ncol, int K, const T* A, int lda, const T* B, int ldb, T* out,
                    int ldc, T alpha, T beta, const int32_t* idx, const T* w, T gscale,
                    const T* B2, void* ws, size_t ws_bytes, cudaStream_t s, bool partial_only) {
  const int gx = (ncol + BN - 1) / BN, gy = (M + BM - 1) / BM;
  int splits = (2 * 152 + gx * gy - 1) / (gx * gy);
  const int max_splits = (K + 63) / 64;
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  const size_t need = size_t(splits) * M * ncol * sizeof(T);
  if (need > ws_bytes) {
    splits = int(ws_bytes / (size_t(M) * ncol * sizeof(T)));
    if (splits < 1) throw DeviceError{cudaErrorMemoryAllocation};
  }
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + 15) / 16 * 16;
  splits = (K + kchunk - 1) / kchunk;
  T* part = static_cast<T*>(ws);
  dim3 grid(gx, gy, splits);
  constexpr int NT = (BM / TM) * (BN / TN);
  count_launches(partial_only ? 1 : 2);
  if (idx != nullptr)
    gemm_kernel<T, BM, BN, TM, TN, true><<<grid, NT, 0, s>>>(M, ncol, K, kchunk, A, lda, B, ldb,
                                                             idx, w, gscale, B2, part);
  else
    gemm_kernel<T, BM, BN, TM, TN, false><<<grid, NT, 0, s>>>(M, ncol, K, kchunk, A, lda, B, ldb,
                                                              nullptr, nullptr, T(0), nullptr,
                                                              part);
  if (!partial_only) {
    const size_t n = size_t(M) * ncol;
    int rb = int((n + 255) / 256);
    if (rb > 4096) rb = 4096;
    splitk_reduce_kernel<T><<<rb, 256, 0, s>>>(M, ncol, splits, part, out, ldc, alpha, beta);
  }
  MDS_CUDA(cudaGetLastError());
  return splits;
}

template <typename T>
static int gemm_any(int M, int ncol, int K, const T* A, int lda, const T* B, int ldb, T* out,
                    int ldc, T alpha, T beta, const int32_t* idx, const T* w, T gscale,
                    const T* B2, void* ws, size_t ws_bytes, cudaStream_t s, bool partial_only) {
  if (M <= 0 || ncol <= 0) return 0;
  if (ncol <= 8)
    return gemm_cfg<T, 128, 8, 4, 1>(M, ncol, K, A, lda, B, ldb, out, ldc, alpha, beta, idx, w,
                                     gscale, B2, ws, ws_bytes, s, partial_only);
  if (ncol <= 32)
    return gemm_cfg<T, 64, 32, 4, 2>(M, ncol, K, A, lda, B, ldb, out, ldc, alpha, beta, idx, w,
                                     gscale, B2, ws, ws_bytes, s, partial_only);
  return gemm_cfg<T, 64, 64, 4, 4>(M, ncol, K, A, lda, B, ldb, out, ldc, alpha, beta, idx, w,
                                   gscale, B2, ws, ws_bytes, s, partial_only);
}

template <typename T>
void launch_gemm(int M, int ncol, int K, const T* A, int lda, const T* B, int ldb, T* out, int ldc,
                 T alpha, T beta, const int32_t* idx, const T* w, T gscale, const T* B2,
                 void* ws, size_t ws_bytes, cudaStream_t s) {
  gemm_any<T>(M, ncol, K, A, lda, B, ldb, out, ldc, alpha, beta, idx, w, gscale, B2, ws, ws_bytes,
              s, false);
}

template <typename T>
int launch_gemm_partials(int M, int ncol, int K, const T* A, int lda, const T* B, int ldb,
                         const int32_t* idx, const T* w, T gscale, const T* B2, void* ws,
                         size_t ws_bytes, cudaStream_t s) {
  return gemm_any<T>(M, ncol, K, A, lda, B, ldb, nullptr, ncol, T(1), T(0), idx, w, gscale, B2, ws,
                     ws_bytes, s, true);
}
template int launch_gemm_partials<double>(int, int, int, const double*, int, const double*, int,
                                          const int32_t*, const double*, double, const double*,
                                          void*, size_t, cudaStream_t);
template int launch_gemm_partials<float>(int, int, int, const float*, int, const float*, int,
                                         const int32_t*, const float*, float, const float*, void*,
                                         size_t, cudaStream_t);

template void launch_gemm<double>(int, int, int, const double*, int, const double*, int, double*,
                                  int, double, double, const int32_t*, const double*, double,
                                  const double*, void*, size_t, cudaStream_t);
template void launch_gemm<float>(int, int, int, const float*, int, const float*, int, float*, int,
                                 float, float, const int32_t*, const float*, float, const float*,
                                 void*, size_t, cudaStream_t);

// ---- Gram: out = A' B ----------------------------------------------------------
// grid.z splits the N rows; each block writes its 16 x 16 partial tile, and a
// second kernel sums the splits in ascending order (deterministic).
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(int N, int p1, int p2, int rows_per_split,
                                                   const T* __restrict__ A,
                                                   const T* __restrict__ B, T* __restrict__ part) {
  constexpr int RC = 32;
  __shared__ T As[RC][17];
  __shared__ T Bs[RC][17];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
  const int nb = blockIdx.z * rows_per_split;
  const int ne = min(N, nb + rows_per_split);
  T acc = T(0);
  for (int n0 = nb; n0 < ne; n0 += RC) {
    for (int t = threadIdx.x; t < RC * 16; t += 256) {
      const int rr = t / 16, cc = t % 16;
      const int n = n0 + rr;
      As[rr][cc] = (n < ne && i0 + cc < p1) ? A[size_t(n) * p1 + i0 + cc] : T(0);
      Bs[rr][cc] = (n < ne && j0 + cc < p2) ? B[size_t(n) * p2 + j0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < RC; ++rr) acc = fma(As[rr][ty], Bs[rr][tx], acc);
    __syncthreads();
  }
  if (i0 + ty < p1 && j0 + tx < p2)
    part[size_t(blockIdx.z) * p1 * p2 + size_t(i0 + ty) * p2 + j0 + tx] = acc;
}

// Gram matrices A' B over N rows (A, B: N x p): 64 x 64 output tile per block,
// 4 x 4 outputs per thread, rows staged 32 at a time; grid.z splits the rows and
// each split writes its partial tile (summed in ascending order afterwards).
// With two=true, blockIdx.y >= gy computes A2' B into the second p x p slot.
template <typename T>
__global__ void __launch_bounds__(256) gram2_kernel(int N, int p, int gy, int rows_per_split,
                                                    const T* __restrict__ A1,
                                                    const T* __restrict__ A2,
                                                    const T* __restrict__ B, int nmat,
                                                    T* __restrict__ part) {
  constexpr int RC = 32;
  __shared__ T As[RC][65];
  __shared__ T Bs[RC][65];
  const int which = blockIdx.y >= gy ? 1 : 0;
  const T* A = which ? A2 : A1;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = (blockIdx.y - which * gy) * 64, j0 = blockIdx.x * 64;
  const int nb = blockIdx.z * rows_per_split;
  const int ne = min(N, nb + rows_per_split);
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int n0 = nb; n0 < ne; n0 += RC) {
    for (int t = threadIdx.x; t < RC * 64; t += 256) {
      const int rr = t / 64, cc = t % 64;
      const int n = n0 + rr;
      As[rr][cc] = (n < ne && i0 + cc < p) ? A[size_t(n) * p + i0 + cc] : T(0);
      Bs[rr][cc] = (n < ne && j0 + cc < p) ? B[size_t(n) * p + j0 + cc] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < RC; ++rr) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[rr][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[rr][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = i0 + ty + 16 * i;
    if (r >= p) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = j0 + tx + 16 * j;
      if (cc < p)
        part[(size_t(blockIdx.z) * nmat + which) * p * p + size_t(r) * p + cc] = acc[i][j];
    }
  }
}

template <typename T>
__global__ void gram_reduce_kernel(int n, int splits, const T* __restrict__ part,
                                   T* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T s = T(0);
  for (int z = 0; z < splits; ++z) s += part[size_t(z) * n + i];
  out[i] = s;
}

template <typename T>
void launch_gram(int N, int p1, int p2, const T* A, const T* B, T* out, void* ws,
                 size_t ws_bytes, cudaStream_t s) {
  const int gx = (p2 + 15) / 16, gy = (p1 + 15) / 16;
  int splits = (2 * 152 + gx * gy - 1) / (gx * gy);
  splits = std::min(splits, (N + 63) / 64);
  const size_t per = size_t(p1) * p2 * sizeof(T);
  if (size_t(splits) * per > ws_bytes) splits = int(ws_bytes / per);
  if (splits < 1) splits = 1;
  int rows = (N + splits - 1) / splits;
  rows = (rows + 31) / 32 * 32;
  splits = (N + rows - 1) / rows;
  if (splits < 1) splits = 1;
  dim3 grid(gx, gy, splits);
  count_launches(2);
  gram_kernel<T><<<grid, 256, 0, s>>>(N, p1, p2, rows, A, B, static_cast<T*>(ws));
  const int n = p1 * p2;
  gram_reduce_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(n, splits, static_cast<T*>(ws), out);
  MDS_CUDA(cudaGetLastError());
}
template void launch_gram<double>(int, int, int, const double*, const double*, double*, void*,
                                  size_t, cudaStream_t);

// out[0 : p*p] = A1' B and, when A2 != nullptr, out[p*p : 2*p*p] = A2' B.
template <typename T>
void launch_gram2(int N, int p, const T* A1, const T* A2, const T* B, T* out, void* ws,
                  size_t ws_bytes, cudaStream_t s) {
  const int nmat = A2 != nullptr ? 2 : 1;
  const int gx = (p + 63) / 64, gy = (p + 63) / 64;
  int splits = (2 * 152 + nmat * gx * gy - 1) / (nmat * gx * gy);
  // FP32 (the tCG Hess-vec, where this Gram is on the critical path): splits of 32 rows
  splits = std::min(splits, sizeof(T) == 4 ? (N + 31) / 32 : (N + 63) / 64);
  const size_t per = size_t(nmat) * p * p * sizeof(T);
  if (size_t(splits) * per > ws_bytes) splits = int(ws_bytes / per);
  if (splits < 1) splits = 1;
  int rows = (N + splits - 1) / splits;
  rows = (rows + 31) / 32 * 32;
  splits = (N + rows - 1) / rows;
  if (splits < 1) splits = 1;
  dim3 grid(gx, nmat * gy, splits);
  count_launches(2);
  gram2_kernel<T><<<grid, 256, 0, s>>>(N, p, gy, rows, A1, A2, B, nmat, static_cast<T*>(ws));
  const int n = nmat * p * p;
  gram_reduce_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(n, splits, static_cast<T*>(ws), out);
  MDS_CUDA(cudaGetLastError());
}
template void launch_gram2<double>(int, int, const double*, const double*, const double*, double*,
                                   void*, size_t, cudaStream_t);
template void launch_gram2<float>(int, int, const float*, const float*, const float*, float*,
                                  void*, size_t, cudaStream_t);
template void launch_gram<float>(int, int, int, const float*, const float*, float*, void*, size_t,
                                 cudaStream_t);

// ---- row-local kernels: one warp per row ---------------------------------------
template <typename T>
__global__ void hess_epilogue_kernel(int N, int p, const T* __restrict__ Tm,
                                     const T* __restrict__ YM, const T* __restrict__ Y,
                                     const T* __restrict__ U, const double* __restrict__ z,
                                     double sigma, double* __restrict__ HU) {
  const int lane = threadIdx.x % 32;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (row >= N) return;  // whole warp exits together
  const size_t o = size_t(row) * p;
  double d = 0.0;
  for (int c = lane; c < p; c += 32) {
    const double ht = 2.0 * double(Tm[o + c]) + 2.0 * sigma * double(YM[o + c]);
    d = fma(ht, double(Y[o + c]), d);
  }
  for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
  const double zz = 2.0 * z[row];
  for (int c = lane; c < p; c += 32) {
    const double ht = 2.0 * double(Tm[o + c]) + 2.0 * sigma * double(YM[o + c]);
    HU[o + c] = ht - d * double(Y[o + c]) - zz * double(U[o + c]);
  }
}

template <typename T>
void launch_hess_epilogue(int N, int p, const T* Tm, const T* YM, const T* Y, const T* U,
                          const double* z, double sigma, double* HU, cudaStream_t s) {
  const int blocks = (N * 32 + 255) / 256;
  count_launches(1);
  hess_epilogue_kernel<T><<<blocks, 256, 0, s>>>(N, p, Tm, YM, Y, U, z, sigma, HU);
  MDS_CUDA(cudaGetLastError());
}
template void launch_hess_epilogue<double>(int, int, const double*, const double*, const double*,
                                           const double*, const double*, double, double*,
                                           cudaStream_t);
template void launch_hess_epilogue<float>(int, int, const float*, const float*, const float*,
                                          const float*, const double*, double, double*,
                                          cudaStream_t);

// Hessian prologue: Up = P_Y(U) in FP64; UpT = T(Up); YT = T(Y) when write_y.
template <typename T>
__global__ void hv_prep_kernel(int N, int p, const double* __restrict__ Y,
                               const double* __restrict__ U, double* __restrict__ Up,
                               T* __restrict__ UpT, T* __restrict__ YT, int write_y) {
  const int lane = threadIdx.x % 32;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (row >= N) return;
  const size_t o = size_t(row) * p;
  double d = 0.0;
  for (int c = lane; c < p; c += 32) d = fma(U[o + c], Y[o + c], d);
  for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
  for (int c = lane; c < p; c += 32) {
    const double up = fma(-d, Y[o + c], U[o + c]);
    Up[o + c] = up;
    if (UpT != nullptr) UpT[o + c] = T(up);
    if (write_y) YT[o + c] = T(Y[o + c]);
  }
}

template <typename T>
void launch_hv_prep(int N, int p, const double* Y, const double* U, double* Up, T* UpT, T* YT,
                    bool write_y, cudaStream_t s) {
  count_launches(1);
  hv_prep_kernel<T><<<(N * 32 + 255) / 256, 256, 0, s>>>(N, p, Y, U, Up, UpT, YT, write_y ? 1 : 0);
  MDS_CUDA(cudaGetLastError());
}
template void launch_hv_prep<double>(int, int, const double*, const double*, double*, double*,
                                     double*, bool, cudaStream_t);
template void launch_hv_prep<float>(int, int, const double*, const double*, double*, float*,
                                    float*, bool, cudaStream_t);

// Hessian epilogue with the split-K sum of T = G U - sigma A*(w) Y and the Gram
// products folded in:  Ht = 2 T + 2 sigma (Y M1 + Up M2),
// HU = Ht - (Ht . Y_b) Y_b - 2 z_b Up_b   (Eq. (4.7)); M = [M1; M2] (2 p x p).
template <typename T>
__global__ void hv_epilogue_kernel(int N, int p, int splits, const T* __restrict__ part,
                                   const T* __restrict__ M, const double* __restrict__ Y,
                                   const double* __restrict__ Up, const double* __restrict__ z,
                                   double sigma, double* __restrict__ HU) {
  const int lane = threadIdx.x % 32;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (row >= N) return;
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
    if (c < p) HU[o + c] = ht[t] - d * Y[o + c] - zz2 * Up[o + c];
  }
}

template <typename T>
void launch_hv_epilogue(int N, int p, int splits, const T* part, const T* M, const double* Y,
                        const double* Up, const double* z, double sigma, double* HU,
                        cudaStream_t s) {
  count_launches(1);
  hv_epilogue_kernel<T><<<(N * 32 + 255) / 256, 256, 0, s>>>(N, p, splits, part, M, Y, Up, z,
                                                            sigma, HU);
  MDS_CUDA(cudaGetLastError());
}
template void launch_hv_epilogue<double>(int, int, int, const double*, const double*,
                                         const double*, const double*, const double*, double,
                                         double*, cudaStream_t);
template void launch_hv_epilogue<float>(int, int, int, const float*, const float*, const double*,
                                        const double*, const double*, double, double*,
                                        cudaStream_t);

// MODE 0: out = U - (U.Y) Y ; MODE 1: out = (Y + t E) / ||Y + t E|| ; MODE 2: out[row] = A.B
template <int MODE>
__global__ void rowop_kernel(int N, int p, const double* __restrict__ Y,
                             const double* __restrict__ E, double t, double* __restrict__ out) {
  const int lane = threadIdx.x % 32;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (row >= N) return;
  const size_t o = size_t(row) * p;
  double d = 0.0;
  for (int c = lane; c < p; c += 32) {
    if (MODE == 1) {
      const double v = fma(t, E[o + c], Y[o + c]);
      d = fma(v, v, d);
    } else {
      d = fma(E[o + c], Y[o + c], d);
    }
  }
  for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
  if (MODE == 2) {
    if (lane == 0) out[row] = d;
    return;
  }
  if (MODE == 1) {
    const double inv = 1.0 / sqrt(d);
    for (int c = lane; c < p; c += 32) out[o + c] = fma(t, E[o + c], Y[o + c]) * inv;
  } else {
    for (int c = lane; c < p; c += 32) out[o + c] = fma(-d, Y[o + c], E[o + c]);
  }
}

void launch_retract(int N, int p, const double* Y, const double* E, double t, double* out,
                    cudaStream_t s) {
  count_launches(1);
  rowop_kernel<1><<<(N * 32 + 255) / 256, 256, 0, s>>>(N, p, Y, E, t, out);
  MDS_CUDA(cudaGetLastError());
}
void launch_rowdot(int N, int p, const double* A, const double* B, double* out, cudaStream_t s) {
  count_launches(1);
  rowop_kernel<2><<<(N * 32 + 255) / 256, 256, 0, s>>>(N, p, B, A, 0.0, out);
  MDS_CUDA(cudaGetLastError());
}

__global__ void grad_kernel(int N, int p, const double* __restrict__ GY,
                            const double* __restrict__ z, const double* __restrict__ Y,
                            double* __restrict__ g) {
  const size_t n = size_t(N) * p;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    g[i] = 2.0 * fma(-z[i / p], Y[i], GY[i]);
}
void launch_grad_from_gy(int N, int p, const double* GY, const double* z, const double* Y,
                         double* grad, cudaStream_t s) {
  const size_t n = size_t(N) * p;
  int b = int((n + 255) / 256);
  if (b > 8192) b = 8192;
  count_launches(1);
  grad_kernel<<<b, 256, 0, s>>>(N, p, GY, z, Y, grad);
  MDS_CUDA(cudaGetLastError());
}

__global__ void to_float_kernel(size_t n, const double* __restrict__ a, float* __restrict__ o) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    o[i] = float(a[i]);
}
static int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return int(b > 8192 ? 8192 : (b == 0 ? 1 : b));
}
void launch_to_float(size_t n, const double* a, float* out, cudaStream_t s) {
  count_launches(1);
  to_float_kernel<<<grid_for(n), 256, 0, s>>>(n, a, out);
  MDS_CUDA(cudaGetLastError());
}

__global__ void axpby_kernel(size_t n, double a, const double* __restrict__ x, double b,
                             const double* __restrict__ y, double* __restrict__ o) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    o[i] = (y == nullptr) ? a * x[i] : fma(a, x[i], b * y[i]);
}
void launch_axpby(size_t n, double a, const double* x, double b, const double* y, double* out,
                  cudaStream_t s) {
  count_launches(1);
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, a, x, b, y, out);
  MDS_CUDA(cudaGetLastError());
}

// ---- deterministic dot products ------------------------------------------------
struct DotArgs {
  const double* x[3];
  const double* y[3];
};
__global__ void __launch_bounds__(kRedThreads) dots_kernel(size_t n, int npairs, DotArgs a,
                                                           double* __restrict__ part) {
  __shared__ double red[3][kRedThreads];
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < npairs) acc[k] = fma(a.x[k][i], a.y[k][i], acc[k]);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < npairs; ++k) part[k * kRedBlocks + blockIdx.x] = red[k][0];
}
__global__ void dots_final_kernel(int npairs, int nb, const double* __restrict__ part,
                                  double* __restrict__ out) {
  __shared__ double red[kRedThreads];
  for (int k = 0; k < npairs; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += kRedThreads) s += part[k * kRedBlocks + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = red[0];
    __syncthreads();
  }
}
// part must hold 3 * kRedBlocks doubles followed by 3 output slots.
void launch_dots(size_t n, int npairs, const double* const* xs, const double* const* ys,
                 double* part, cudaStream_t s) {
  DotArgs a;
  for (int k = 0; k < 3; ++k) {
    a.x[k] = k < npairs ? xs[k] : nullptr;
    a.y[k] = k < npairs ? ys[k] : nullptr;
  }
  size_t nbz = (n + kRedThreads - 1) / kRedThreads;
  const int nb = int(nbz < size_t(kRedBlocks) ? (nbz == 0 ? 1 : nbz) : kRedBlocks);
  count_launches(1);
  dots_kernel<<<nb, kRedThreads, 0, s>>>(n, npairs, a, part);
  count_launches(1);
  dots_final_kernel<<<1, kRedThreads, 0, s>>>(npairs, nb, part, part + 3 * kRedBlocks);
  MDS_CUDA(cudaGetLastError());
}

// ---- certificate helpers ----------------------------------------------------------
__global__ void xd_kernel(size_t NN, int mode, const double* __restrict__ in,
                          const int32_t* __restrict__ idx, const double* __restrict__ bm,
                          double* __restrict__ out) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < NN;
       i += size_t(gridDim.x) * blockDim.x)
    out[i] = mode == 0 ? in[i] + bm[idx[i]] : in[i] - bm[idx[i]];
}
void launch_xd_from_xt(size_t NN, int mode, const double* in, const int32_t* idx, const double* bm,
                       double* out, cudaStream_t s) {
  count_launches(1);
  xd_kernel<<<grid_for(NN), 256, 0, s>>>(NN, mode, in, idx, bm, out);
  MDS_CUDA(cudaGetLastError());
}

// w = XD v - z o v, one warp per row
__global__ void gemv_cert_kernel(int N, const double* __restrict__ XD,
                                 const double* __restrict__ z, const double* __restrict__ v,
                                 double* __restrict__ w) {
  const int lane = threadIdx.x % 32;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (row >= N) return;
  const double* a = XD + size_t(row) * N;
  double s = 0.0;
  for (int c = lane; c < N; c += 32) s = fma(a[c], v[c], s);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) w[row] = fma(-z[row], v[row], s);
}
void launch_gemv_cert(int N, const double* XD, const double* z, const double* v, double* w,
                      cudaStream_t s) {
  count_launches(1);
  gemv_cert_kernel<<<(N * 32 + 255) / 256, 256, 0, s>>>(N, XD, z, v, w);
  MDS_CUDA(cudaGetLastError());
}

// h[j] = V_j . w  (V is k x N, one block per j)
__global__ void __launch_bounds__(256) basis_dots_kernel(int N, const double* __restrict__ V,
                                                         const double* __restrict__ w,
                                                         double* __restrict__ h) {
  __shared__ double red[256];
  const double* vj = V + size_t(blockIdx.x) * N;
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += 256) s = fma(vj[i], w[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) h[blockIdx.x] = red[0];
}
void launch_basis_dots(int N, int k, const double* V, const double* w, double* h,
                       cudaStream_t s) {
  if (k <= 0) return;
  count_launches(1);
  basis_dots_kernel<<<k, 256, 0, s>>>(N, V, w, h);
  MDS_CUDA(cudaGetLastError());
}
// w[i] -= sum_j h[j] V[j, i]
__global__ void basis_update_kernel(int N, int k, const double* __restrict__ V,
                                    const double* __restrict__ h, double* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double s = 0.0;
  for (int j = 0; j < k; ++j) s = fma(h[j], V[size_t(j) * N + i], s);
  w[i] -= s;
}
void launch_basis_update(int N, int k, const double* V, const double* h, double* w,
                         cudaStream_t s) {
  if (k <= 0) return;
  count_launches(1);
  basis_update_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, k, V, h, w);
  MDS_CUDA(cudaGetLastError());
}

__global__ void sign_kernel(int n, const double* __restrict__ u, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = u[i] < 0.0 ? -1.0 : 1.0;
}
void launch_sign(int n, const double* u, double* out, cudaStream_t s) {
  count_launches(1);
  sign_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, u, out);
  MDS_CUDA(cudaGetLastError());
}

__global__ void pad_cols_kernel(int N, int p_old, int p_new, const double* __restrict__ in,
                                double* __restrict__ out) {
  const size_t n = size_t(N) * p_new;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const int r = int(i / p_new), c = int(i % p_new);
    out[i] = c < p_old ? in[size_t(r) * p_old + c] : 0.0;
  }
}
void launch_pad_cols(int N, int p_old, int p_new, const double* in, double* out, cudaStream_t s) {
  count_launches(1);
  pad_cols_kernel<<<grid_for(size_t(N) * p_new), 256, 0, s>>>(N, p_old, p_new, in, out);
  MDS_CUDA(cudaGetLastError());
}
__global__ void set_cols_kernel(int N, int p, int c0, int nc, const double* __restrict__ src,
                                double* __restrict__ out) {
  const size_t n = size_t(N) * nc;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const int r = int(i / nc), c = int(i % nc);
    out[size_t(r) * p + c0 + c] = src[i];
  }
}
void launch_set_cols(int N, int p, int c0, int nc, const double* src, double* out,
                     cudaStream_t s) {
  count_launches(1);
  set_cols_kernel<<<grid_for(size_t(N) * nc), 256, 0, s>>>(N, p, c0, nc, src, out);
  MDS_CUDA(cudaGetLastError());
}

}  // namespace mds

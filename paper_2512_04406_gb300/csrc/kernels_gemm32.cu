// FP32 gather GEMM of the Hessian-vector product (Proposition 4.2):
//   T = G U - sigma A*(w) Y  = [G | -sigma A*(w)] [U ; Y]
// where A*(w)[b, g] = w[idx[b, g]] is gathered on the fly from the index map.
// Block tile 128 x BN, K slab of 8, thread tile 8 x TN (256 threads), the next
// slab's global loads prefetched into registers while the current one is
// consumed; grid.z splits K, each split writing its partial product.
#include "common.cuh"

namespace mds {

template <int BN, int TN>
__global__ void __launch_bounds__(256) gemm32_kernel(int N, int ncol, int kchunk,
                                                     const float* __restrict__ G,
                                                     const float* __restrict__ U,
                                                     const int32_t* __restrict__ idx,
                                                     const float* __restrict__ w, float gscale,
                                                     const float* __restrict__ Y,
                                                     float* __restrict__ part) {
  constexpr int BM = 128, BK = 8, TM = 8;
  constexpr int TX = BN / TN;  // threads along columns
  static_assert(TX * (BM / TM) == 256, "256 threads");
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Ws[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  __shared__ __align__(16) float B2s[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * kchunk, ke = min(N, kb + kchunk);
  // A-tile loader: thread loads row (tid >> 1), columns (tid & 1) * 4 .. +3 of the slab
  const int ar = tid >> 1, ac = (tid & 1) * 4;
  const int grow = m0 + ar;
  // B-tile loader: BK x BN elements, 256 threads
  constexpr int BLOADS = (BK * BN + 255) / 256;
  float ra[4], rw[4], rb[BLOADS], rb2[BLOADS];
  auto load = [&](int k0) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int gk = k0 + ac + t;
      const bool ok = grow < N && gk < ke;
      const size_t e = size_t(grow) * N + gk;
      ra[t] = ok ? G[e] : 0.f;
      rw[t] = ok ? gscale * w[idx[e]] : 0.f;
    }
#pragma unroll
    for (int t = 0; t < BLOADS; ++t) {
      const int li = tid + t * 256;
      const int kk = li / BN, c = li % BN;
      const int gk = k0 + kk, gc = n0 + c;
      const bool ok = li < BK * BN && gk < ke && gc < ncol;
      rb[t] = ok ? U[size_t(gk) * ncol + gc] : 0.f;
      rb2[t] = ok ? Y[size_t(gk) * ncol + gc] : 0.f;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      As[ac + t][ar] = ra[t];
      Ws[ac + t][ar] = rw[t];
    }
#pragma unroll
    for (int t = 0; t < BLOADS; ++t) {
      const int li = tid + t * 256;
      if (li < BK * BN) {
        Bs[li / BN][li % BN] = rb[t];
        B2s[li / BN][li % BN] = rb2[t];
      }
    }
  };
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  if (kb < ke) load(kb);
  for (int k0 = kb; k0 < ke; k0 += BK) {
    __syncthreads();
    store();
    __syncthreads();
    if (k0 + BK < ke) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], aw[TM], b[TN], b2[TN];
      const float4* pa = reinterpret_cast<const float4*>(&As[kk][ty * TM]);
      const float4* pw = reinterpret_cast<const float4*>(&Ws[kk][ty * TM]);
#pragma unroll
      for (int v = 0; v < TM / 4; ++v) {
        const float4 x = pa[v], y = pw[v];
        a[4 * v] = x.x; a[4 * v + 1] = x.y; a[4 * v + 2] = x.z; a[4 * v + 3] = x.w;
        aw[4 * v] = y.x; aw[4 * v + 1] = y.y; aw[4 * v + 2] = y.z; aw[4 * v + 3] = y.w;
      }
      if (TN % 4 == 0) {
        const float4* pb = reinterpret_cast<const float4*>(&Bs[kk][tx * TN]);
        const float4* pb2 = reinterpret_cast<const float4*>(&B2s[kk][tx * TN]);
#pragma unroll
        for (int v = 0; v < TN / 4; ++v) {
          const float4 x = pb[v], y = pb2[v];
          b[4 * v] = x.x; b[4 * v + 1] = x.y; b[4 * v + 2] = x.z; b[4 * v + 3] = x.w;
          b2[4 * v] = y.x; b2[4 * v + 1] = y.y; b2[4 * v + 2] = y.z; b2[4 * v + 3] = y.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          b[j] = Bs[kk][tx * TN + j];
          b2[j] = B2s[kk][tx * TN + j];
        }
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], fmaf(aw[i], b2[j], acc[i][j]));
    }
  }
  float* op = part + size_t(blockIdx.z) * N * ncol;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = m0 + ty * TM + i;
    if (r >= N) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = n0 + tx * TN + j;
      if (c < ncol) op[size_t(r) * ncol + c] = acc[i][j];
    }
  }
}

// out[r, c] = scale * sum_k (Y[r, k] M1[k, c] + Up[r, k] M2[k, c]) for the
// Q(W) Y = Y (U'Y) + U (Y'Y) part of the Hessian (Proposition 4.2); M = [M1; M2]
// (2p x p).  32 x 64 output tile per block, 2 x 4 per thread, K chunks of 16.
__global__ void __launch_bounds__(256) ym_kernel(int N, int p, const float* __restrict__ Y,
                                                 const float* __restrict__ Up,
                                                 const float* __restrict__ M, float scale,
                                                 float* __restrict__ out) {
  __shared__ float As[16][33], Bs[16][64];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 64;
  float acc[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const int K = 2 * p;  // k < p: Y with M1; k >= p: Up with M2
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int t = threadIdx.x; t < 32 * 16; t += 256) {
      const int rr = t / 16, kk = t % 16;
      const int r = r0 + rr, k = k0 + kk;
      float v = 0.f;
      if (r < N && k < K) v = k < p ? Y[size_t(r) * p + k] : Up[size_t(r) * p + (k - p)];
      As[kk][rr] = v;
    }
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      const int kk = t / 64, cc = t % 64;
      const int k = k0 + kk, c = c0 + cc;
      Bs[kk][cc] = (k < K && c < p) ? M[size_t(k) * p + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[2], b[4];
#pragma unroll
      for (int i = 0; i < 2; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = r0 + ty + 16 * i;
    if (r >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < p) out[size_t(r) * p + c] = scale * acc[i][j];
    }
  }
}

void launch_ym32(int N, int p, const float* Y, const float* Up, const float* M, float scale,
                 float* out, cudaStream_t s) {
  dim3 grid((p + 63) / 64, (N + 31) / 32);
  count_launches(1);
  ym_kernel<<<grid, 256, 0, s>>>(N, p, Y, Up, M, scale, out);
  MDS_CUDA(cudaGetLastError());
}

template <int BN>
static int gemm32_split_count(int N, int ncol, size_t ws_bytes, int* kchunk_out) {
  const int gx = (ncol + BN - 1) / BN, gy = (N + 127) / 128;
  // about four blocks per SM (the kernel holds up to three per SM), each split >= 64 K-rows
  int splits = (4 * 152 + gx * gy - 1) / (gx * gy);
  splits = std::min(splits, std::max(1, N / 64));
  const size_t per = size_t(N) * ncol * sizeof(float);
  if (size_t(splits + 1) * per > ws_bytes) splits = int(ws_bytes / per) - 1;  // +1: YM slice
  if (splits < 1) throw DeviceError{cudaErrorMemoryAllocation};
  int kchunk = (N + splits - 1) / splits;
  kchunk = (kchunk + 7) / 8 * 8;
  if (kchunk_out) *kchunk_out = kchunk;
  return (N + kchunk - 1) / kchunk;
}

template <int BN, int TN>
static int gemm32_cfg(int N, int ncol, const float* G, const float* U, const int32_t* idx,
                      const float* w, float gscale, const float* Y, void* ws, size_t ws_bytes,
                      cudaStream_t s) {
  int kchunk = 0;
  const int splits = gemm32_split_count<BN>(N, ncol, ws_bytes, &kchunk);
  dim3 grid((ncol + BN - 1) / BN, (N + 127) / 128, splits);
  count_launches(1);
  gemm32_kernel<BN, TN><<<grid, 256, 0, s>>>(N, ncol, kchunk, G, U, idx, w, gscale, Y,
                                             static_cast<float*>(ws));
  MDS_CUDA(cudaGetLastError());
  return splits;
}

int gemm32_splits(int N, int ncol, size_t ws_bytes) {
  if (ncol <= 16) return gemm32_split_count<16>(N, ncol, ws_bytes, nullptr);
  if (ncol <= 32) return gemm32_split_count<32>(N, ncol, ws_bytes, nullptr);
  if (ncol <= 64) return gemm32_split_count<64>(N, ncol, ws_bytes, nullptr);
  return gemm32_split_count<128>(N, ncol, ws_bytes, nullptr);
}

int launch_gemm32_partials(int N, int ncol, const float* G, const float* U, const int32_t* idx,
                           const float* w, float gscale, const float* Y, void* ws, size_t ws_bytes,
                           cudaStream_t s) {
  if (ncol <= 16) return gemm32_cfg<16, 1>(N, ncol, G, U, idx, w, gscale, Y, ws, ws_bytes, s);
  if (ncol <= 32) return gemm32_cfg<32, 2>(N, ncol, G, U, idx, w, gscale, Y, ws, ws_bytes, s);
  if (ncol <= 64) return gemm32_cfg<64, 4>(N, ncol, G, U, idx, w, gscale, Y, ws, ws_bytes, s);
  return gemm32_cfg<128, 8>(N, ncol, G, U, idx, w, gscale, Y, ws, ws_bytes, s);
}

}  // namespace mds

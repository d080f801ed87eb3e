// Projector kernels: per-class means over the inverse map (the SDDMM of Y Y' or
// Y U' + U Y' at the indexed entries followed by a segmented per-class mean,
// Section 3: y(S) = (AA*)^{-1} A(S + C)), and the full-matrix pass that forms
// R = A*(y) - S - C and with it G = Xt + D - sigma R (Lemma 3.1) or the
// multiplier update Xt <- Xt - sigma R (Algorithm 1, step 6).
#include "common.cuh"

namespace mds {

// One group of LG lanes per piece; lanes split the p columns of each dot.
template <typename T, int LG, int MODE>
__global__ void __launch_bounds__(256) class_means_kernel(
    int n_pieces, int N, int p, const uint32_t* __restrict__ ent,
    const int32_t* __restrict__ piece_start, const int32_t* __restrict__ piece_class,
    const T* __restrict__ Y, const T* __restrict__ U, const double* __restrict__ C,
    const double* __restrict__ mult, T* __restrict__ piece_buf, T* __restrict__ out) {
  const int lane = threadIdx.x % LG;
  const int piece = (blockIdx.x * blockDim.x + threadIdx.x) / LG;
  const bool active = piece < n_pieces;
  T acc = T(0);
  int cls = 0;
  if (active) {
    const int e0 = piece_start[piece], e1 = piece_start[piece + 1];
    cls = piece_class[piece];
    for (int e = e0; e < e1; ++e) {
      const uint32_t code = ent[e];
      const int b = int(code >> 16), g = int(code & 0xFFFFu);
      const T wt = (b == g) ? T(1) : T(2);
      const T* yb = Y + size_t(b) * p;
      const T* yg = Y + size_t(g) * p;
      T v = T(0);
      if (MODE == 0) {
        for (int c = lane; c < p; c += LG) v = fma(yb[c], yg[c], v);
        if (C != nullptr && lane == 0) v += T(C[size_t(b) * N + g]);
      } else {
        const T* ub = U + size_t(b) * p;
        const T* ug = U + size_t(g) * p;
        for (int c = lane; c < p; c += LG) {
          v = fma(yb[c], ug[c], v);
          v = fma(ub[c], yg[c], v);
        }
      }
      acc = fma(wt, v, acc);
    }
  }
#pragma unroll
  for (int off = LG / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (active && lane == 0) {
    if (cls >= 0) {
      out[cls] = T(double(acc) / mult[cls]);
    } else {
      piece_buf[piece] = acc;
    }
  }
}

// Classes split over several pieces: sum their pieces in ascending order.
template <typename T>
__global__ void class_finalize_kernel(int n_multi, const int32_t* __restrict__ multi_class,
                                      const int32_t* __restrict__ multi_range,
                                      const T* __restrict__ piece_buf,
                                      const double* __restrict__ mult, T* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_multi) return;
  const int cls = multi_class[j];
  double s = 0.0;
  for (int pc = multi_range[2 * j]; pc < multi_range[2 * j + 1]; ++pc) s += double(piece_buf[pc]);
  out[cls] = T(s / mult[cls]);
}

template <typename T, int LG>
static void dispatch_means(const ClassMap& cm, int N, int p, int mode, const T* Y, const T* U,
                           const double* C, const double* mult, T* piece_buf, T* out,
                           cudaStream_t s) {
  const int threads = 256;
  const long long lanes = (long long)cm.n_pieces * LG;
  const int blocks = int((lanes + threads - 1) / threads);
  if (blocks > 0) {
    count_launches(1);
    if (mode == 0)
      class_means_kernel<T, LG, 0><<<blocks, threads, 0, s>>>(cm.n_pieces, N, p, cm.ent,
                                                              cm.piece_start, cm.piece_class, Y,
                                                              U, C, mult, piece_buf, out);
    else
      class_means_kernel<T, LG, 1><<<blocks, threads, 0, s>>>(cm.n_pieces, N, p, cm.ent,
                                                              cm.piece_start, cm.piece_class, Y,
                                                              U, C, mult, piece_buf, out);
  }
  if (cm.n_multi > 0) count_launches(1);
  if (cm.n_multi > 0)
    class_finalize_kernel<T><<<(cm.n_multi + 255) / 256, 256, 0, s>>>(
        cm.n_multi, cm.multi_class, cm.multi_range, piece_buf, mult, out);
  MDS_CUDA(cudaGetLastError());
}

template <typename T>
void launch_class_means(const ClassMap& cm, int N, int p, int mode, const T* Y, const T* U,
                        const double* C, const double* mult, T* piece_buf, T* out,
                        cudaStream_t s) {
  // lanes per group: about p/2 columns per lane pair, a power of two in [1, 32]
  if (p <= 2)
    dispatch_means<T, 1>(cm, N, p, mode, Y, U, C, mult, piece_buf, out, s);
  else if (p <= 4)
    dispatch_means<T, 2>(cm, N, p, mode, Y, U, C, mult, piece_buf, out, s);
  else if (p <= 8)
    dispatch_means<T, 4>(cm, N, p, mode, Y, U, C, mult, piece_buf, out, s);
  else if (p <= 16)
    dispatch_means<T, 8>(cm, N, p, mode, Y, U, C, mult, piece_buf, out, s);
  else if (p <= 32)
    dispatch_means<T, 16>(cm, N, p, mode, Y, U, C, mult, piece_buf, out, s);
  else
    dispatch_means<T, 32>(cm, N, p, mode, Y, U, C, mult, piece_buf, out, s);
}

template void launch_class_means<double>(const ClassMap&, int, int, int, const double*,
                                         const double*, const double*, const double*, double*,
                                         double*, cudaStream_t);
template void launch_class_means<float>(const ClassMap&, int, int, int, const float*,
                                        const float*, const double*, const double*, float*,
                                        float*, cudaStream_t);

// ---- G pass -----------------------------------------------------------------
// Upper-triangle tiles only (G, R and XD are symmetric): a 64 x 64 tile of
// entries per block, 16 x 16 threads, 4 x 4 entries per thread (rows ty + 16 i,
// columns tx + 16 j); Y rows staged through shared memory in chunks of 16
// columns.  Off-diagonal tiles also write their transpose through a shared-memory
// tile so that both writes are coalesced, and count twice in the sums.
constexpr int GP_TILE = 64, GP_KC = 16;

__device__ __forceinline__ void gp_tile_coords(int t, int nt, int* by, int* bx) {
  int r = 0;
  while (t >= nt - r) {
    t -= nt - r;
    ++r;
  }
  *by = r;
  *bx = r + t;
}

template <int MODE>
__global__ void __launch_bounds__(256) gpass_kernel(int N, int p, const double* __restrict__ Y,
                                                    const int32_t* __restrict__ idx,
                                                    const double* __restrict__ y,
                                                    const double* __restrict__ C, double sigma,
                                                    double* __restrict__ XD, double* __restrict__ G,
                                                    float* __restrict__ Gf,
                                                    double* __restrict__ part) {
  __shared__ double smem[GP_TILE * (GP_TILE + 1)];  // Y chunks, then the transpose tile
  __shared__ double red[2][256];
  double (*Yr)[GP_KC + 1] = reinterpret_cast<double (*)[GP_KC + 1]>(smem);
  double (*Yc)[GP_KC + 1] = reinterpret_cast<double (*)[GP_KC + 1]>(smem + GP_TILE * (GP_KC + 1));
  const int nt = (N + GP_TILE - 1) / GP_TILE;
  int tby, tbx;
  gp_tile_coords(blockIdx.x, nt, &tby, &tbx);
  const bool diag = tby == tbx;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = tby * GP_TILE, c0 = tbx * GP_TILE;
  double s[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s[i][j] = 0.0;
  for (int k0 = 0; k0 < p; k0 += GP_KC) {
    for (int t = threadIdx.x; t < GP_TILE * GP_KC; t += 256) {
      const int rr = t / GP_KC, kk = t % GP_KC;
      const int gr = r0 + rr, gc = c0 + rr, k = k0 + kk;
      Yr[rr][kk] = (gr < N && k < p) ? Y[size_t(gr) * p + k] : 0.0;
      Yc[rr][kk] = (gc < N && k < p) ? Y[size_t(gc) * p + k] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GP_KC; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Yr[ty + 16 * i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Yc[tx + 16 * j][kk];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) s[i][j] = fma(a[i], b[j], s[i][j]);
    }
    __syncthreads();
  }
  // smem now free: reuse as the transpose tile T[c_local][r_local]
  double (*Tt)[GP_TILE + 1] = reinterpret_cast<double (*)[GP_TILE + 1]>(smem);
  const double wgt = diag ? 1.0 : 2.0;
  double sr2 = 0.0, sxs = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rl = ty + 16 * i, r = r0 + rl;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cl = tx + 16 * j, c = c0 + cl;
      double out = 0.0;
      if (r < N && c < N) {
        const size_t e = size_t(r) * N + c;
        const double sv = s[i][j];
        double rv = y[idx[e]] - sv;
        if (C != nullptr) rv -= C[e];
        sr2 = fma(wgt * rv, rv, sr2);
        if (MODE == 0) {
          const double xd = XD[e];
          out = fma(-sigma, rv, xd);
          G[e] = out;
          if (Gf != nullptr) Gf[e] = float(out);
          sxs = fma(wgt * xd, sv, sxs);
        } else {
          out = fma(-sigma, rv, XD[e]);
          XD[e] = out;
          sxs = fma(wgt * out, sv, sxs);
        }
      }
      if (!diag) Tt[cl][rl] = out;
    }
  }
  if (!diag) {
    __syncthreads();
    // write the mirrored tile: row c0 + cl, columns r0 + rl (rl fastest across threads)
    for (int t = threadIdx.x; t < GP_TILE * GP_TILE; t += 256) {
      const int cl = t / GP_TILE, rl = t % GP_TILE;
      const int r = r0 + rl, c = c0 + cl;
      if (r < N && c < N) {
        const size_t e = size_t(c) * N + r;
        const double v = Tt[cl][rl];
        if (MODE == 0) {
          G[e] = v;
          if (Gf != nullptr) Gf[e] = float(v);
        } else {
          XD[e] = v;
        }
      }
    }
  }
  red[0][threadIdx.x] = sr2;
  red[1][threadIdx.x] = sxs;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = red[0][0];
    part[2 * blockIdx.x + 1] = red[1][0];
  }
}

__global__ void __launch_bounds__(256) pair_sum_kernel(int nb, const double* __restrict__ part,
                                                       double* __restrict__ out2) {
  __shared__ double red[2][256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = red[0][0];
    out2[1] = red[1][0];
  }
}

size_t gpass_partials(int N) {
  const size_t nt = (size_t(N) + GP_TILE - 1) / GP_TILE;
  return nt * (nt + 1);
}

void launch_gpass(int N, int p, int mode, const double* Y, const int32_t* idx, const double* y,
                  const double* C, double sigma, double* XD, double* G, float* Gf, double* part,
                  double* out2, cudaStream_t s) {
  const int nt = (N + GP_TILE - 1) / GP_TILE;
  const int grid = nt * (nt + 1) / 2;
  count_launches(2);
  if (mode == 0)
    gpass_kernel<0><<<grid, 256, 0, s>>>(N, p, Y, idx, y, C, sigma, XD, G, Gf, part);
  else
    gpass_kernel<1><<<grid, 256, 0, s>>>(N, p, Y, idx, y, C, sigma, XD, G, Gf, part);
  pair_sum_kernel<<<1, 256, 0, s>>>(grid, part, out2);
  MDS_CUDA(cudaGetLastError());
}

}  // namespace mds

// FP64-accurate evaluation of the subproblem on the FP32 pipe (df64.cuh):
//   * y(S) = (AA*)^{-1} A(Y Y')  (Section 3) — per-class means of Y_b . Y_g,
//   * the G pass: R = A*(y) - S, G = XD - sigma R, Psi partials (Lemma 3.1),
//   * the gradient product G Y (Proposition 4.2),
// each dot product of p (or N) terms accumulated as a compensated float pair.
// The inputs arrive split into float pairs (hi, lo) once per evaluation.
#include "common.cuh"
#include "df64.cuh"

namespace mds {

__global__ void split_kernel(size_t n, const double* __restrict__ x, float* __restrict__ hi,
                             float* __restrict__ lo) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    float h, l;
    df64_split(x[i], &h, &l);
    hi[i] = h;
    lo[i] = l;
  }
}

void launch_split(size_t n, const double* x, float* hi, float* lo, cudaStream_t s) {
  size_t b = (n + 255) / 256;
  if (b > 8192) b = 8192;
  if (b == 0) b = 1;
  count_launches(1);
  split_kernel<<<int(b), 256, 0, s>>>(n, x, hi, lo);
  MDS_CUDA(cudaGetLastError());
}

// ---- y(S): the multi-piece classes' sums of the per-piece df64 partials ------------
__global__ void class_finalize_df_kernel(int n_multi, const int32_t* __restrict__ multi_class,
                                         const int32_t* __restrict__ multi_range,
                                         const double* __restrict__ piece_buf,
                                         const double* __restrict__ mult, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_multi) return;
  const int cls = multi_class[j];
  double s = 0.0;
  for (int pc = multi_range[2 * j]; pc < multi_range[2 * j + 1]; ++pc) s += piece_buf[pc];
  out[cls] = s / mult[cls];
}


// ---- G pass (upper-triangle tiles, mirrored writes; see gpass_kernel) -------------------
constexpr int DT = 64, DKC = 16;

__device__ __forceinline__ void df_tile_coords(int t, int nt, int* by, int* bx) {
  int r = 0;
  while (t >= nt - r) {
    t -= nt - r;
    ++r;
  }
  *by = r;
  *bx = r + t;
}

template <int MODE>
__global__ void __launch_bounds__(256) gpass_df_kernel(
    int N, int p, const float* __restrict__ Yh, const float* __restrict__ Yl,
    const int32_t* __restrict__ idx, const double* __restrict__ y, const double* __restrict__ C,
    double sigma, double* __restrict__ XD, double* __restrict__ G, float* __restrict__ Gh,
    float* __restrict__ Gl, double* __restrict__ part, const double* __restrict__ Sup) {
  __shared__ double smem[DT * (DT + 1)];  // float Y chunks, then the transpose tile
  __shared__ double red[2][256];
  float(*Rh)[DKC + 1] = reinterpret_cast<float(*)[DKC + 1]>(smem);
  float(*Rl)[DKC + 1] = Rh + DT;
  float(*Ch)[DKC + 1] = Rh + 2 * DT;
  float(*Cl)[DKC + 1] = Rh + 3 * DT;
  const int nt = (N + DT - 1) / DT;
  int tby, tbx;
  df_tile_coords(blockIdx.x, nt, &tby, &tbx);
  const bool diag = tby == tbx;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = tby * DT, c0 = tbx * DT;
  df64acc a[4][4];
  double ad[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      a[i][j] = df64acc{0.f, 0.f};
      ad[i][j] = 0.0;
    }
  int chunk = 0;
  for (int k0 = 0; k0 < (Sup == nullptr ? p : 0); k0 += DKC) {
    for (int t = threadIdx.x; t < DT * DKC; t += 256) {
      const int rr = t / DKC, kk = t % DKC;
      const int gr = r0 + rr, gc = c0 + rr, k = k0 + kk;
      const bool okr = gr < N && k < p, okc = gc < N && k < p;
      Rh[rr][kk] = okr ? Yh[size_t(gr) * p + k] : 0.f;
      Rl[rr][kk] = okr ? Yl[size_t(gr) * p + k] : 0.f;
      Ch[rr][kk] = okc ? Yh[size_t(gc) * p + k] : 0.f;
      Cl[rr][kk] = okc ? Yl[size_t(gc) * p + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < DKC; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = Rh[ty + 16 * i][kk];
        al[i] = Rl[ty + 16 * i][kk];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bh[j] = Ch[tx + 16 * j][kk];
        bl[j] = Cl[tx + 16 * j][kk];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df64_fma(a[i][j], ah[i], al[i], bh[j], bl[j]);
    }
    __syncthreads();
    if (++chunk == 4 && k0 + DKC < p) {
      chunk = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ad[i][j] += df64_value(a[i][j]);
          a[i][j] = df64acc{0.f, 0.f};
        }
    }
  }
  double(*Tt)[DT + 1] = reinterpret_cast<double(*)[DT + 1]>(smem);
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
        const double sv = Sup != nullptr ? Sup[e] : ad[i][j] + df64_value(a[i][j]);
        double rv = y[idx[e]] - sv;
        if (C != nullptr) rv -= C[e];
        sr2 = fma(wgt * rv, rv, sr2);
        if (MODE == 0) {
          const double xd = XD[e];
          out = fma(-sigma, rv, xd);
          if (G != nullptr) G[e] = out;
          if (Gh != nullptr) {
            float h, l;
            df64_split(out, &h, &l);
            Gh[e] = h;
            Gl[e] = l;
          }
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
    for (int t = threadIdx.x; t < DT * DT; t += 256) {
      const int cl = t / DT, rl = t % DT;
      const int r = r0 + rl, c = c0 + cl;
      if (r < N && c < N) {
        const size_t e = size_t(c) * N + r;
        const double v = Tt[cl][rl];
        if (MODE == 0) {
          if (G != nullptr) G[e] = v;
          if (Gh != nullptr) {
            float h, l;
            df64_split(v, &h, &l);
            Gh[e] = h;
            Gl[e] = l;
          }
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

__global__ void __launch_bounds__(256) df_pair_sum_kernel(int nb, const double* __restrict__ part,
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

void launch_gpass_df(int N, int p, int mode, const float* Yh, const float* Yl,
                     const int32_t* idx, const double* y, const double* C, double sigma,
                     double* XD, double* G, float* Gh, float* Gl, double* part, double* out2,
                     cudaStream_t s, const double* Sup) {
  const int nt = (N + DT - 1) / DT;
  const int grid = nt * (nt + 1) / 2;
  count_launches(2);
  if (mode == 0)
    gpass_df_kernel<0><<<grid, 256, 0, s>>>(N, p, Yh, Yl, idx, y, C, sigma, XD, G, Gh, Gl, part,
                                            Sup);
  else
    gpass_df_kernel<1><<<grid, 256, 0, s>>>(N, p, Yh, Yl, idx, y, C, sigma, XD, G, Gh, Gl, part,
                                            Sup);
  df_pair_sum_kernel<<<1, 256, 0, s>>>(grid, part, out2);
  MDS_CUDA(cudaGetLastError());
}

// ---- tiled y(S): S = Y Y' once, df64, upper-triangle tiles --------------------------------
// Writes S[r, c] for every entry of the tile to Sup (the G pass then reads it instead
// of recomputing the dot products) and wt * (S + C) of each upper entry (r <= c) to
// its slot of the class-ordered buffer permd (wt = 2 off the diagonal).
__global__ void __launch_bounds__(256) spass_df_kernel(int N, int p, const float* __restrict__ Yh,
                                                       const float* __restrict__ Yl,
                                                       const double* __restrict__ C,
                                                       const int32_t* __restrict__ slot,
                                                       double* __restrict__ Sup,
                                                       double* __restrict__ permd) {
  __shared__ float Rh[DT][DKC + 1], Rl[DT][DKC + 1], Ch[DT][DKC + 1], Cl[DT][DKC + 1];
  const int nt = (N + DT - 1) / DT;
  int tby, tbx;
  df_tile_coords(blockIdx.x, nt, &tby, &tbx);
  const bool diag = tby == tbx;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = tby * DT, c0 = tbx * DT;
  df64acc a[4][4];
  double ad[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      a[i][j] = df64acc{0.f, 0.f};
      ad[i][j] = 0.0;
    }
  int chunk = 0;
  for (int k0 = 0; k0 < p; k0 += DKC) {
    for (int t = threadIdx.x; t < DT * DKC; t += 256) {
      const int rr = t / DKC, kk = t % DKC;
      const int gr = r0 + rr, gc = c0 + rr, k = k0 + kk;
      const bool okr = gr < N && k < p, okc = gc < N && k < p;
      Rh[rr][kk] = okr ? Yh[size_t(gr) * p + k] : 0.f;
      Rl[rr][kk] = okr ? Yl[size_t(gr) * p + k] : 0.f;
      Ch[rr][kk] = okc ? Yh[size_t(gc) * p + k] : 0.f;
      Cl[rr][kk] = okc ? Yl[size_t(gc) * p + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < DKC; ++kk) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = Rh[ty + 16 * i][kk];
        al[i] = Rl[ty + 16 * i][kk];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bh[j] = Ch[tx + 16 * j][kk];
        bl[j] = Cl[tx + 16 * j][kk];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) df64_fma(a[i][j], ah[i], al[i], bh[j], bl[j]);
    }
    __syncthreads();
    if (++chunk == 4 && k0 + DKC < p) {
      chunk = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ad[i][j] += df64_value(a[i][j]);
          a[i][j] = df64acc{0.f, 0.f};
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rl = ty + 16 * i, r = r0 + rl;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cl = tx + 16 * j, c = c0 + cl;
      if (r < N && c < N) {
        const size_t e = size_t(r) * N + c;
        const double sv = ad[i][j] + df64_value(a[i][j]);
        Sup[e] = sv;
        if (!diag || rl <= cl) {
          const double v = C != nullptr ? sv + C[e] : sv;
          permd[slot[e]] = (r == c) ? v : 2.0 * v;
        }
      }
    }
  }
}

__global__ void piece_sum_d_kernel(int n_pieces, const int32_t* __restrict__ piece_start,
                                   const int32_t* __restrict__ piece_class,
                                   const double* __restrict__ permd,
                                   const double* __restrict__ mult,
                                   double* __restrict__ piece_buf, double* __restrict__ out) {
  const int pc = blockIdx.x * blockDim.x + threadIdx.x;
  if (pc >= n_pieces) return;
  double s = 0.0;
  for (int e = piece_start[pc]; e < piece_start[pc + 1]; ++e) s += permd[e];
  const int cls = piece_class[pc];
  if (cls >= 0)
    out[cls] = s / mult[cls];
  else
    piece_buf[pc] = s;
}

void launch_spass_df(const ClassMap& cm, int N, int p, const float* Yh, const float* Yl,
                     const double* C, const int32_t* slot, double* Sup, double* permd,
                     const double* mult, double* piece_buf, double* y, cudaStream_t s) {
  const int nt = (N + DT - 1) / DT;
  const int grid = nt * (nt + 1) / 2;
  count_launches(2);
  spass_df_kernel<<<grid, 256, 0, s>>>(N, p, Yh, Yl, C, slot, Sup, permd);
  piece_sum_d_kernel<<<(cm.n_pieces + 255) / 256, 256, 0, s>>>(
      cm.n_pieces, cm.piece_start, cm.piece_class, permd, mult, piece_buf, y);
  if (cm.n_multi > 0) {
    count_launches(1);
    class_finalize_df_kernel<<<(cm.n_multi + 255) / 256, 256, 0, s>>>(
        cm.n_multi, cm.multi_class, cm.multi_range, piece_buf, mult, y);
  }
  MDS_CUDA(cudaGetLastError());
}

// ---- gradient product GY = G Y with G = (Gh, Gl), Y = (Yh, Yl) ---------------------------
// Block tile 64 rows x BN columns, thread tile 4 x TN, K chunk 16, split-K over grid.z;
// each split writes FP64 partials, summed in ascending order by gemm_df_reduce_kernel.
template <int BN, int TN>
__global__ void __launch_bounds__(256) gemm_df_kernel(int N, int ncol, int kchunk,
                                                      const float* __restrict__ Gh,
                                                      const float* __restrict__ Gl,
                                                      const float* __restrict__ Yh,
                                                      const float* __restrict__ Yl,
                                                      double* __restrict__ part) {
  constexpr int BM = 64, TM = 4, BK = 16;
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  __shared__ float Ah[BK][BM + 1], Al[BK][BM + 1];
  __shared__ float Bh[BK][BN], Bl[BK][BN];
  const int tx = threadIdx.x % (BN / TN), ty = threadIdx.x / (BN / TN);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * kchunk, ke = min(N, kb + kchunk);
  df64acc acc[TM][TN];
  double accd[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      acc[i][j] = df64acc{0.f, 0.f};
      accd[i][j] = 0.0;
    }
  int chunk = 0;
  for (int k0 = kb; k0 < ke; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += 256) {
      const int r = t / BK, kk = t % BK;
      const int gr = m0 + r, gk = k0 + kk;
      const bool ok = gr < N && gk < ke;
      Ah[kk][r] = ok ? Gh[size_t(gr) * N + gk] : 0.f;
      Al[kk][r] = ok ? Gl[size_t(gr) * N + gk] : 0.f;
    }
    for (int t = threadIdx.x; t < BK * BN; t += 256) {
      const int kk = t / BN, c = t % BN;
      const int gk = k0 + kk, gc = n0 + c;
      const bool ok = gk < ke && gc < ncol;
      Bh[kk][c] = ok ? Yh[size_t(gk) * ncol + gc] : 0.f;
      Bl[kk][c] = ok ? Yl[size_t(gk) * ncol + gc] : 0.f;
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < BK; ++kk) {
      float ah[TM], al[TM], bh[TN], bl[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        ah[i] = Ah[kk][ty * TM + i];
        al[i] = Al[kk][ty * TM + i];
      }
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        bh[j] = Bh[kk][tx * TN + j];
        bl[j] = Bl[kk][tx * TN + j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) df64_fma(acc[i][j], ah[i], al[i], bh[j], bl[j]);
    }
    __syncthreads();
    // fold the float pairs into FP64 every 64 terms: bounds the growth of the
    // float compensation term over long (K = N) sums
    if (++chunk == 4) {
      chunk = 0;
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          accd[i][j] += df64_value(acc[i][j]);
          acc[i][j] = df64acc{0.f, 0.f};
        }
    }
  }
  double* op = part + size_t(blockIdx.z) * N * ncol;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int r = m0 + ty * TM + i;
    if (r >= N) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int c = n0 + tx * TN + j;
      if (c < ncol) op[size_t(r) * ncol + c] = accd[i][j] + df64_value(acc[i][j]);
    }
  }
}

__global__ void gemm_df_reduce_kernel(size_t n, int splits, const double* __restrict__ part,
                                      double* __restrict__ out) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[size_t(z) * n + i];
    out[i] = s;
  }
}

template <int BN, int TN>
static void gemm_df_cfg(int N, int ncol, const float* Gh, const float* Gl, const float* Yh,
                        const float* Yl, double* out, void* ws, size_t ws_bytes, cudaStream_t s) {
  const int gx = (ncol + BN - 1) / BN, gy = (N + 63) / 64;
  int splits = (2 * 152 + gx * gy - 1) / (gx * gy);
  splits = std::min(splits, (N + 63) / 64);
  const size_t per = size_t(N) * ncol * sizeof(double);
  if (size_t(splits) * per > ws_bytes) splits = int(ws_bytes / per);
  if (splits < 1) throw DeviceError{cudaErrorMemoryAllocation};
  int kchunk = (N + splits - 1) / splits;
  kchunk = (kchunk + 15) / 16 * 16;
  splits = (N + kchunk - 1) / kchunk;
  dim3 grid(gx, gy, splits);
  count_launches(2);
  gemm_df_kernel<BN, TN><<<grid, 256, 0, s>>>(N, ncol, kchunk, Gh, Gl, Yh, Yl,
                                              static_cast<double*>(ws));
  const size_t n = size_t(N) * ncol;
  size_t rb = (n + 255) / 256;
  if (rb > 4096) rb = 4096;
  gemm_df_reduce_kernel<<<int(rb), 256, 0, s>>>(n, splits, static_cast<const double*>(ws), out);
  MDS_CUDA(cudaGetLastError());
}

void launch_gemm_df(int N, int ncol, const float* Gh, const float* Gl, const float* Yh,
                    const float* Yl, double* out, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (ncol <= 16)
    gemm_df_cfg<16, 1>(N, ncol, Gh, Gl, Yh, Yl, out, ws, ws_bytes, s);
  else if (ncol <= 32)
    gemm_df_cfg<32, 2>(N, ncol, Gh, Gl, Yh, Yl, out, ws, ws_bytes, s);
  else
    gemm_df_cfg<64, 4>(N, ncol, Gh, Gl, Yh, Yl, out, ws, ws_bytes, s);
}

}  // namespace mds

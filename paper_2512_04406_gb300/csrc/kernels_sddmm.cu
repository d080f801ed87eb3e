// Tiled SDDMM for the class sums of the Hessian-vector product (Section 3,
// Proposition 4.2): w = (AA*)^{-1} A(Y U' + U Y').
//   pass 1: upper-triangle 64 x 64 tiles of W = Y U' + U Y' (rows of Y and U
//           staged through shared memory, 4 x 4 entries per thread); each entry
//           (r <= c), weighted 2 off the diagonal, is written to its slot in the
//           class-ordered buffer `perm` (slot[r*N + c] = its position in the
//           per-class inverse map);
//   pass 2: per piece, a contiguous sum of perm; single-piece classes divide by
//           the multiplicity at once, split classes are finished in ascending
//           piece order — the same deterministic order for every call.
#include "common.cuh"

namespace mds {

constexpr int ST = 64, SKC = 16;

__device__ __forceinline__ void sd_tile_coords(int t, int nt, int* by, int* bx) {
  int r = 0;
  while (t >= nt - r) {
    t -= nt - r;
    ++r;
  }
  *by = r;
  *bx = r + t;
}

__global__ void __launch_bounds__(256) sddmm_tile_kernel(int N, int p, const float* __restrict__ Y,
                                                         const float* __restrict__ U,
                                                         const int32_t* __restrict__ slot,
                                                         float* __restrict__ perm) {
  __shared__ float Yr[ST][SKC + 1], Ur[ST][SKC + 1], Yc[ST][SKC + 1], Uc[ST][SKC + 1];
  const int nt = (N + ST - 1) / ST;
  int tby, tbx;
  sd_tile_coords(blockIdx.x, nt, &tby, &tbx);
  const bool diag = tby == tbx;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int r0 = tby * ST, c0 = tbx * ST;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  // register prefetch of the next K chunk: each thread stages 4 elements of each array
  constexpr int PER = ST * SKC / 256;  // 4
  float pyr[PER], pur[PER], pyc[PER], puc[PER];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int t = threadIdx.x + q * 256;
      const int rr = t / SKC, kk = t % SKC;
      const int gr = r0 + rr, gc = c0 + rr, k = k0 + kk;
      const bool okr = gr < N && k < p, okc = gc < N && k < p;
      pyr[q] = okr ? Y[size_t(gr) * p + k] : 0.f;
      pur[q] = okr ? U[size_t(gr) * p + k] : 0.f;
      pyc[q] = okc ? Y[size_t(gc) * p + k] : 0.f;
      puc[q] = okc ? U[size_t(gc) * p + k] : 0.f;
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < p; k0 += SKC) {
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int t = threadIdx.x + q * 256;
      const int rr = t / SKC, kk = t % SKC;
      Yr[rr][kk] = pyr[q];
      Ur[rr][kk] = pur[q];
      Yc[rr][kk] = pyc[q];
      Uc[rr][kk] = puc[q];
    }
    __syncthreads();
    if (k0 + SKC < p) fetch(k0 + SKC);
#pragma unroll
    for (int kk = 0; kk < SKC; ++kk) {
      float yr[4], ur[4], yc[4], uc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        yr[i] = Yr[ty + 16 * i][kk];
        ur[i] = Ur[ty + 16 * i][kk];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        yc[j] = Yc[tx + 16 * j][kk];
        uc[j] = Uc[tx + 16 * j][kk];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(yr[i], uc[j], fmaf(ur[i], yc[j], acc[i][j]));
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int rl = ty + 16 * i, r = r0 + rl;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cl = tx + 16 * j, c = c0 + cl;
      if (r < N && c < N && (!diag || rl <= cl)) {
        const float wt = (r == c) ? 1.f : 2.f;
        perm[slot[size_t(r) * N + c]] = wt * acc[i][j];
      }
    }
  }
}

// Pass 2: one thread per piece.
__global__ void piece_sum_kernel(int n_pieces, const int32_t* __restrict__ piece_start,
                                 const int32_t* __restrict__ piece_class,
                                 const float* __restrict__ perm, const double* __restrict__ mult,
                                 float* __restrict__ piece_buf, float* __restrict__ out) {
  const int pc = blockIdx.x * blockDim.x + threadIdx.x;
  if (pc >= n_pieces) return;
  float s = 0.f;
  for (int e = piece_start[pc]; e < piece_start[pc + 1]; ++e) s += perm[e];
  const int cls = piece_class[pc];
  if (cls >= 0)
    out[cls] = float(double(s) / mult[cls]);
  else
    piece_buf[pc] = s;
}

__global__ void piece_finalize_kernel(int n_multi, const int32_t* __restrict__ multi_class,
                                      const int32_t* __restrict__ multi_range,
                                      const float* __restrict__ piece_buf,
                                      const double* __restrict__ mult, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_multi) return;
  const int cls = multi_class[j];
  double s = 0.0;
  for (int pc = multi_range[2 * j]; pc < multi_range[2 * j + 1]; ++pc) s += double(piece_buf[pc]);
  out[cls] = float(s / mult[cls]);
}

void launch_piece_sums(const ClassMap& cm, const float* perm, const double* mult,
                       float* piece_buf, float* out, cudaStream_t s) {
  count_launches(1);
  piece_sum_kernel<<<(cm.n_pieces + 255) / 256, 256, 0, s>>>(cm.n_pieces, cm.piece_start,
                                                            cm.piece_class, perm, mult, piece_buf,
                                                            out);
  if (cm.n_multi > 0) {
    count_launches(1);
    piece_finalize_kernel<<<(cm.n_multi + 255) / 256, 256, 0, s>>>(
        cm.n_multi, cm.multi_class, cm.multi_range, piece_buf, mult, out);
  }
  MDS_CUDA(cudaGetLastError());
}

void launch_sddmm_means(const ClassMap& cm, int N, int p, const float* Y, const float* U,
                        const int32_t* slot, float* perm, const double* mult, float* piece_buf,
                        float* out, cudaStream_t s) {
  const int nt = (N + ST - 1) / ST;
  const int tiles = nt * (nt + 1) / 2;
  count_launches(2);
  sddmm_tile_kernel<<<tiles, 256, 0, s>>>(N, p, Y, U, slot, perm);
  piece_sum_kernel<<<(cm.n_pieces + 255) / 256, 256, 0, s>>>(cm.n_pieces, cm.piece_start,
                                                            cm.piece_class, perm, mult, piece_buf,
                                                            out);
  if (cm.n_multi > 0) {
    count_launches(1);
    piece_finalize_kernel<<<(cm.n_multi + 255) / 256, 256, 0, s>>>(
        cm.n_multi, cm.multi_class, cm.multi_range, piece_buf, mult, out);
  }
  MDS_CUDA(cudaGetLastError());
}

}  // namespace mds

// Internal declarations shared by the CUDA translation units of libmanidsdp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "../../include/manidsdp.h"

namespace mds {

// Entries of the per-class inverse map pack (row, col) as (row << 16) | col,
// so N must stay below 65536.
constexpr int kMaxN = 65535;
constexpr int kMaxP = 512;  // widest factor: row-local kernels hold 16 columns per lane
// A class's entries are processed in pieces of at most this many entries.
constexpr int kPieceLen = 32;
// Threads of the reduction kernels; the partial-sum buffers hold kRedBlocks values.
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;  // 2 x 152 SMs

struct DeviceError {
  cudaError_t err;
};

#define MDS_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) throw ::mds::DeviceError{e_}; \
  } while (0)

// ---- the per-class inverse map (built on the host at setup) -----------------
struct ClassMap {
  int32_t n_entries = 0;  // entries (b <= g), grouped by class
  int32_t n_pieces = 0;
  int32_t n_multi = 0;    // classes split into more than one piece
  uint32_t* ent = nullptr;        // [n_entries] (b << 16) | g
  int32_t* piece_start = nullptr; // [n_pieces + 1]
  int32_t* piece_class = nullptr; // [n_pieces]
  int32_t* multi_class = nullptr; // [n_multi] classes with > 1 piece
  int32_t* multi_range = nullptr; // [2 n_multi] first piece and end piece of each such class
};

// Count of kernel launches issued by this library (all contexts, all threads).
void count_launches(long long n);

// ---- kernel launchers (defined in kernels_*.cu) ----------------------------
// Segmented per-class sums over the inverse map:
//   mode 0: out[a] = (sum_{(b,g) in a} wt * (Y_b . Y_g + C_bg)) / mult[a]     -> y(S)
//   mode 1: out[a] = (sum_{(b,g) in a} wt * (Y_b . U_g + U_b . Y_g)) / mult[a] -> w
// wt = 2 off the diagonal, 1 on it.  piece_buf holds one partial per piece.
template <typename T>
void launch_class_means(const ClassMap& cm, int N, int p, int mode, const T* Y, const T* U,
                        const double* C, const double* mult, T* piece_buf, T* out, cudaStream_t s);

// G-pass over all N x N entries (FP64):
//   s = Y_b . Y_g, a = idx[b,g], r = y[a] - s - C_bg
//   mode 0 (evaluate):  G = XD - sigma r ; optionally Gf = float(G);
//                       partials: sum r^2, sum XD*s
//   mode 1 (multiplier): XD <- XD - sigma r ; partials: sum r^2, sum XD_new*s
// part holds 2 partial sums per block; out2 receives (sum r^2, sum XD*s) summed in a
// fixed order.
void launch_gpass(int N, int p, int mode, const double* Y, const int32_t* idx, const double* y,
                  const double* C, double sigma, double* XD, double* G, float* Gf, double* part,
                  double* out2, cudaStream_t s);
size_t gpass_partials(int N);

// out[M x ncol] = alpha * A[M x K] B[K x ncol] + beta * out, row-major with leading dims.
// With idx/w non-null ("gather" mode) the product also adds
//   alpha * sum_g (gscale * w[idx[b, g]]) * B2[g, :]
// i.e. the moment matrix A*(w) applied to B2 (K must equal M = N then).
template <typename T>
void launch_gemm(int M, int ncol, int K, const T* A, int lda, const T* B, int ldb, T* out, int ldc,
                 T alpha, T beta, const int32_t* idx, const T* w, T gscale, const T* B2,
                 void* ws, size_t ws_bytes, cudaStream_t s);

// Split-K partial products only (no reduce): returns the number of splits written
// to ws as [splits][M][ncol].
template <typename T>
int launch_gemm_partials(int M, int ncol, int K, const T* A, int lda, const T* B, int ldb,
                         const int32_t* idx, const T* w, T gscale, const T* B2, void* ws,
                         size_t ws_bytes, cudaStream_t s);
// out = [A1' B ; A2' B] (2 p x p), A1, A2, B: N x p.
template <typename T>
void launch_gram2(int N, int p, const T* A1, const T* A2, const T* B, T* out, void* ws,
                  size_t ws_bytes, cudaStream_t s);
// Up = P_Y(U) (FP64), UpT = T(Up), YT = T(Y) if write_y.
template <typename T>
void launch_hv_prep(int N, int p, const double* Y, const double* U, double* Up, T* UpT, T* YT,
                    bool write_y, cudaStream_t s);
// HU from the split-K partials of T = G U - sigma A*(w) Y and M = [U'Y; Y'Y].
template <typename T>
void launch_hv_epilogue(int N, int p, int splits, const T* part, const T* M, const double* Y,
                        const double* Up, const double* z, double sigma, double* HU,
                        cudaStream_t s);
// ---- df64 evaluation (kernels_df64.cu): FP64-accurate on the FP32 pipe ----
void launch_split(size_t n, const double* x, float* hi, float* lo, cudaStream_t s);

void launch_gpass_df(int N, int p, int mode, const float* Yh, const float* Yl,
                     const int32_t* idx, const double* y, const double* C, double sigma,
                     double* XD, double* G, float* Gh, float* Gl, double* part, double* out2,
                     cudaStream_t s, const double* Sup = nullptr);
// y(S) by tiles: S = Y Y' (df64) into Sup (N x N, tiles of the upper triangle), class
// sums through the slot map into permd, per-piece FP64 sums into y.
void launch_spass_df(const ClassMap& cm, int N, int p, const float* Yh, const float* Yl,
                     const double* C, const int32_t* slot, double* Sup, double* permd,
                     const double* mult, double* piece_buf, double* y, cudaStream_t s);
void launch_gemm_df(int N, int ncol, const float* Gh, const float* Gl, const float* Yh,
                    const float* Yl, double* out, void* ws, size_t ws_bytes, cudaStream_t s);

// ---- TMA-fed tensor-core engine of the FP32 Hess-vec (kernels_tcx.cu) ------
// Operands are FP32 values held as TF32 pairs (hi, lo) in row-major arrays whose
// leading dimensions are multiples of 4 (tcx_ld).
int tcx_ld(int n);
// X (N x p FP64) as TF32 pairs: rows (leading dimension ld) and, when hiT is not
// null, transposed (p x N, leading dimension ldt).
void launch_tcx_split_rows(int N, int p, const double* X, float* hi, float* lo, int ld, float* hiT,
                           float* loT, int ldt, cudaStream_t s);
// G (N x N FP32, leading dimension N) or, when idx is given, the projector residual
// gscale * (G - w[idx]) with G the full W (leading dimension ld), as TF32 pairs.
void launch_tcx_split_matrix(int N, const float* G, const int32_t* idx, const float* w,
                             float gscale, float* hi, float* lo, int ld, cudaStream_t s);
// Split-K partials [splits][N][p] of T = G Up + QW Y (QW = sigma Q(W)) from TF32 pairs;
// returns the number of splits, tcx_gather_splits(N).  pairs = 0: only the hi parts, one TF32 product per step (about 2^-11 relative
// per operand; the precision schedule's early iterations).
int tcx_gather_splits(int N);
int launch_tcx_gather(int N, int p, const float* Ghi, const float* Glo, const float* QWhi,
                      const float* QWlo, int ldg, const float* UThi, const float* UTlo,
                      const float* YThi, const float* YTlo, int ldt, float* part, size_t ws_bytes,
                      int* err, cudaStream_t s, int pairs = 1);
// W = Y U' + U Y' on the upper-triangle tiles: entry (r <= c) weighted 2 off the
// diagonal written to perm[slot[r N + c]], and every entry of W into wfull (ldw).
void launch_tcx_sddmm(int N, int p, const float* Yhi, const float* Ylo, const float* Uhi,
                      const float* Ulo, int ld, const int32_t* slot, float* perm, float* wfull,
                      int ldw, const int2* tiles, int ntiles, int* err, cudaStream_t s,
                      int pairs = 1);
std::vector<int2> tcx_upper_tiles(int N);
// Per-piece sums of the class-ordered buffer into out[a] / mult[a] (kernels_sddmm.cu).
void launch_piece_sums(const ClassMap& cm, const float* perm, const double* mult,
                       float* piece_buf, float* out, cudaStream_t s);

// Tiled SDDMM class sums (kernels_sddmm.cu): out[a] = A(Y U' + U Y')_a / mult[a] in FP32.
void launch_sddmm_means(const ClassMap& cm, int N, int p, const float* Y, const float* U,
                        const int32_t* slot, float* perm, const double* mult, float* piece_buf,
                        float* out, cudaStream_t s);

// FP32 gather GEMM partials (kernels_gemm32.cu): [splits][N][ncol] of
// G U - sigma A*(w) Y; returns the number of splits.
int launch_gemm32_partials(int N, int ncol, const float* G, const float* U, const int32_t* idx,
                           const float* w, float gscale, const float* Y, void* ws, size_t ws_bytes,
                           cudaStream_t s);

// Number of split-K partial products launch_gemm32_partials writes for these sizes;
// the YM slice goes right after them.
int gemm32_splits(int N, int ncol, size_t ws_bytes);

// out = scale * (Y M1 + Up M2), M = [M1; M2] (2p x p), FP32 (kernels_gemm32.cu)
void launch_ym32(int N, int p, const float* Y, const float* Up, const float* M, float scale,
                 float* out, cudaStream_t s);

// ---- device-driven tCG (kernels_tcg.cu) ----
size_t tcg_state_bytes();
int tcg_epilogue_blocks(int N);
int tcg_update_blocks();
void launch_tcg_init(void* st, const double* rr0, double delta, double floor_rel, double abs_target,
                     int max_iters, cudaStream_t s);
template <typename T>
void launch_tcg_prep(int N, int p, const void* st, const double* Y, const double* r, double* delta,
                     double* Up, T* UpT, cudaStream_t s);
template <typename T>
void launch_tcg_epilogue(int N, int p, int splits, const T* part, const T* M, const double* Y,
                         const double* Up, const double* z, double sigma, const double* delta,
                         double* Hd, double* kpart, cudaStream_t s);
void launch_tcg_alpha(int nparts, const double* kpart, void* st, cudaStream_t s);
void launch_tcg_update(size_t n, const void* st, const double* delta, const double* Hd,
                       double* eta, double* Heta, double* r, double* rpart, cudaStream_t s);
void launch_tcg_beta(int nparts, const double* rpart, void* st, cudaGraphConditionalHandle h,
                     cudaStream_t s);
void tcg_read_state(const void* st, int* flag, int* iters, void* pinned, cudaStream_t s);
long long launches_now();
void uncount_launches(long long n);

// out[p1 x p2] = A[N x p1]' B[N x p2]  (deterministic: one block per output tile,
// a fixed reduction order over N).
template <typename T>
void launch_gram(int N, int p1, int p2, const T* A, const T* B, T* out, void* ws, size_t ws_bytes,
                 cudaStream_t s);

// Row-local epilogue of the Hessian (Eq. (4.7)) on T = G U - sigma A*(w) Y:
//   Ht = 2 T + 2 sigma (Y M1 + U M2)   (M1 = U'Y, M2 = Y'Y already folded into YM)
//   HU = Ht - (Ht . Y_b) Y_b - 2 z_b U_b
template <typename T>
void launch_hess_epilogue(int N, int p, const T* Tm, const T* YM, const T* Y, const T* U,
                          const double* z, double sigma, double* HU, cudaStream_t s);

// Row-local ops (FP64)
void launch_retract(int N, int p, const double* Y, const double* E, double t, double* out,
                    cudaStream_t s);  // rows of Y + t E normalised
void launch_rowdot(int N, int p, const double* A, const double* B, double* out, cudaStream_t s);
// grad = 2 (GY - z o Y)
void launch_grad_from_gy(int N, int p, const double* GY, const double* z, const double* Y,
                         double* grad, cudaStream_t s);
void launch_to_float(size_t n, const double* a, float* out, cudaStream_t s);
// out = a*x + b*y (elementwise, n)
void launch_axpby(size_t n, double a, const double* x, double b, const double* y, double* out,
                  cudaStream_t s);
// Deterministic dot products: up to 3 pairs at once. part: 3 * kRedBlocks doubles.
void launch_dots(size_t n, int npairs, const double* const* xs, const double* const* ys,
                 double* part, cudaStream_t s);
// XD = Xt + b/mult at idx (D's values) (mode 0) or Xt = XD - D (mode 1)
void launch_xd_from_xt(size_t NN, int mode, const double* in, const int32_t* idx, const double* bm,
                       double* out, cudaStream_t s);
// Lanczos helpers
void launch_gemv_cert(int N, const double* XD, const double* z, const double* v, double* w,
                      cudaStream_t s);  // w = XD v - z o v
void launch_basis_dots(int N, int k, const double* V, const double* w, double* h, cudaStream_t s);
void launch_basis_update(int N, int k, const double* V, const double* h, double* w, cudaStream_t s);
// Copy N x p_old into N x p_new (zero-padding new columns) or select columns via a p_old x p_new
// matrix (out = A W) - via launch_gemm.
void launch_pad_cols(int N, int p_old, int p_new, const double* in, double* out, cudaStream_t s);
// out[i] = +1 if u[i] >= 0 else -1
void launch_sign(int n, const double* u, double* out, cudaStream_t s);
void launch_set_cols(int N, int p, int c0, int nc, const double* src /*N x nc*/, double* out,
                     cudaStream_t s);

}  // namespace mds

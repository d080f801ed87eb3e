// Types shared by the host side of the batched solver (batched.cu) and its
// device code, which batched_k128.cu, batched_k256.cu and batched_k512.cu
// compile once per CTA size (in parallel: each instance of the device code is
// a large kernel).
#pragma once

#include <cstdint>

#include "common.cuh"

namespace mds {
namespace batch {

constexpr int kBMaxN = 128;
constexpr int kBMaxP = 32;
constexpr int kBPiece = 8;  // entries per piece of a class sum

struct BInst {
  int N, m, np;
  long long off_idx;    // N*N int32 (class of each entry)
  long long off_idx16;  // N*N uint16, the same
  long long off_cptr;   // m+1 int32: entries of class a at cent[cptr[a] .. cptr[a+1])
  long long off_cent;   // upper-triangle entries (r << 16) | c (r <= c), uint32
  long long off_cls;    // 3m doubles: mult, b, 1/mult
  long long off_invmf;  // m floats: 1/mult
  long long off_pstart; // np+1 int32: piece k holds entries pstart[k] .. pstart[k+1]
  long long off_pcls;   // np int32: class of each piece
  long long off_cpc;    // m+1 int32: pieces of class a at cpc[a] .. cpc[a+1]
  long long off_y0;     // element offset of the N x p0 starting factor in Y0
};

struct BParams {
  double sigma0, sigma_min, sigma_max, gamma, kappa1, kappa2, tol;
  double tol_grad_min, tol_grad_max, tol_grad_factor, rank_tol, neg_tol, tcg_floor, tcg_abs;
  double carry_t0, round_eta, sigma_stall;
  int p0, p_min, p_max, delta_max, max_outer, max_rtr, max_tcg, carry_halvings;
  int fp64;     // 1: FP64 Hessian-vector products (MANIDSDP_PREC_FP64)
  int profile;  // 1: per-phase clock64 cycles into BOut::cycles
};

struct BOut {  // per instance (the layout of manidsdp_batch_out)
  double value, eta_p, eta_d, eta_g, lambda_min;
  int status, p, outer, hessvecs;
  long long cycles[5];
};

// Per-CTA workspace offsets (doubles), for Nmax, mmax.
struct BLayout {
  long long XD, G, E;                                          // N*N (E: N*N + 6N + 32)
  long long S, St, ps;                                         // N(N+1)/2 upper entries
  long long Y, Yt, grad, eta, Heta, r, dlt, Hd, Up, U, GY, T;  // N*P
  long long y, yt, wd;                                         // m
  long long z, zt, tmpN, d, e, e2, beta, pv;                   // N
  long long ev;                                                // N + P
  long long Vk, ivs;                                           // P*N, 2*P*N
  long long M1d, M2d, gram, gvec, gev, cert;                   // P*P (gev P, cert 8)
  long long total;
};

__host__ __device__ inline BLayout make_layout(int N, int m) {
  BLayout L;
  long long o = 0;
  const long long nn = (long long)N * N, np = (long long)N * kBMaxP, pp = kBMaxP * kBMaxP;
  const long long nu = (long long)N * (N + 1) / 2;
  L.XD = o; o += nn; L.G = o; o += nn; L.E = o; o += nn + 6 * N + 32;
  L.S = o; o += nu; L.St = o; o += nu; L.ps = o; o += nu;
  L.Y = o; o += np; L.Yt = o; o += np; L.grad = o; o += np; L.eta = o; o += np;
  L.Heta = o; o += np; L.r = o; o += np; L.dlt = o; o += np; L.Hd = o; o += np;
  L.Up = o; o += np; L.U = o; o += np; L.GY = o; o += np; L.T = o; o += np;
  L.y = o; o += m; L.yt = o; o += m; L.wd = o; o += m;
  L.z = o; o += N; L.zt = o; o += N; L.tmpN = o; o += N; L.d = o; o += N;
  L.e = o; o += N; L.e2 = o; o += N; L.beta = o; o += N; L.pv = o; o += N;
  L.ev = o; o += N + kBMaxP;
  L.Vk = o; o += np; L.ivs = o; o += 2 * np;
  L.M1d = o; o += pp; L.M2d = o; o += pp; L.gram = o; o += pp; L.gvec = o; o += pp;
  L.gev = o; o += kBMaxP; L.cert = o; o += 8;
  L.total = o;
  return L;
}

using KernelFn = void (*)(int, const BInst*, const int*, const char*, const double*, BParams,
                          double*, long long, int, int, int*, BOut*, double*, const long long*);

// Per CTA size: the kernel and its dynamic shared memory for an instance
// (N, m, pieces np, row stride P4).
#define MDS_BATCH_SHAPE(NS)                                  \
  namespace NS {                                             \
  KernelFn kernel();                                         \
  unsigned smem_bytes(int N, int m, int np, int P4);         \
  }
MDS_BATCH_SHAPE(bt128)
MDS_BATCH_SHAPE(bt256)
MDS_BATCH_SHAPE(bt512)
#undef MDS_BATCH_SHAPE

}  // namespace batch
}  // namespace mds

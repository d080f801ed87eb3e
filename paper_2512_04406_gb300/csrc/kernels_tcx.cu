// Tensor-core products of the FP32 Hessian-vector product (Proposition 4.2) on
// the 5th-generation tensor cores, every operand staged by TMA:
//
//   SDDMM        W = Y Up' + Up Y' on upper-triangle 128 x 128 tiles: each entry
//                written to its slot of the class-ordered buffer (for the class
//                means w) and to the full N x N matrix W (both triangles)
//   gather GEMM  T = [G | sigma Q(W)] [Up ; Y] = G Up + sigma Q(W) Y   (K = 2N),
//                Q(W) = W - A*(w) formed entrywise in FP32 before the split, so
//                the large, nearly cancelling terms W Y and A*(w) Y never pass
//                through the tensor core's accumulator
//
// All are C = A B' with A (M x K) and B (ncol x K) K-major ("row-major with K
// contiguous") FP32 matrices given as TF32 pairs x = hi + lo (hi = tf32(x),
// lo = tf32(x - hi), both exact TF32 values, |x - hi - lo| <= 2^-23 |x|).  Each
// K step of 8 issues three tcgen05.mma kind::tf32 products lo*hi + hi*lo + hi*hi
// (the lo*lo term is below the representation error), accumulating in FP32 in
// tensor memory.  K is a sequence of segments, each with its own tensor maps
// (the blocks of the concatenation above, the two terms of the SDDMM).
//
// CTA: 192 threads.  Warp 0 (one lane) issues the TMA loads of a stage: 32
// K-values of each operand tile (A hi, A lo, B hi, B lo), one box of 128-byte
// rows per tile, landing in the 128-byte swizzled K-major layout (8-row atoms of
// 1024 bytes; 16-byte chunk j of row r stored at chunk j ^ (r % 8)).  Warp 1
// (one lane) issues the MMAs of a stage once its mbarrier reports the bytes
// landed (each K step of 8 is a 32-byte offset of the descriptor's start address
// inside the atom) and commits them to the stage's "empty" mbarrier, which hands
// the buffers back to the producer.  Warps 2-5 read the accumulator back with
// tcgen05.ld (each warp its quarter of the 128 TMEM lanes) and write the
// epilogue.  The tensor core's FP32 accumulation loses accuracy with the chain
// length, so a chain holds at most kXChain K-values: longer K ranges are split
// across CTAs (split-K partials) or across two TMEM accumulators added in the
// epilogue (SDDMM).
//
// Every mbarrier wait is bounded (about two seconds of SM clock); on expiry the
// CTA records an error in *err, waits (bounded) for the copies and MMAs it
// issued, frees its tensor memory and returns.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched through the runtime)

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace mds {
namespace {

constexpr int kXBM = 128;             // rows per CTA (MMA M)
constexpr int kXBK = 32;              // K values per pipeline stage (one 128-byte row)
constexpr int kXSeg = 4;              // K segments at most
constexpr int kXThreads = 192;
constexpr int kXChain = 640;          // K values per accumulation chain
constexpr long long kXSpin = 4000000000LL;  // ~2 s at 2 GHz

struct TcxArgs {
  CUtensorMap a_hi[kXSeg], a_lo[kXSeg], b_hi[kXSeg], b_lo[kXSeg];
  int koff[kXSeg + 1];  // segment s covers K values [koff[s], koff[s+1]), each a multiple of kXBK
  int ktot;             // koff[nseg]
  int M, ncol, bn;    // rows of A, rows of B (output columns), columns per CTA
  int kchunk;         // K values per CTA (split-K), a multiple of kXBK
  int nacc;           // TMEM accumulators per CTA (chains of <= kXChain each)
  int mode;           // 0: partial product out[split][M][ldo]; 1: SDDMM scatter
  int pairs;          // 1: TF32 pairs, three products per step; 0: hi parts only, one product
  float* out;
  int ldo;
  const int32_t* slot;  // mode 1: N x N slot map; perm: class-ordered buffer
  float* perm;
  float* wfull;         // mode 1: W at every entry (both triangles), leading dimension ldw
  int ldw;
  const int2* tiles;    // mode 1: (row tile, column tile) of each CTA, row <= column
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory descriptor of a K-major tile: start address,
// leading-dimension byte offset (between K-adjacent core matrices), stride byte
// offset (between row-adjacent core matrices), the fixed 0b001 at bits 46-48.
// Swizzle mode at bits 61-63: 0 none, 2 the 128-byte swizzle.
__device__ __forceinline__ uint64_t x_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo,
                                           uint32_t swizzle) {
  uint64_t d = uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(swizzle & 7u) << 61;
  return d;
}

// Instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t x_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) |
         (uint32_t(kXBM >> 4) << 24);
}

__device__ __forceinline__ void x_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                      uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void x_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void x_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void x_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void x_bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void x_bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool x_bar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete; false after ~2 s.
__device__ bool x_bar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!x_bar_test(bar, parity))
    if (clock64() - t0 > kXSpin) return false;
  return true;
}

// One TMA box {4 K-values, rows} of a 2-D tensor map at (x = k, y = row) into
// shared memory, completing bytes on the mbarrier.
__device__ __forceinline__ void x_tma2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                        uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 16 FP32 columns of this warp's 32 TMEM lanes: thread i gets lane (base + i).
__device__ __forceinline__ void x_tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}


// BK K-values per stage: 32, 128-byte rows with the 128-byte swizzle (16, 64-byte
// rows with the 64-byte swizzle, measured slower: not instantiated).
template <int BK>
__global__ void __launch_bounds__(kXThreads, 1) tcx3_kernel(const __grid_constant__ TcxArgs P,
                                                            int nstage) {
  extern __shared__ __align__(1024) unsigned char x_smem[];
  constexpr uint32_t kAtom = 8 * BK * 4;             // 8-row swizzle atom (bytes)
  constexpr uint32_t kSwz = BK == 32 ? 2u : 4u;      // descriptor swizzle mode
  const int bn = P.bn;
  const int a_bytes = kXBM * BK * 4;  // one A tile (hi or lo)
  const int b_bytes = bn * BK * 4;    // one B tile
  const int nt = P.pairs ? 2 : 1;     // tiles per operand
  const int stage_bytes = nt * (a_bytes + b_bytes);
  // 1024-byte aligned working area (the swizzle pattern repeats every 1024 bytes)
  const uint32_t sraw = smem_u32(x_smem);
  const uint32_t sbase = (sraw + 1023u) & ~1023u;
  unsigned char* gbase = x_smem + (sbase - sraw);
  uint64_t* full = reinterpret_cast<uint64_t*>(gbase + size_t(nstage) * stage_bytes);
  uint64_t* empty = full + nstage;
  uint64_t* accbar = empty + nstage;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accbar + 1);
  // issued, consumed, failed, epilogue go
  volatile int* counts = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  int m0, n0, split;
  if (P.mode == 1) {
    const int2 t = P.tiles[blockIdx.x];
    m0 = t.x * kXBM;
    n0 = t.y * bn;
    split = 0;
  } else {
    m0 = blockIdx.y * kXBM;
    n0 = blockIdx.x * bn;
    split = blockIdx.z;
  }
  const int kb = split * P.kchunk;
  const int ke = min(P.ktot, kb + P.kchunk);
  const int nst = ke > kb ? (ke - kb) / BK : 0;
  const int per_chain = (nst + P.nacc - 1) / max(1, P.nacc);
  int ncols_alloc = 32;
  while (ncols_alloc < P.nacc * bn) ncols_alloc <<= 1;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols_alloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < nstage; ++s) {
      x_bar_init(&full[s], 1);
      x_bar_init(&empty[s], 1);
    }
    x_bar_init(accbar, 1);
    counts[0] = counts[1] = counts[2] = counts[3] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  x_fence_before();
  __syncthreads();
  x_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- producer: one box per operand tile and stage ----
    for (int it = 0; it < nst; ++it) {
      const int s = it % nstage;
      if (it >= nstage && !x_bar_wait(&empty[s], uint32_t(((it / nstage) - 1) & 1))) {
        counts[2] = 1;
        break;
      }
      if (counts[2]) break;
      x_bar_expect_tx(&full[s], uint32_t(stage_bytes));
      const int k = kb + it * BK;
      int seg = 0;
      while (seg + 1 < kXSeg && k >= P.koff[seg + 1]) ++seg;
      const int kl = k - P.koff[seg];
      const uint32_t st = sbase + uint32_t(s * stage_bytes);
      x_tma2d(st, &P.a_hi[seg], kl, m0, &full[s]);
      x_tma2d(st + uint32_t(nt * a_bytes), &P.b_hi[seg], kl, n0, &full[s]);
      if (P.pairs) {
        x_tma2d(st + uint32_t(a_bytes), &P.a_lo[seg], kl, m0, &full[s]);
        x_tma2d(st + uint32_t(2 * a_bytes + b_bytes), &P.b_lo[seg], kl, n0, &full[s]);
      }
      counts[0] = it + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: three products per K step of 8 ----
    const uint32_t idesc = x_idesc(bn);
    int it = 0;
    for (; it < nst; ++it) {
      const int s = it % nstage;
      if (!x_bar_wait(&full[s], uint32_t((it / nstage) & 1)) || counts[2]) {
        counts[2] = 1;
        break;
      }
      x_fence_after();
      const int chain = it / per_chain;
      const bool first = it % per_chain == 0;
      const uint32_t acc = tmem + uint32_t(chain * bn);
      const uint32_t st = sbase + uint32_t(s * stage_bytes);
      const uint32_t ahi = st, alo = st + a_bytes;
      const uint32_t bhi = st + nt * a_bytes, blo = bhi + b_bytes;
#pragma unroll
      for (int ks = 0; ks < BK / 8; ++ks) {
        // K step of 8 values = a 32-byte offset inside the swizzled row;
        // row-adjacent 8-row atoms kAtom bytes apart
        const uint32_t o = uint32_t(ks * 32);
        const uint64_t dah = x_desc(ahi + o, 16, kAtom, kSwz), dal = x_desc(alo + o, 16, kAtom, kSwz);
        const uint64_t dbh = x_desc(bhi + o, 16, kAtom, kSwz), dbl = x_desc(blo + o, 16, kAtom, kSwz);
        if (P.pairs) {
          x_mma(acc, dal, dbh, idesc, (first && ks == 0) ? 0u : 1u);
          x_mma(acc, dah, dbl, idesc, 1u);
          x_mma(acc, dah, dbh, idesc, 1u);
        } else {
          x_mma(acc, dah, dbh, idesc, (first && ks == 0) ? 0u : 1u);
        }
      }
      x_commit(&empty[s]);
      counts[1] = it + 1;
    }
    if (it == nst) x_commit(accbar);  // arrives once every MMA above has completed
  } else if (warp >= 2) {
    // ---- epilogue: lane quarter (warp % 4) of the accumulator ----
    const int q = warp & 3;
    const int rl = q * 32 + lane;
    const int row = m0 + rl;
    const bool ok = nst == 0 || x_bar_wait(accbar, 0u);
    if (!ok) counts[2] = 1;
    x_fence_after();
    // one decision for all four epilogue warps (tcgen05.ld is a whole-warp
    // instruction and the staging below synchronises the four warps)
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (tid == 64) counts[3] = counts[2] ? 0 : 1;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (counts[3]) {
      const uint32_t lbase = tmem + (uint32_t(q * 32) << 16);
      float* tile = reinterpret_cast<float*>(gbase);  // mode 1: 128 x 129 staging tile
      for (int c0 = 0; c0 < bn; c0 += 16) {
        float v[16];
        if (nst > 0) {
          x_tmem_ld16(lbase + uint32_t(c0), v);
          for (int j = 1; j < P.nacc; ++j) {
            float u[16];
            x_tmem_ld16(lbase + uint32_t(j * bn + c0), u);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] += u[i];
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
        if (P.mode == 1) {
#pragma unroll
          for (int i = 0; i < 16; ++i) tile[rl * 129 + c0 + i] = v[i];
          continue;
        }
        if (row >= P.M) continue;
        const int cb = n0 + c0;
        float* dst = P.out + (size_t(split) * P.M + row) * P.ldo + cb;
        if (cb + 16 <= P.ncol && (P.ldo & 3) == 0) {
#pragma unroll
          for (int i = 0; i < 16; i += 4)
            *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else {
          for (int i = 0; i < 16; ++i)
            if (cb + i < P.ncol) dst[i] = v[i];
        }
      }
      if (P.mode == 1) {
        // the 128 epilogue threads, one column t each: the tile's rows into W
        // (and, off the diagonal, its columns into the mirrored rows of W) with
        // coalesced stores, then the upper-triangle entries to their class slots,
        // sixteen slot reads in flight per thread before the scattered writes
        asm volatile("bar.sync 1, 128;" ::: "memory");
        const int t = tid - 64;
        const int col = n0 + t;
        const int rn = min(kXBM, P.M - m0);
        if (col < P.ncol)
          for (int r = 0; r < rn; ++r) P.wfull[size_t(m0 + r) * P.ldw + col] = tile[r * 129 + t];
        if (n0 != m0 && m0 + t < P.M) {
          const int cn = min(kXBM, P.ncol - n0);
          for (int r = 0; r < cn; ++r) P.wfull[size_t(n0 + r) * P.ldw + m0 + t] = tile[t * 129 + r];
        }
        if (col < P.ncol) {
          const int rmax = min(rn, col - m0 + 1);  // rows r <= col
          for (int r0 = 0; r0 < rmax; r0 += 16) {
            int sl[16];
#pragma unroll
            for (int u = 0; u < 16; ++u)
              sl[u] = r0 + u < rmax ? P.slot[size_t(m0 + r0 + u) * P.ncol + col] : -1;
#pragma unroll
            for (int u = 0; u < 16; ++u)
              if (sl[u] >= 0)
                P.perm[sl[u]] = (col == m0 + r0 + u ? 1.f : 2.f) * tile[(r0 + u) * 129 + t];
          }
        }
      }
    }
  }
  __syncthreads();
  if (counts[2]) {
    // a wait expired: record it, then wait (bounded) for what this CTA issued
    if (tid == 0) {
      atomicExch(P.err, 1);
      for (int it = counts[1]; it < counts[0]; ++it)
        x_bar_wait(&full[it % nstage], uint32_t((it / nstage) & 1));
    }
    if (tid == 32 && counts[1] > 0) {
      const int it = counts[1] - 1;
      x_bar_wait(&empty[it % nstage], uint32_t((it / nstage) & 1));
    }
  }
  x_fence_before();
  __syncthreads();
  if (warp == 1) {
    x_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(ncols_alloc)
                 : "memory");
  }
}

// ---- operand preparation: FP32 values split into TF32 pairs ----------------
// Round to the nearest TF32 value (ties away from zero): add half a TF32 unit to
// the magnitude bits and clear the 13 low bits.
__device__ __forceinline__ float x_round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void x_split(float x, float& hi, float& lo) {
  hi = x_round_tf32(x);
  lo = x_round_tf32(x - hi);
}

// X (N x p FP64, leading dimension p) as TF32 pairs, row-major (leading dimension
// ld; skipped when hi is null) and, when hiT is given, transposed (p x N, leading
// dimension ldt).
__global__ void __launch_bounds__(256) x_split_rows_kernel(int N, int p, const double* __restrict__ X,
                                                           float* __restrict__ hi,
                                                           float* __restrict__ lo, int ld,
                                                           float* __restrict__ hiT,
                                                           float* __restrict__ loT, int ldt) {
  __shared__ float th[32][33], tl[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int r = r0 + i, c = c0 + tx;
    float h = 0.f, l = 0.f;
    if (r < N && c < p) {
      x_split(float(X[size_t(r) * p + c]), h, l);
      if (hi != nullptr) {
        hi[size_t(r) * ld + c] = h;
        lo[size_t(r) * ld + c] = l;
      }
    }
    th[i][tx] = h;
    tl[i][tx] = l;
  }
  if (hiT == nullptr) return;
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int c = c0 + i, r = r0 + tx;
    if (c < p && r < N) {
      hiT[size_t(c) * ldt + r] = th[tx][i];
      loT[size_t(c) * ldt + r] = tl[tx][i];
    }
  }
}

// G (N x N FP32, leading dimension N) or, with idx given, the projector residual
// gscale * (G - w[idx]) (G then the full W, leading dimension ld) as TF32 pairs with
// leading dimension ld.
__global__ void __launch_bounds__(256) x_split_matrix_kernel(int N, const float* __restrict__ G,
                                                             const int32_t* __restrict__ idx,
                                                             const float* __restrict__ w,
                                                             float gscale, float* __restrict__ hi,
                                                             float* __restrict__ lo, int ld) {
  const int r = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const size_t e = size_t(r) * N + c;
    const float x = idx != nullptr ? gscale * (G[size_t(r) * ld + c] - w[idx[e]]) : G[e];
    float h, l;
    x_split(x, h, l);
    hi[size_t(r) * ld + c] = h;
    lo[size_t(r) * ld + c] = l;
  }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (so
// the library does not link libcuda directly).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled x_encoder() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
  });
  if (fn == nullptr) throw DeviceError{cudaErrorNotSupported};
  return fn;
}

// 2-D map of a row-major FP32 matrix (rows x cols, leading dimension ld, ld a
// multiple of 4): boxes of 32 columns (128 bytes) x box_rows rows with the
// 128-byte swizzle; reads outside the matrix fill zeros.
void x_map(CUtensorMap* m, const float* base, int rows, int cols, int ld, int box_rows) {
  const int bk = kXBK;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld & 3) != 0 || box_rows < 1 ||
      box_rows > 256 || rows < 1 || cols < 1 || ld < cols)
    throw DeviceError{cudaErrorInvalidValue};
  const cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(ld) * sizeof(float)};
  const cuuint32_t box[2] = {uint32_t(bk), cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = x_encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base),
                                 dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 bk == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw DeviceError{cudaErrorInvalidValue};
}

int x_stage_bytes(int bn, int bk, int pairs) {
  return (pairs ? 2 : 1) * (kXBM * bk * 4 + bn * bk * 4);
}
int x_stages(int bn, int bk, int pairs) {
  return std::max(2, std::min(8, (200 * 1024) / x_stage_bytes(bn, bk, pairs)));
}
// stages + barriers + the 1024-byte alignment slack
size_t x_smem_bytes(int bn, int bk, int pairs, int nstage) {
  return size_t(nstage) * x_stage_bytes(bn, bk, pairs) + 256 + 1024;
}

void x_launch(const TcxArgs& a, dim3 grid, cudaStream_t s) {
  const int nst = x_stages(a.bn, kXBK, a.pairs);
  const size_t smem = x_smem_bytes(a.bn, kXBK, a.pairs, nst);
  static std::once_flag once;
  std::call_once(once, [] {
    size_t mx = 0;
    for (int bn = 16; bn <= 256; bn += 16)
      for (int pr : {0, 1}) mx = std::max(mx, x_smem_bytes(bn, kXBK, pr, x_stages(bn, kXBK, pr)));
    MDS_CUDA(cudaFuncSetAttribute(tcx3_kernel<kXBK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(mx)));
  });
  count_launches(1);
  tcx3_kernel<kXBK><<<grid, kXThreads, smem, s>>>(a, nst);
  MDS_CUDA(cudaGetLastError());
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }
// Output columns per CTA: all of them up to 256, else two halves.
int x_bn(int ncol) { return ncol <= 256 ? round_up(ncol, 16) : round_up((ncol + 1) / 2, 16); }

}  // namespace

int tcx_ld(int n) { return round_up(n, 4); }

void launch_tcx_split_rows(int N, int p, const double* X, float* hi, float* lo, int ld, float* hiT,
                           float* loT, int ldt, cudaStream_t s) {
  dim3 grid((p + 31) / 32, (N + 31) / 32);
  count_launches(1);
  x_split_rows_kernel<<<grid, 256, 0, s>>>(N, p, X, hi, lo, ld, hiT, loT, ldt);
  MDS_CUDA(cudaGetLastError());
}

void launch_tcx_split_matrix(int N, const float* G, const int32_t* idx, const float* w,
                             float gscale, float* hi, float* lo, int ld, cudaStream_t s) {
  dim3 grid(std::max(1, std::min(4, (N + 255) / 256)), N);
  count_launches(1);
  x_split_matrix_kernel<<<grid, 256, 0, s>>>(N, G, idx, w, gscale, hi, lo, ld);
  MDS_CUDA(cudaGetLastError());
}

int tcx_gather_splits(int N) { return (2 * round_up(N, kXBK) + kXChain - 1) / kXChain; }

int launch_tcx_gather(int N, int p, const float* Ghi, const float* Glo, const float* QWhi,
                      const float* QWlo, int ldg, const float* UThi, const float* UTlo,
                      const float* YThi, const float* YTlo, int ldt, float* part, size_t ws_bytes,
                      int* err, cudaStream_t s, int pairs) {
  if (p < 1 || p > kMaxP) throw DeviceError{cudaErrorInvalidValue};
  TcxArgs a{};
  const int bn = x_bn(p);
  // [G | sigma Q(W)] against [Up' ; Y']
  x_map(&a.a_hi[0], Ghi, N, N, ldg, kXBM);
  x_map(&a.a_lo[0], Glo, N, N, ldg, kXBM);
  x_map(&a.b_hi[0], UThi, p, N, ldt, bn);
  x_map(&a.b_lo[0], UTlo, p, N, ldt, bn);
  x_map(&a.a_hi[1], QWhi, N, N, ldg, kXBM);
  x_map(&a.a_lo[1], QWlo, N, N, ldg, kXBM);
  x_map(&a.b_hi[1], YThi, p, N, ldt, bn);
  x_map(&a.b_lo[1], YTlo, p, N, ldt, bn);
  const int kN = round_up(N, kXBK);
  a.koff[0] = 0;
  a.koff[1] = kN;
  a.koff[2] = a.koff[3] = a.koff[4] = 2 * kN;
  a.ktot = 2 * kN;
  a.M = N;
  a.ncol = p;
  a.bn = bn;
  a.kchunk = kXChain;
  a.nacc = 1;
  a.mode = 0;
  a.pairs = pairs;
  a.out = part;
  a.ldo = p;
  a.err = err;
  const int splits = tcx_gather_splits(N);
  if (size_t(splits) * N * p * sizeof(float) > ws_bytes) throw DeviceError{cudaErrorMemoryAllocation};
  x_launch(a, dim3((p + bn - 1) / bn, (N + kXBM - 1) / kXBM, splits), s);
  return splits;
}

void launch_tcx_sddmm(int N, int p, const float* Yhi, const float* Ylo, const float* Uhi,
                      const float* Ulo, int ld, const int32_t* slot, float* perm, float* wfull,
                      int ldw, const int2* tiles, int ntiles, int* err, cudaStream_t s,
                      int pairs) {
  if (p < 1 || p > kMaxP) throw DeviceError{cudaErrorInvalidValue};
  TcxArgs a{};
  // segment 0: Y Up' (A = Y, B = Up); segment 1: Up Y'
  x_map(&a.a_hi[0], Yhi, N, p, ld, kXBM);
  x_map(&a.a_lo[0], Ylo, N, p, ld, kXBM);
  x_map(&a.b_hi[0], Uhi, N, p, ld, kXBM);
  x_map(&a.b_lo[0], Ulo, N, p, ld, kXBM);
  x_map(&a.a_hi[1], Uhi, N, p, ld, kXBM);
  x_map(&a.a_lo[1], Ulo, N, p, ld, kXBM);
  x_map(&a.b_hi[1], Yhi, N, p, ld, kXBM);
  x_map(&a.b_lo[1], Ylo, N, p, ld, kXBM);
  const int kp = round_up(p, kXBK);
  a.koff[0] = 0;
  a.koff[1] = kp;
  a.koff[2] = a.koff[3] = a.koff[4] = 2 * kp;
  a.ktot = 2 * kp;
  a.M = N;
  a.ncol = N;
  a.bn = kXBM;
  a.kchunk = a.ktot;
  a.nacc = (a.ktot + kXChain - 1) / kXChain;  // <= 2 for p <= 512
  a.mode = 1;
  a.pairs = pairs;
  a.slot = slot;
  a.perm = perm;
  a.wfull = wfull;
  a.ldw = ldw;
  a.tiles = tiles;
  a.err = err;
  x_launch(a, dim3(ntiles), s);
}

// Upper-triangle 128 x 128 tile pairs (row tile <= column tile) of an N x N matrix.
std::vector<int2> tcx_upper_tiles(int N) {
  const int nt = (N + kXBM - 1) / kXBM;
  std::vector<int2> t;
  for (int i = 0; i < nt; ++i)
    for (int j = i; j < nt; ++j) t.push_back(make_int2(i, j));
  return t;
}

}  // namespace mds

// Gather GEMM of the Hessian-vector product (Proposition 4.2) on the
// 5th-generation tensor cores:
//   T = G U + A*(gscale w) Y  = [G | A*(gscale w)] [U ; Y],   gscale = -sigma,
// with A*(w)[b, g] = w[idx[b, g]] gathered from the index map while the operand
// tile is built.
//
// One CTA computes a 128-row block of T (all p columns) over one K range of g
// (split K; each split writes its partial product, reduced by the Hessian
// epilogue).  Per chunk of 16 values of g, 256 threads load 128 x 16 entries of
// G and of the index map (gathering w), 16 rows of U and of Y, split every
// value x into x ~ hi + lo (hi = tf32(x), lo = tf32(x - hi)) and store both
// halves in shared memory in the
// K-major core-matrix layout of tcgen05 (8 rows x 16 bytes per core matrix).
// One thread then issues tcgen05.mma kind::tf32 for the four products
// lo*lo + lo*hi + hi*lo + hi*hi per K step of 8 (smallest first; about 2^-22
// relative error per product, FP32 accumulation in tensor memory) and commits
// them to an mbarrier; two shared-memory stages let the next chunk's loads and
// stores overlap the running MMAs.  Every 20 chunks, and at the end, the
// accumulator (128 lanes x p columns of FP32 in TMEM) is read back with
// tcgen05.ld by the four warps whose lane quarters cover the 128 rows and added
// into the CTA's partial product in global memory.
//
// Every wait on an mbarrier is bounded (about two seconds of SM clock); on
// expiry the CTA records an error in *err, waits (bounded) for its MMAs in
// flight, frees its tensor memory and returns.
#include <algorithm>

#include "common.cuh"

namespace mds {
namespace {

constexpr int kTcBM = 128;          // rows of T per CTA (MMA M)
constexpr int kTcG = 16;            // values of g per chunk
constexpr int kTcThreads = 256;
constexpr int kTcATile = kTcBM * 2 * kTcG * 4;  // bytes of one 128 x 32 FP32 operand tile
constexpr long long kTcSpinCycles = 4000000000LL;  // ~2 s at 2 GHz
// Chunks accumulated in tensor memory before the accumulator is added into the
// partial product in global memory (FP32, round to nearest): 20 chunks = 640 K
// values per accumulation chain (at N = 3241 a split holds 19 chunks, so the
// drain only runs for larger N, where each drain costs ~20 us of pipeline stall).  The tensor core's own FP32 accumulation loses
// accuracy in proportion to the chain length (measured: 1.3e-5 relative Hess-vec
// error with 590-term chains at N = 3241, 9.5e-5 with 2906-term chains at N = 7261).
constexpr int kTcDrain = 20;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of tcgen05: start address, leading-dimension
// byte offset (between core matrices adjacent in K), stride byte offset
// (between core matrices adjacent in M/N), the fixed 0b001 at bits 46-48, no
// swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D in F32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) |
         (uint32_t(kTcBM >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes become visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete; false after ~2 s.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > kTcSpinCycles) return false;
  return true;
}

// Round to the nearest TF32 value (ties away from zero): add half a TF32 unit to
// the magnitude bits and clear the 13 low bits.
__device__ __forceinline__ float round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
// x ~ hi + lo, both exact TF32 values: hi = tf32(x), lo = tf32(x - hi) (x - hi is
// exact in FP32 by Sterbenz, |x - hi| <= 2^-11 |x|), so |x - hi - lo| <= 2^-23 |x|,
// the representation error of FP32 itself; rounding lo in software keeps the
// tensor core from truncating it (a bias that grows with the length of the sum).
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = round_tf32(x);
  lo = round_tf32(x - hi);
}

// 16 FP32 columns of this warp's 32 TMEM lanes: thread i gets lane (base lane + i).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
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

// Byte offset of element (row, k) of a K-major operand tile with 32 values of
// K: core matrix (row / 8, k / 4) at ((row / 8) * 8 + k / 4) * 128, its rows 16
// bytes apart.  So the leading-dimension (K) offset is 128 B and the stride (M/N)
// offset 1024 B; a K step of 8 starts at (k / 4) * 128.
__device__ __forceinline__ uint32_t tile_off(int row, int kg) {
  return uint32_t(((row >> 3) * 8 + kg) * 128 + (row & 7) * 16);
}

__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gather_gemm_kernel(int N, int ncol, int np, int kchunk, const float* __restrict__ G,
                          const float* __restrict__ U, const int32_t* __restrict__ idx,
                          const float* __restrict__ w, float gscale,
                          const float* __restrict__ Y, float* __restrict__ part,
                          int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  const int btile = np * 2 * kTcG * 4;                   // bytes of one np x 32 operand tile
  const int stage_bytes = 2 * kTcATile + 2 * btile;       // A hi, A lo, B hi, B lo
  uint64_t* bars = reinterpret_cast<uint64_t*>(tc_smem + 2 * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcBM;
  const int kb = blockIdx.y * kchunk, ke = min(N, kb + kchunk);
  const int nchunks = ke > kb ? (ke - kb + kTcG - 1) / kTcG : 0;
  const uint32_t ncols = np <= 32 ? 32u : np <= 64 ? 64u : np <= 128 ? 128u : 256u;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // A loader: row r = tid / 2 of the block, values of g at h * 8 .. h * 8 + 7 of the chunk
  const int ar = tid >> 1, ah = tid & 1;
  const int grow = m0 + ar;
  const bool row_ok = grow < N;
  const size_t rowbase = size_t(row_ok ? grow : 0) * N;
  // B loader: items (n, kg), kg < 4 from U, kg >= 4 from Y, 4 consecutive g each
  const int nitems = 8 * np;

  float ga[8], wa[8];
  int ia[8];
  float4 bq[8];
  auto load_idx = [&](int c) {
    const int g0 = kb + c * kTcG + ah * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int g = g0 + i;
      ia[i] = (row_ok && g < ke) ? idx[rowbase + g] : -1;
    }
  };
  auto load_rest = [&](int c) {  // G and gathered w (from ia), and the B items
    const int g0 = kb + c * kTcG + ah * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int g = g0 + i;
      ga[i] = (row_ok && g < ke) ? G[rowbase + g] : 0.f;
      wa[i] = ia[i] >= 0 ? gscale * w[ia[i]] : 0.f;
    }
    const int gb = kb + c * kTcG;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int it = tid + q * kTcThreads;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (it < nitems) {
        const int n = it % np, kg = it / np;
        const float* src = kg < 4 ? U : Y;
        const int g = gb + (kg & 3) * 4;
        if (n < ncol) {
          v.x = g + 0 < ke ? src[size_t(g + 0) * ncol + n] : 0.f;
          v.y = g + 1 < ke ? src[size_t(g + 1) * ncol + n] : 0.f;
          v.z = g + 2 < ke ? src[size_t(g + 2) * ncol + n] : 0.f;
          v.w = g + 3 < ke ? src[size_t(g + 3) * ncol + n] : 0.f;
        }
      }
      bq[q] = v;
    }
  };
  auto store = [&](int s) {
    unsigned char* base = tc_smem + s * stage_bytes;
    unsigned char* ahi = base;
    unsigned char* alo = base + kTcATile;
    unsigned char* bhi = base + 2 * kTcATile;
    unsigned char* blo = bhi + btile;
#pragma unroll
    for (int part_ = 0; part_ < 2; ++part_) {
      const float* v = part_ == 0 ? ga : wa;
#pragma unroll
      for (int e2 = 0; e2 < 2; ++e2) {
        const int kg = part_ * 4 + ah * 2 + e2;
        float4 hi, lo;
        split_tf32(v[e2 * 4 + 0], hi.x, lo.x);
        split_tf32(v[e2 * 4 + 1], hi.y, lo.y);
        split_tf32(v[e2 * 4 + 2], hi.z, lo.z);
        split_tf32(v[e2 * 4 + 3], hi.w, lo.w);
        const uint32_t off = tile_off(ar, kg);
        *reinterpret_cast<float4*>(ahi + off) = hi;
        *reinterpret_cast<float4*>(alo + off) = lo;
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int it = tid + q * kTcThreads;
      if (it < nitems) {
        const int n = it % np, kg = it / np;
        float4 hi, lo;
        split_tf32(bq[q].x, hi.x, lo.x);
        split_tf32(bq[q].y, hi.y, lo.y);
        split_tf32(bq[q].z, hi.z, lo.z);
        split_tf32(bq[q].w, hi.w, lo.w);
        const uint32_t off = tile_off(n, kg);
        *reinterpret_cast<float4*>(bhi + off) = hi;
        *reinterpret_cast<float4*>(blo + off) = lo;
      }
    }
  };

  const uint32_t idesc = tc_idesc(np);
  bool failed = false;
  int last = -1;  // last chunk whose MMAs were committed
  bool drained = false;  // the partial product already holds earlier chains
  float* op = part + size_t(blockIdx.y) * N * ncol;
  // warps 0-3 (lane quarters 0-3 of TMEM): row m0 + warp * 32 + lane of the
  // accumulator into the partial product, written (add = false) or added
  auto drain = [&](bool add) {
    if (warp < 4) {
      const int row = m0 + warp * 32 + lane;
      for (int c0 = 0; c0 < np; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c0), v);
        if (row < N) {
          float* dst = op + size_t(row) * ncol + c0;
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c0 + i < ncol) dst[i] = add ? dst[i] + v[i] : v[i];
        }
      }
    }
  };
  if (nchunks > 0) {
    load_idx(0);
    load_rest(0);
    if (nchunks > 1) load_idx(1);
  }
  for (int c = 0; c < nchunks; ++c) {
    const int s = c & 1;
    if (c >= 2) {
      const bool ok = mbar_wait(&bars[s], uint32_t(((c - 2) >> 1) & 1));
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    store(s);
    if (c + 1 < nchunks) {
      load_rest(c + 1);  // uses the index values loaded one chunk earlier
      if (c + 2 < nchunks) load_idx(c + 2);
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t base = smem_addr(tc_smem + s * stage_bytes);
      const uint32_t ahi = base, alo = base + kTcATile;
      const uint32_t bhi = base + 2 * kTcATile, blo = bhi + btile;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t ko = kk * 256;  // two core matrices of K per step of 8
        const uint64_t dah = tc_desc(ahi + ko, 128, 1024), dal = tc_desc(alo + ko, 128, 1024);
        const uint64_t dbh = tc_desc(bhi + ko, 128, 1024), dbl = tc_desc(blo + ko, 128, 1024);
        tc_mma(tmem, dal, dbl, idesc, (c % kTcDrain != 0 || kk > 0) ? 1u : 0u);
        tc_mma(tmem, dal, dbh, idesc, 1u);
        tc_mma(tmem, dah, dbl, idesc, 1u);
        tc_mma(tmem, dah, dbh, idesc, 1u);
      }
      tc_commit(&bars[s]);
    }
    last = c;
    if ((c + 1) % kTcDrain == 0 && c + 1 < nchunks) {
      // end of an accumulation chain: wait for its MMAs, add the accumulator into
      // the partial product; the next chunk starts a new chain
      const bool ok = mbar_wait(&bars[s], uint32_t((c >> 1) & 1));
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after();
      drain(drained);
      drained = true;
      tc_fence_before();
      __syncthreads();
    }
  }
  // wait for the last committed chunk's MMAs (its commit covers all earlier
  // ones); after a failed wait this is the bounded wait for MMAs in flight
  if (last >= 0) {
    const bool ok = mbar_wait(&bars[last & 1], uint32_t((last >> 1) & 1));
    if (__syncthreads_or(!ok)) failed = true;
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
  } else if (nchunks > 0) {
    tc_fence_after();
    drain(drained);
  } else if (warp < 4) {  // empty K range: a zero partial product
    const int row = m0 + warp * 32 + lane;
    if (row < N)
      for (int c0 = 0; c0 < ncol; ++c0) op[size_t(row) * ncol + c0] = 0.f;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
}

size_t tc_smem_bytes(int np) {
  return size_t(2) * (2 * kTcATile + 2 * np * 2 * kTcG * 4) + 64;
}

}  // namespace

void tc_gather_gemm_prepare() {
  MDS_CUDA(cudaFuncSetAttribute(tc_gather_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(tc_smem_bytes(256))));
}

// Split-K layout of the kernel: one wave of CTAs (two per SM when the shared
// memory allows), each split at least 64 values of g, K ranges in whole chunks.
static int tc_split_count(int N, int ncol, size_t ws_bytes, int* kchunk_out) {
  const int np = (ncol + 15) / 16 * 16;
  const int per_sm = tc_smem_bytes(np) <= 110 * 1024 ? 2 : 1;
  const int gy = (N + kTcBM - 1) / kTcBM;
  int splits = std::max(1, (152 * per_sm) / gy);
  splits = std::min(splits, std::max(1, N / 64));
  const size_t per = size_t(N) * ncol * sizeof(float);
  if (size_t(splits + 1) * per > ws_bytes) splits = int(ws_bytes / per) - 1;  // +1: YM slice
  if (splits < 1) throw DeviceError{cudaErrorMemoryAllocation};
  int kchunk = (N + splits - 1) / splits;
  kchunk = (kchunk + kTcG - 1) / kTcG * kTcG;
  if (kchunk_out) *kchunk_out = kchunk;
  return (N + kchunk - 1) / kchunk;
}

int tc_gather_gemm_splits(int N, int ncol, size_t ws_bytes) {
  return tc_split_count(N, ncol, ws_bytes, nullptr);
}

int launch_tc_gather_gemm_partials(int N, int ncol, const float* G, const float* U,
                                   const int32_t* idx, const float* w, float gscale,
                                   const float* Y, void* ws, size_t ws_bytes, int* err,
                                   cudaStream_t s) {
  if (ncol < 1 || ncol > 256) throw DeviceError{cudaErrorInvalidValue};
  const int np = (ncol + 15) / 16 * 16;
  int kchunk = 0;
  const int splits = tc_split_count(N, ncol, ws_bytes, &kchunk);
  dim3 grid((N + kTcBM - 1) / kTcBM, splits);
  count_launches(1);
  tc_gather_gemm_kernel<<<grid, kTcThreads, tc_smem_bytes(np), s>>>(
      N, ncol, np, kchunk, G, U, idx, w, gscale, Y, static_cast<float*>(ws), err);
  MDS_CUDA(cudaGetLastError());
  return splits;
}

}  // namespace mds

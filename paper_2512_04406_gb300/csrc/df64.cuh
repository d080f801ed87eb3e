// Double-float ("df64") arithmetic on the FP32 pipe.
//
// GB300 issues FP64 FMAs at 1/64 of the FP32 rate, so dot products that need
// FP64-level accuracy are computed here as compensated FP32 sums:
//   * a value x in FP64 is held as the float pair (hi, lo) with hi = fl32(x),
//     lo = fl32(x - hi): about 48 significant bits;
//   * a product a*b is hi*hi (exact as p + e via the FMA-based TwoProd of
//     Dekker's error-free transformations) plus the cross terms hi*lo + lo*hi;
//   * sums use Knuth's TwoSum (exact error of a float addition), so the
//     accumulated main part and its running compensation together carry about
//     2^-46 relative accuracy, like an FP64 recursive sum of the same terms.
// Only the published error-free transformations are used; nothing here depends
// on a vendor math routine.  The explicitly rounded intrinsics (__fmul_rn,
// __fadd_rn, __fsub_rn) keep the compiler from contracting a product and a sum
// into one FMA, which would break the transformations.
#pragma once

struct df64acc {
  float s;  // running float sum of the hi*hi products
  float c;  // running compensation: TwoSum errors, product errors, cross terms
};

__device__ __forceinline__ void df64_split(double x, float* hi, float* lo) {
  const float h = __double2float_rn(x);
  *hi = h;
  *lo = __double2float_rn(__dsub_rn(x, double(h)));
}

// acc += (ah + al) * (bh + bl), dropping al*bl (below 2^-48 of the product).
__device__ __forceinline__ void df64_fma(df64acc& acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);  // p + e == ah*bh exactly
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  // TwoSum(acc.s, p): t + err == acc.s + p exactly
  const float t = __fadd_rn(acc.s, p);
  const float bb = __fsub_rn(t, acc.s);
  const float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  acc.s = t;
  acc.c = __fadd_rn(acc.c, __fadd_rn(err, e));
}

__device__ __forceinline__ double df64_value(const df64acc& a) {
  return double(a.s) + double(a.c);
}

// Double-float ("float-float") arithmetic for FP64 products on the FP32 pipes.
//
// On this part an FP64 fused multiply-add issues at about 1/64 of the FP32 rate, and the
// FP64 conversions and adds share that pipe.  The tall-skinny FP64 products of the
// refinement phase therefore keep their data in FP64 but form their sums from pairs of
// floats, with the classical error-free transformations:
//   * splitting: x = hi + lo with hi the leading 24 bits of the double and lo the rest
//     rounded to a float (|x - hi - lo| <= 2^-47 |x|), done with integer operations only;
//   * TwoProduct with a fused multiply-add (the exact error of a float product), and
//     Knuth's TwoSum (the exact error of a float sum);
// and the sums follow the compensated dot product of Ogita, Rump and Oishi ("Accurate
// sum and dot product", 2005): each term's product error and each addition's error go
// to a second float, so a chunk of k terms is summed to about sqrt(k) 2^-48 relative to
// the sum of |terms|.  Chunks are combined in FP64.  Every float operation below is an
// explicit round-to-nearest intrinsic, so the compiler cannot contract or reorder them.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace lobpcg {

// x = hi + lo, hi = x truncated to 24 significant bits, lo = the remaining bits rounded
// to a float.  |x| outside [2^-74, 2^127] loses lo (|x| < 2^-74: hi and lo may be 0;
// the absolute error is below 2^-74 |x|'s scale, far under the blocks' rounding) or gives
// +-inf; NaN stays NaN.
__device__ __forceinline__ float2 df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);  // biased double exponent
  if (e >= 1151) {                           // |x| >= 2^128, inf or NaN
    const bool nan = e == 0x7ff && (((hw & 0xfffffu) | lw) != 0u);
    return make_float2(__uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u)), 0.f);
  }
  if (e < 897) return make_float2(__uint_as_float(sign), 0.f);  // |x| < 2^-126
  const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | m23);
  float lo = 0.f;
  if (e >= 949) {
    // low 29 mantissa bits, weight 2^(e - 1075) per unit
    const unsigned r = lw & 0x1fffffffu;
    const float scale = __uint_as_float((unsigned)(e - 948) << 23);
    lo = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(r), scale)) | sign);
  }
  return make_float2(hi, lo);
}

// Exact float -> double by bit assembly (no FP64 instruction); subnormal floats map to 0.
__device__ __forceinline__ double df_widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0xffu) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull |
                                                           ((unsigned long long)(u & 0x7fffffu) << 29)));
  const unsigned long long bits = sign | ((unsigned long long)(e + 896u) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// Running double-float sum (hi, lo) of products.
struct DfAcc {
  float h, l;
};

__device__ __forceinline__ void df_zero(DfAcc& a) { a.h = 0.f, a.l = 0.f; }

// a += x * y for x, y given as (hi, lo) pairs: TwoProduct of the leading parts, the cross
// terms and the product error in the low word, TwoSum of the leading part into the sum,
// then a Fast2Sum renormalisation so |a.l| stays below half an ulp of a.h.
__device__ __forceinline__ void df_fma(DfAcc& a, float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  const float s = __fadd_rn(a.h, p);
  const float bb = __fsub_rn(s, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float t = __fadd_rn(a.l, __fadd_rn(err, e));
  a.h = __fadd_rn(s, t);
  a.l = __fsub_rn(t, __fsub_rn(a.h, s));
}

// The pair's value in FP64 (two widenings and one FP64 add).
__device__ __forceinline__ double df_value(const DfAcc& a) { return df_widen(a.h) + df_widen(a.l); }

}  // namespace lobpcg

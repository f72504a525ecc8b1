// Float-float ("double-float") arithmetic: a value is the unevaluated sum
// h + l of two floats, |l| <= ulp(h).  The error-free sum and product are
// Knuth's TwoSum and the fma form of Dekker's product (Knuth, TAOCP vol. 2,
// 4.2.2; Dekker 1971); the operations built on them keep about 47 bits of
// precision.  Used where the float64 pipe of this part (about 1/64 of the
// float32 rate) would bound a latency chain: the 64-wide diagonal blocks of
// the split-precision Cholesky.  Every rounding step is an explicit _rn
// intrinsic so that the compiler cannot contract or reorder them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qmlgb {

struct dfl {
  float h, l;
};

// a + b exactly as s + e (TwoSum)
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// a + b exactly when |a| >= |b| (FastTwoSum)
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a b exactly as p + e
__device__ __forceinline__ dfl df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// x y
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return df_fast_two_sum(p, e);
}
// a - x y; the error is a few units of 2^-48 (|a| + |x y|)
__device__ __forceinline__ dfl df_fms(dfl a, dfl x, dfl y) {
  const float p = __fmul_rn(x.h, y.h);
  float pe = __fmaf_rn(x.h, y.h, -p);
  pe = __fmaf_rn(x.h, y.l, pe);
  pe = __fmaf_rn(x.l, y.h, pe);  // x y = p + pe
  const dfl s = df_two_sum(a.h, -p);
  return df_two_sum(s.h, __fadd_rn(s.l, __fsub_rn(a.l, pe)));
}
// x + y
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  const dfl s = df_two_sum(x.h, y.h);
  return df_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
// 1 / sqrt(d), d > 0: the float estimate y, then one Halley step
// r = y (1 + e / 2 + 3 e^2 / 8) on the residual e = 1 - d y^2, which is formed
// in float-float (d y^2 is within 2^-20 of 1, so 1 - (d y^2)_h is exact); the
// cubic term of the step leaves O(e^3), below the float-float rounding.
__device__ __forceinline__ dfl df_rsqrt(dfl d) {
  const float y = rsqrtf(d.h);
  const dfl u = df_mul(d, df_two_prod(y, y));
  const float e = __fsub_rn(__fsub_rn(1.0f, u.h), u.l);
  const dfl ye = df_two_prod(y, e);  // exact; halving is exact too
  const float cubic = __fmul_rn(__fmul_rn(0.375f, e), ye.h);
  const dfl r = df_fast_two_sum(y, __fmul_rn(0.5f, ye.h));
  return df_fast_two_sum(r.h, __fadd_rn(r.l, __fmaf_rn(0.5f, ye.l, cubic)));
}

// float64 x times 2^-s as float-float, by integer operations on the bit
// pattern (no float64 instruction): the leading 24 significand bits
// (truncated) and the next 29 rounded to a float, then renormalised so that
// |l| <= ulp(h) / 2.  Magnitudes below 2^-126 after scaling become 0;
// infinities and NaN become NaN.
__device__ __forceinline__ float pow2f(int e) {  // 2^e for -126 <= e <= 127
  return __int_as_float((e + 127) << 23);
}
__device__ __forceinline__ dfl df_from_double(double x, int s) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int E = (int)((hi >> 20) & 0x7FFu);
  if (E == 0x7FF) return {__int_as_float(0x7FC00000), 0.0f};
  const int e = E - 1023 - s;
  if (E == 0 || e < -126) return {0.0f, 0.0f};
  if (e > 127) return {__int_as_float((int)(sign | 0x7F800000u)), 0.0f};
  const unsigned mh = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const float h = __int_as_float((int)(sign | ((unsigned)(e + 127) << 23) | mh));
  const float r = __fmul_rn(__fmul_rn(__uint2float_rn(lo & 0x1FFFFFFFu), 0x1p-52f), pow2f(e));
  return df_fast_two_sum(h, sign ? -r : r);
}
// float f times 2^s as float64 by integer operations (f normal or zero;
// subnormal f become 0)
__device__ __forceinline__ double double_from_float(float f, int s) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned E = (u >> 23) & 0xFFu;
  if (E == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (E == 0xFFu) return __hiloint2double((int)((u & 0x80000000u) | 0x7FF80000u), 0);
  const unsigned hi = (u & 0x80000000u) | ((E + 896u + (unsigned)s) << 20) | ((u & 0x7FFFFFu) >> 3);
  return __hiloint2double((int)hi, (int)((u & 7u) << 29));
}
// (h + l) 2^s rounded to float64: one float64 add
__device__ __forceinline__ double df_to_double(dfl v, int s) {
  return double_from_float(v.h, s) + double_from_float(v.l, s);
}

// Packed lower triangle of a kNB x kNB float-float matrix, column-major:
// entry (j, c), j >= c, at c kNB - c (c - 1) / 2 + (j - c); 2080 entries for
// kNB = 64, followed by the 64 row exponents (as int) in the slot layout of
// the split Cholesky.
__host__ __device__ constexpr int packed_off(int c, int nb) { return c * nb - c * (c - 1) / 2; }

}  // namespace qmlgb

// Double-word ("double-float") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| below one
// unit in the last place of hi, about 48 significant bits.  The operations are
// the classical error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact rounding
//     error of that sum, six additions, no condition on |a|, |b|;
//   Fast2Sum (Dekker 1971): the same in three additions when |a| >= |b|;
//   TwoProd with a fused multiply-add: p = fl(a b), e = fma(a, b, -p) is the
//     exact error of the product;
// composed as in the "sloppy" double-word addition and the double-word product
// analysed by Joldes, Muller and Popescu (ACM TOMS 44, 2017): relative error a
// few units of 2^-48 per operation, measured against the sum of the operands'
// magnitudes when an addition cancels (the same form FP64 rounding has for
// data that carry their own rounding error).  Every operation goes through
// the _rn intrinsics, which the compiler never contracts or reassociates.
//
// Why: this GPU retires 2 FP64 fused multiply-adds per clock per SM against 128
// FP32 ones, so an element kernel in double-word arithmetic (7 to 15 FP32
// instructions per FP64-class operation) outruns the same kernel in FP64.
//
// Conversions from and to FP64 use integer bit manipulation only (no FP64
// instruction).  A double of magnitude below 2^-126 converts to zero; values
// of that size do not occur in the operator's inputs (displacements, and the
// element geometry and material scales).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace gsw {

// keep the FP64 / FP32 fma visible next to the double-word overload below
using ::fma;

struct dw {
  float hi, lo;
  dw() = default;
  __host__ __device__ constexpr dw(float h, float l) : hi(h), lo(l) {}
  // small integer constants of the element formulas (exact in a float)
  __host__ __device__ constexpr explicit dw(int c) : hi((float)c), lo(0.0f) {}
};

// ---- error-free transformations -------------------------------------------------

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ dw fast_two_sum(float a, float b) {  // |a| >= |b| (or a = 0)
  const float s = __fadd_rn(a, b);
  return dw(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// ---- arithmetic ---------------------------------------------------------------

__device__ __forceinline__ dw operator+(dw a, dw b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s, e);
}

__device__ __forceinline__ dw operator-(dw a) { return dw(-a.hi, -a.lo); }

__device__ __forceinline__ dw operator-(dw a, dw b) { return a + (-b); }

__device__ __forceinline__ dw& operator+=(dw& a, dw b) {
  a = a + b;
  return a;
}

__device__ __forceinline__ dw operator*(dw a, dw b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a b + c with one final normalisation
__device__ __forceinline__ dw fma(dw a, dw b, dw c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  two_sum(p, c.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return fast_two_sum(s, t);
}

// Unnormalised variants for intermediate results that feed another
// double-word operation at once: the final Fast2Sum is skipped, so lo may
// exceed half an ulp of hi (it stays below about 2^-22 |hi| unless the sum
// cancels, and then its error is still bounded by the operands' magnitudes).
// Every operation above accepts such a pair as input.
__device__ __forceinline__ dw add_u(dw a, dw b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return dw(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dw sub_u(dw a, dw b) { return add_u(a, -b); }

__device__ __forceinline__ dw mul_u(dw a, dw b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  return dw(p, __fmaf_rn(a.lo, b.hi, e));
}

__device__ __forceinline__ dw fma_u(dw a, dw b, dw c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  two_sum(p, c.hi, s, t);
  return dw(s, __fadd_rn(t, __fadd_rn(e, c.lo)));
}

// ---- products with an exact float constant ----------------------------------------

__host__ __device__ constexpr bool pow2_const(float c) {
  return c == 1.0f || c == 2.0f || c == 4.0f || c == 8.0f || c == 16.0f || c == -1.0f || c == -2.0f ||
         c == -4.0f || c == -8.0f || c == -16.0f;
}

// c x; the branch folds at compile time for a literal c
__device__ __forceinline__ dw kmul(float c, dw x) {
  if (pow2_const(c)) return dw(__fmul_rn(c, x.hi), __fmul_rn(c, x.lo));
  const float p = __fmul_rn(c, x.hi);
  float e = __fmaf_rn(c, x.hi, -p);
  e = __fmaf_rn(c, x.lo, e);
  return fast_two_sum(p, e);
}

// c x + y
__device__ __forceinline__ dw kfma(float c, dw x, dw y) {
  float p, e;
  if (pow2_const(c)) {
    p = __fmul_rn(c, x.hi);
    e = __fmul_rn(c, x.lo);
  } else {
    p = __fmul_rn(c, x.hi);
    e = __fmaf_rn(c, x.hi, -p);
    e = __fmaf_rn(c, x.lo, e);
  }
  float s, t;
  two_sum(p, y.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(e, y.lo));
  return fast_two_sum(s, t);
}

// c x + y, unnormalised
__device__ __forceinline__ dw kfma_u(float c, dw x, dw y) {
  float p, e;
  if (pow2_const(c)) {
    p = __fmul_rn(c, x.hi);
    e = __fmul_rn(c, x.lo);
  } else {
    p = __fmul_rn(c, x.hi);
    e = __fmaf_rn(c, x.hi, -p);
    e = __fmaf_rn(c, x.lo, e);
  }
  float s, t;
  two_sum(p, y.hi, s, t);
  return dw(s, __fadd_rn(t, __fadd_rn(e, y.lo)));
}

// ---- conversions ------------------------------------------------------------------

// 2^k as a float for k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }

// Split a double into hi (its leading 24 significant bits, truncated) and lo
// (the next 23, truncated): relative error below 2^-46.  Integer operations,
// two FP32 multiplications and one FP32 addition.
__device__ __forceinline__ dw to_dw(double x) {
  const uint32_t h = (uint32_t)__double2hiint(x);
  const uint32_t l = (uint32_t)__double2loint(x);
  const uint32_t sign = h & 0x80000000u;
  const int e = (int)((h >> 20) & 0x7FFu);  // biased FP64 exponent
  const int fe = e - 1023 + 127;            // biased FP32 exponent of hi
  if (fe <= 0) return dw(__uint_as_float(sign), 0.0f);
  if (fe >= 255)  // overflow to infinity; a NaN stays a NaN
    return dw(__uint_as_float(sign | 0x7F800000u | ((e == 2047 && ((h & 0xFFFFFu) | l)) ? 0x400000u : 0u)), 0.0f);
  const uint32_t m23 = ((h & 0xFFFFFu) << 3) | (l >> 29);
  const float hi = __uint_as_float(sign | ((uint32_t)fe << 23) | m23);
  // the 29 remaining significand bits, top 23 kept: r23 * 2^(e - 1023 - 46)
  const uint32_t r23 = (l & 0x1FFFFFFFu) >> 6;
  const float r = __fsub_rn(__uint_as_float(0x4B000000u | r23), 8388608.0f);  // exact: r23 < 2^23
  const int k = e - 1069;  // in [-172, 81]: applied as two normal powers of two
  const int k1 = k >> 1, k2 = k - k1;
  const float lo = __fmul_rn(__fmul_rn(r, pow2f(k1)), pow2f(k2));
  // |lo| < ulp(hi): one Fast2Sum gives the round-to-nearest pair
  return fast_two_sum(hi, __uint_as_float(__float_as_uint(lo) | sign));
}

// A float as a double (exact), by bit manipulation; subnormal floats give 0.
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t fe = (u >> 23) & 0xFFu;
  if (fe == 0u) return __hiloint2double((int)sign, 0);
  const uint32_t m = u & 0x7FFFFFu;
  if (fe == 255u) return __hiloint2double((int)(sign | 0x7FF00000u | (m ? 0x80000u : 0u)), 0);
  return __hiloint2double((int)(sign | ((fe + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// hi + lo rounded to a double (one FP64 addition)
__device__ __forceinline__ double to_double(dw a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

}  // namespace gsw

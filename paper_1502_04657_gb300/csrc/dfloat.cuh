// Double-float arithmetic for the nonlinear kernels of the mixed-precision modes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, which
// carries about 48 significant bits (relative rounding ~2^-47 per operation instead of FP64's
// 2^-53).  Everything runs on the FP32 pipes, which issue at 64x the FP64 rate on this part:
// a product costs 7 FP32 instructions, a sum 11 and a fused multiply-add 15, against one
// FP64 instruction at 1/64 of the rate.  The building blocks are the error-free
// transformations of Dekker and Knuth (T. J. Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971; D. E. Knuth, TAOCP vol. 2,
// section 4.2.2): two_prod gives the exact rounding error of an FP32 product with one FMA,
// two_sum that of a sum with six additions, fast_two_sum renormalises a pair whose first
// member dominates.  Sums use the "sloppy" double-float addition, exact to ~2^-47 relative
// to |x| + |y|: the kernels that use it add terms of one sign (products of the positive
// ground-state values), where that is ~2^-47 relative to the result.  Every FP32 operation is
// an explicitly rounded intrinsic (__fadd_rn, __fmul_rn, fmaf), so the compiler cannot fuse a
// product into a following sum and break an error-free transformation.
#pragma once

#include <stdint.h>

#include "fmg_internal.h"

namespace fmg {

using ::fma;  // the FP64 / FP32 overloads stay visible beside the double-float one below

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // small integers (exact in FP32)
  __host__ __device__ constexpr dfloat(int v) : hi((float)v), lo(0.0f) {}
  // compile-time constants: nearest FP32 and the nearest FP32 of the remainder
  __host__ __device__ constexpr explicit dfloat(double v)
      : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return dfloat(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  const dfloat s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }

__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }

// 2 x, exact (both parts scaled), and its FP64 counterpart: one FP64 addition
__device__ __forceinline__ dfloat twice(dfloat x) {
  return dfloat(__fmul_rn(2.0f, x.hi), __fmul_rn(2.0f, x.lo));
}
__device__ __forceinline__ double twice(double x) { return x + x; }

__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);  // exact: x.hi y.hi = p + e
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// x y + z with one renormalisation
__device__ __forceinline__ dfloat fma(dfloat x, dfloat y, dfloat z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  const dfloat s = two_sum(p, z.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, z.lo)));
}

// FP32 -> FP64, exact, on the integer pipes (normal numbers and zero; double-float values of
// the kernels' magnitudes are never subnormal in FP32)
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0) return 0.0;
  if (e == 0xffu) return (double)f;  // inf / NaN pass through
  const uint64_t d = ((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                     ((uint64_t)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

__device__ __forceinline__ double to_double(dfloat x) { return f2d_exact(x.hi) + f2d_exact(x.lo); }

// FP64 -> FP32 rounded to nearest (ties to even) on the integer pipes: for results in the
// normal FP32 range the same bits as the hardware conversion, which takes everything else
// (zero, magnitudes below the smallest normal float, inf, NaN).
__device__ __forceinline__ float d2f_rn(double v) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  if (e < 897u || e > 1150u) return __double2float_rn(v);
  uint64_t m = b & 0x7fffffffffffffffull;   // exponent and significand
  m += 0x0fffffffull + ((m >> 29) & 1ull);  // round half to even at bit 29 (a carry may reach inf)
  const uint32_t r = (uint32_t)((m >> 29) - (896ull << 23));
  return __uint_as_float(r | ((uint32_t)(b >> 32) & 0x80000000u));
}

// The nonlinear kernels read u either as FP64 or as its split copy (SplitVec: hi and lo
// arrays written by split_df) and compute in T.
template <typename T>
__device__ __forceinline__ T get(const double* __restrict__ u, size_t k) {
  return (T)u[k];
}
template <typename T>
__device__ __forceinline__ T get(const SplitVec& u, size_t k) {
  return dfloat(u.hi[k], u.lo[k]);
}

// A density-stencil entry: FP64, or (mixed-precision modes) its double-float split stored in
// the same 8 bytes as (hi, lo), so the coarsening chain stays in double-float arithmetic.
__device__ __forceinline__ void put_entry(double* p, size_t k, double v) { p[k] = v; }
__device__ __forceinline__ void put_entry(double* p, size_t k, dfloat v) {
  reinterpret_cast<float2*>(p)[k] = make_float2(v.hi, v.lo);
}
template <typename T>
__device__ __forceinline__ T get_entry(const double* __restrict__ p, size_t k) {
  return p[k];
}
template <>
__device__ __forceinline__ dfloat get_entry<dfloat>(const double* __restrict__ p, size_t k) {
  const float2 v = reinterpret_cast<const float2*>(p)[k];
  return dfloat(v.x, v.y);
}
// an entry as FP64 whichever way it is stored
__device__ __forceinline__ double entry_fp64(const double* __restrict__ p, size_t k, bool split) {
  return split ? to_double(get_entry<dfloat>(p, k)) : p[k];
}

// result of a T computation as FP64
__device__ __forceinline__ double out_of(double v) { return v; }
__device__ __forceinline__ double out_of(float v) { return (double)v; }
__device__ __forceinline__ double out_of(dfloat v) { return to_double(v); }

}  // namespace fmg

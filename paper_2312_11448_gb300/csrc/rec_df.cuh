// Double-float arithmetic: a value carried as the unevaluated sum hi + lo of
// two binary32 numbers (about 48 significant bits), built from error-free
// transformations: Knuth's TwoSum, the fast TwoSum of Dekker (1971) for
// |a| >= |b|, and the TwoProduct from one fused multiply-add (Ogita, Rump &
// Oishi, SIAM J. Sci. Comput. 26, 1955 (2005)).  On GB300 the binary64 pipe
// issues about 1/58 of the binary32 rate, so a residual that needs more than
// binary32 but is evaluated once per cell per pass costs far less this way.
// The __fadd_rn / __fmul_rn intrinsics keep the compiler from fusing the
// transforms' operations into multiply-adds (which would break exactness).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rec {

struct dfloat {
  float hi, lo;
};

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fadd_rn(s, -a);
  const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
  return {s, e};
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fadd_rn(b, -__fadd_rn(s, -a))};
}

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  const dfloat s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfloat df_neg(dfloat a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ dfloat df_mul_f(dfloat a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
  return df_fast_two_sum(p, e);
}

// Split a binary64 value into hi + lo with integer operations only (no
// binary64 arithmetic or conversion, which issue on the slow binary64 pipe):
// hi takes the sign, the exponent and the leading 24 significand bits, lo the
// remaining 29 bits (rounded to 24).  Exact to 2^-48 relative for
// 2^-74 <= |x| < 2^127.  Below that range the result is 0 (ionisation
// fractions never get there); above it, infinities and NaN give a NaN.
__device__ __forceinline__ dfloat df_from_double(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const uint32_t ec = e < 949u ? 949u : (e > 1150u ? 1150u : e);
  float hi = __uint_as_float(sign | ((ec - 896u) << 23) | ((uint32_t)(b >> 29) & 0x7fffffu));
  const float scale = __uint_as_float((ec - 948u) << 23);  // 2^(e - 1075)
  float lo = __fmul_rn(__uint2float_rn((uint32_t)b & 0x1fffffffu), scale);
  lo = sign ? -lo : lo;
  if (e < 949u) { hi = 0.0f; lo = 0.0f; }
  if (e > 1150u) { hi = __uint_as_float(0x7fc00000u); lo = 0.0f; }
  return {hi, lo};
}

// A binary32 value as binary64, exactly, with integer operations only (zero
// and subnormal inputs give zero; infinities and NaN keep their class).
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint64_t mant = (uint64_t)(u & 0x7fffffu) << 29;
  const uint64_t ed = e == 0xffu ? 0x7ffull : (uint64_t)(e + 896u);
  const uint64_t bits = e == 0u ? sign : (sign | (ed << 52) | mant);
  return __longlong_as_double((long long)bits);
}

// x + d as a binary64 value for the increment d of a backward-Euler state,
// with integer operations in the common case |d| < x/4: d is aligned to x's
// last place 2^(ex - 1075) and added to x's significand, carrying or borrowing
// at most one binade.  The result is x + d rounded to 53 bits (the bits of d
// beyond x's last place rounded to nearest, ties away).  Larger increments,
// special values and x outside the normal range take one binary64 addition,
// which on this chip issues on the slow binary64 pipe.
// The rare case of add_small, kept out of line so that the compiler branches to
// it instead of predicating a binary64 addition for every cell.
static __device__ __noinline__ double add_wide(double x, float d) { return x + f2d_bits(d); }

__device__ __forceinline__ double add_small(double x, float d) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t ud = __float_as_uint(d);
  const uint32_t ed = (ud >> 23) & 0xffu;
  const int ex = (int)((b >> 52) & 0x7ffu);
  // d's significand sd = 1.m (24 bits) at 2^(ed - 150); right shift into x's last place
  const int sh = (ex - 1075) - ((int)ed - 150);
  if ((ed != 0u && sh < -26) || ed == 0xffu || ex == 0 || ex >= 0x7fe) return add_wide(x, d);
  const uint64_t sd = (uint64_t)((ud & 0x7fffffu) | 0x800000u);
  uint64_t add;
  if (ed == 0u || sh >= 25) {
    add = 0;  // zero, subnormal or below half a last place of x
  } else if (sh > 0) {
    add = (sd >> sh) + ((sd >> (sh - 1)) & 1u);
  } else {
    add = sd << (-sh);  // d within 2^29 of x's last place: exact
  }
  // x's significand with the implicit bit, signed addition of d
  int64_t S = (int64_t)((b & 0xfffffffffffffull) | 0x10000000000000ull);
  S = (ud & 0x80000000u) ? S - (int64_t)add : S + (int64_t)add;
  int e = ex;
  if (S >= (int64_t)0x20000000000000ll) {  // carried into the next binade: round the dropped bit
    S = (S >> 1) + (S & 1);
    ++e;
  } else if (S < (int64_t)0x10000000000000ll) {  // borrowed from the binade below (one bit suffices)
    S <<= 1;
    --e;
  }
  const uint64_t out = (b & 0x8000000000000000ull) | ((uint64_t)e << 52) | ((uint64_t)S & 0xfffffffffffffull);
  return __longlong_as_double((long long)out);
}

// hi + lo rounded to one binary32 value
__device__ __forceinline__ float df_to_float(dfloat a) { return __fadd_rn(a.hi, a.lo); }

}  // namespace rec

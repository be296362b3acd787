// Double-float arithmetic (an unevaluated sum hi + lo of two FP32 numbers,
// about 48 significant bits) for the refinement residual.  GB300 issues FP64
// at about 2 operations per clock per SM and FP32 at 128, so the residual is
// evaluated with the error-free transformations of Knuth (two-sum) and Dekker
// (fast two-sum, FMA-based two-product), and FP64 <-> (hi, lo) conversions are
// done with integer bit operations instead of FP64-pipe conversions.
#pragma once
#include <cstdint>

namespace fdi {
namespace df {

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 make(float h, float l) { return F2{h, l}; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ F2 two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return F2{s, e};
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
  float s = a + b;
  return F2{s, b - (s - a)};
}

__device__ __forceinline__ F2 add(F2 a, F2 b) {
  F2 s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ F2 neg(F2 a) { return F2{-a.hi, -a.lo}; }

__device__ __forceinline__ F2 sub(F2 a, F2 b) { return add(a, neg(b)); }

__device__ __forceinline__ F2 mul(F2 a, F2 b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// exact FP32 value -> FP64 bits, integer operations only (normal numbers and zero)
__device__ __forceinline__ double f2d(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u) {
    if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((uint64_t)(b & 0x80000000u) << 32));
    return (double)f;  // subnormal: rare
  }
  if (e == 255u) return (double)f;
  const uint64_t d = ((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(e - 127u + 1023u) << 52) |
                     ((uint64_t)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// The same conversion for code that a whole warp executes together (every
// lane must call it): no per-lane branch for normal numbers and zero, whose 31
// exponent-and-significand bits are rebased from bias 127 to 1023 by one
// 64-bit add and shifted into place; a warp holding a subnormal, infinite or
// NaN value takes the FP64-pipe conversion on every lane.
__device__ __forceinline__ double f2d_warp(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t mag = b & 0x7fffffffu;
  const uint32_t e = mag >> 23;
  if (__any_sync(0xffffffffu, (e == 0u && mag != 0u) || e == 255u)) return (double)f;
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  const uint64_t d = (((uint64_t)mag + (896ull << 23)) << 29) | sign;
  return __longlong_as_double((long long)(mag == 0u ? sign : d));
}

// hi + lo as the nearest FP64 (one FP64 add)
__device__ __forceinline__ double to_f64(F2 a) { return f2d(a.hi) + f2d(a.lo); }

// hi + lo as FP64 with integer operations only, for a normalised pair
// (|lo| <= ulp(hi)) with hi normal: the significands are aligned at a common
// binary point and added as 64-bit integers; bits of lo below the FP64
// significand are truncated (error below one FP64 ulp).  Other inputs take the
// FP64 addition.
__device__ __forceinline__ double to_f64_bits(F2 a) {
  const uint32_t bh = __float_as_uint(a.hi), bl = __float_as_uint(a.lo);
  const int eh = (int)((bh >> 23) & 0xffu), el = (int)((bl >> 23) & 0xffu);
  if (eh == 0 || eh == 255 || el == 0 || el == 255 || el > eh - 23) {
    if ((bl & 0x7fffffffu) == 0u && eh != 0 && eh != 255) {
      // lo = 0: exact widening of hi
      return __longlong_as_double((long long)(((uint64_t)(bh & 0x80000000u) << 32) |
                                              ((uint64_t)(eh - 127 + 1023) << 52) |
                                              ((uint64_t)(bh & 0x7fffffu) << 29)));
    }
    return to_f64(a);
  }
  // hi significand with its leading bit at 2^52
  long long T = (long long)((bh & 0x7fffffu) | 0x800000u) << 29;
  const unsigned long long ml = (unsigned long long)((bl & 0x7fffffu) | 0x800000u);
  const int shl = el - eh + 29;  // <= 6
  long long L = shl >= 0 ? (long long)(ml << shl) : (shl > -40 ? (long long)(ml >> (-shl)) : 0ll);
  if ((bh ^ bl) & 0x80000000u) L = -L;
  T += L;
  int e = eh;
  if (T >= (1ll << 53)) {
    T >>= 1;
    e += 1;
  } else if (T < (1ll << 52)) {
    T <<= 1;
    e -= 1;
  }
  return __longlong_as_double((long long)(((uint64_t)(bh & 0x80000000u) << 32) | ((uint64_t)(e - 127 + 1023) << 52) |
                                          ((uint64_t)T & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ float pow2f(int e) {
  // 2^e for -126 <= e <= 127
  return __uint_as_float((uint32_t)(e + 127) << 23);
}

// FP64 -> (hi, lo) with integer operations: hi keeps the leading 24 bits of the
// significand (truncated), lo the next bits rounded to 24; |error| <= 2^-48 |v|.
__device__ __forceinline__ F2 from_f64(double v) {
  const uint64_t u = (uint64_t)__double_as_longlong(v);
  const int e = (int)((u >> 52) & 0x7ff);
  if (e < 921 || e > 1150) {
    // zero, tiny or huge: outside the range handled by bit manipulation
    if ((u & 0x7fffffffffffffffull) == 0ull) return F2{__uint_as_float((uint32_t)(u >> 32)), 0.f};
    float h = __double2float_rn(v);
    float l = __double2float_rn(v - (double)h);
    return F2{h, l};
  }
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const uint64_t mant = u & 0xFFFFFFFFFFFFFull;
  const float h = __uint_as_float(sign | ((uint32_t)(e - 1023 + 127) << 23) | (uint32_t)(mant >> 29));
  const uint32_t rem = (uint32_t)(mant & 0x1FFFFFFFull);
  float l = (float)rem;                       // <= 29-bit integer, rounded to 24 bits
  const int sc = e - 1075;                    // weight of the lowest significand bit
  const int s1 = sc / 2, s2 = sc - s1;
  l = l * pow2f(s1) * pow2f(s2);
  return F2{h, sign ? -l : l};
}

}  // namespace df
}  // namespace fdi

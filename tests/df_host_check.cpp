// Host build of the double-float helpers (paper_1107_2461_gb300/csrc/df.cuh)
// checked against IEEE FP64 arithmetic: the device intrinsics they use are
// given their plain host meanings below (one lane per "warp").  Prints "ok"
// and exits 0 when every check holds.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#define __device__
#define __forceinline__ inline

static inline uint32_t __float_as_uint(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
static inline float __uint_as_float(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
static inline long long __double_as_longlong(double d) {
  long long v;
  std::memcpy(&v, &d, 8);
  return v;
}
static inline double __longlong_as_double(long long v) {
  double d;
  std::memcpy(&d, &v, 8);
  return d;
}
static inline float __double2float_rn(double d) { return (float)d; }
static inline bool __any_sync(unsigned, bool p) { return p; }

#include "df.cuh"

static long long g_fail = 0;

static uint64_t bits(double d) { return (uint64_t)__double_as_longlong(d); }

int main() {
  std::mt19937_64 rng(12345);
  auto rnd_float = [&](int emin, int emax) {
    const uint32_t e = (uint32_t)(emin + (int)(rng() % (uint64_t)(emax - emin + 1)));
    const uint32_t m = (uint32_t)(rng() & 0x7fffffu), s = (uint32_t)(rng() & 1u) << 31;
    return __uint_as_float(s | (e << 23) | m);
  };
  // f2d: exact widening of normal numbers and zero
  for (int t = 0; t < 1000000; ++t) {
    const float a = rnd_float(1, 254);
    if (bits(fdi::df::f2d(a)) != bits((double)a)) ++g_fail;
    if (bits(fdi::df::f2d_warp(a)) != bits((double)a)) ++g_fail;
  }
  if (bits(fdi::df::f2d(-0.f)) != bits(-0.0) || bits(fdi::df::f2d_warp(0.f)) != bits(0.0)) ++g_fail;
  // two_sum and fast_two_sum are error free: s + e equals a + b exactly
  for (int t = 0; t < 1000000; ++t) {
    const float a = rnd_float(60, 190), b = rnd_float(60, 190);
    const fdi::df::F2 s2 = fdi::df::two_sum(a, b);
    if ((double)s2.hi + (double)s2.lo != (double)a + (double)b || s2.hi != a + b) ++g_fail;
    const float x = std::fabs(a) >= std::fabs(b) ? a : b, y = std::fabs(a) >= std::fabs(b) ? b : a;
    const fdi::df::F2 f2 = fdi::df::fast_two_sum(x, y);
    if ((double)f2.hi + (double)f2.lo != (double)x + (double)y) ++g_fail;
  }
  // from_f64: hi + lo within 2^-48 |v|; to_f64_bits of that pair back within
  // one FP64 ulp
  for (int t = 0; t < 1000000; ++t) {
    const double v = std::ldexp((double)(rng() >> 11) / 9007199254740992.0 + 0.5, (int)(rng() % 200) - 100) *
                     ((rng() & 1) ? -1.0 : 1.0);
    const fdi::df::F2 p = fdi::df::from_f64(v);
    const double back = (double)p.hi + (double)p.lo;
    if (std::fabs(back - v) > std::ldexp(std::fabs(v), -48)) ++g_fail;
    const double b2 = fdi::df::to_f64_bits(p);
    if (std::fabs(b2 - back) > std::ldexp(std::fabs(back), -52)) ++g_fail;
  }
  if (g_fail) {
    std::printf("%lld failures\n", g_fail);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}

// Exact fixed-point accumulation of float32 values, for sums that must keep float64 rounding
// (the charge-neutrality sums of the projection, Eq. 9) without float64 adds: a two's-complement
// 128-bit integer in units of 2^-FX_F.  A float enters exactly (its 24-bit mantissa shifted into
// place; only parts below 2^-FX_F, about 3e-27, are dropped), so a sum of any number of floats is
// exact while |sum| < 2^(127 - FX_F), about 5e11 (a single value of magnitude 2^39 or more, and
// zero, subnormal or non-finite values, add nothing); value() converts to float64 within two units
// in the last place.  Integer adds keep such sums off GB300's narrow float64 pipe.
//
// Host and device code: the same functions compile with a host compiler, so that the host test
// suite can check them against exact rational sums.
#pragma once

#include <cstring>

#ifdef __CUDACC__
#define CPM_FX_HD __host__ __device__ __forceinline__
#else
#define CPM_FX_HD inline
#endif

namespace cpm {

constexpr int FX_F = 88;

CPM_FX_HD unsigned int fx_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned int u;
  std::memcpy(&u, &x, sizeof(u));
  return u;
#endif
}

struct Fx128 {
  unsigned long long lo = 0, hi = 0;
  CPM_FX_HD void add(unsigned long long al, unsigned long long ah) {
    lo += al;
    hi += ah + (lo < al ? 1ull : 0ull);
  }
  // the 128-bit image of x
  CPM_FX_HD static void image(float x, unsigned long long& l, unsigned long long& h) {
    const unsigned int bits = fx_bits(x);
    const int e = (int)((bits >> 23) & 0xffu);
    const unsigned long long m = (bits & 0x7fffffu) | 0x800000u;
    const int sh = e - 150 + FX_F;                      // |x| = m 2^(e - 150) = m units << sh
    l = 0;
    h = 0;
    if (e == 0 || e == 0xff || sh <= -24 || sh > 103) return;
    if (sh >= 64) {
      h = m << (sh - 64);
    } else if (sh > 0) {
      l = m << sh;
      h = m >> (64 - sh);
    } else {
      l = m >> (-sh);
    }
    if (bits >> 31) {                                   // two's complement of the magnitude
      l = ~l + 1ull;
      h = ~h + (l == 0ull ? 1ull : 0ull);
    }
  }
  CPM_FX_HD void add(float x) {
    unsigned long long l, h;
    image(x, l, h);
    add(l, h);
  }
  CPM_FX_HD void add(const Fx128& o) { add(o.lo, o.hi); }
#ifdef __CUDACC__
  __device__ __forceinline__ void shfl_add(int o) {
    const unsigned long long ol = __shfl_xor_sync(0xffffffffu, lo, o), oh = __shfl_xor_sync(0xffffffffu, hi, o);
    add(ol, oh);
  }
#endif
  CPM_FX_HD double value() const {
    const bool neg = (hi >> 63) != 0;
    unsigned long long l = lo, h = hi;
    if (neg) {
      l = ~l + 1ull;
      h = ~h + (l == 0ull ? 1ull : 0ull);
    }
    const double v = (double)h * 0x1p-24 + (double)l * 0x1p-88;   // 2^(64 - FX_F), 2^-FX_F
    return neg ? -v : v;
  }
};
static_assert(FX_F == 88, "value() scales by 2^(64 - FX_F) and 2^-FX_F");

}  // namespace cpm

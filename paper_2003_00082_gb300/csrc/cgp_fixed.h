// Exact fixed-point accumulation of FP64 values on the integer pipe.
//
// On GB300 a warp-wide FP64 instruction occupies the narrow FP64 pipe for
// tens of cycles, so a dependent chain of FP64 adds (a reduction tree) is
// slow.  The reductions of the solver therefore convert each double to a
// signed 128-bit integer aligned to a common exponent and add integers:
//
//   a finite double v = M * 2^(e - 1075), M < 2^53 (e the biased exponent,
//   with the implicit bit; subnormals use e = 1);
//   relative to a reference exponent E >= e its fixed-point image is
//   X = M * 2^(54 - (E - e)), truncated toward zero below 2^0,
//   i.e. X = v * 2^(1129 - E), |X| < 2^107.
//
// Sums of up to 2^20 images fit in 128 bits.  Integer addition is
// associative, so the total does not depend on the order of the terms (the
// result is identical in every block and every run), and the only error is
// the truncation of each term 2^-106 below the largest one: far below FP64
// rounding.  The total is converted back to the nearest double (ties to
// even) with integer operations only.
//
// The functions are __host__ __device__ so the arithmetic can be checked on
// the CPU against exact rational sums.
#pragma once

#include <cstdint>
#include <cstring>

#ifndef __CUDACC__
#define CGP_HD
#else
#define CGP_HD __host__ __device__
#endif

namespace cgp {
namespace fx {

constexpr int kFrac = 54;          // fraction bits below the reference exponent's unit
constexpr int kBadExp = 0x7FFF;    // exponent marker of a non-finite contribution

typedef __int128 I128;
typedef unsigned __int128 U128;

CGP_HD inline uint64_t dbits(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  std::memcpy(&b, &v, 8);
  return b;
#endif
}

CGP_HD inline double from_bits(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  std::memcpy(&v, &b, 8);
  return v;
#endif
}

CGP_HD inline int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// Biased exponent used for alignment: 1 for zero and subnormals, kBadExp for
// Inf and NaN, else the IEEE biased exponent.
CGP_HD inline int exponent_of(double v) {
  const int e = (int)((dbits(v) >> 52) & 0x7FF);
  if (e == 0x7FF) return kBadExp;
  return e == 0 ? 1 : e;
}

// Arithmetic shift right by s >= 0 (rounds toward minus infinity).
CGP_HD inline I128 sar(I128 a, int s) { return a >> (s > 127 ? 127 : s); }

// Fixed-point image of a finite v relative to reference exponent E >= exponent_of(v).
CGP_HD inline I128 image(double v, int E) {
  const uint64_t b = dbits(v);
  const int eb = (int)((b >> 52) & 0x7FF);
  const uint64_t m = b & ((1ull << 52) - 1);
  const uint64_t M = eb == 0 ? m : (m | (1ull << 52));
  const int e = eb == 0 ? 1 : eb;
  const int sh = kFrac - (E - e);   // shift left when >= 0 (at most 54)
  const I128 x = sh >= 0 ? (I128)M << sh : (I128)((-sh) >= 64 ? 0 : (M >> (-sh)));
  return (b >> 63) ? -x : x;
}

// Nearest double (ties to even) of X * 2^(E - 1075 - kFrac).
CGP_HD inline double to_double(I128 X, int E) {
  if (E >= kBadExp) return from_bits(0x7FF8000000000000ull);  // NaN
  const bool negative = X < 0;
  const U128 U = negative ? (U128)(-X) : (U128)X;
  if (U == 0) return 0.0;
  const uint64_t hi = (uint64_t)(U >> 64), lo = (uint64_t)U;
  int lead = hi ? 127 - clz64(hi) : 63 - clz64(lo);  // index of the leading one
  uint64_t mant;
  if (lead <= 52) {
    mant = lo << (52 - lead);
  } else {
    const int s = lead - 52;  // dropped bits, 1..75
    mant = (uint64_t)(U >> s);
    const U128 rem = U & (((U128)1 << s) - 1), half = (U128)1 << (s - 1);
    if (rem > half || (rem == half && (mant & 1u))) {
      ++mant;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        ++lead;
      }
    }
  }
  // value = mant * 2^(lead - 52) * 2^(E - 1129)
  const uint64_t sign = negative ? (1ull << 63) : 0;
  const int biased = lead + E - 106;
  if (biased >= 2047) return from_bits(sign | 0x7FF0000000000000ull);
  if (biased <= 0) {
    // subnormal result: shift the 53-bit mantissa into place, rounding to nearest even
    const int s = 1 - biased;
    uint64_t m2 = 0;
    if (s < 64) {
      m2 = mant >> s;
      const uint64_t rem = mant & ((1ull << s) - 1), half = 1ull << (s - 1);
      if (rem > half || (rem == half && (m2 & 1u))) ++m2;
    }
    return from_bits(sign | m2);
  }
  return from_bits(sign | ((uint64_t)biased << 52) | (mant & ((1ull << 52) - 1)));
}

CGP_HD inline I128 add(I128 a, I128 b) { return a + b; }

// 64-bit images for the tagged reductions of the solver: relative to a
// reference exponent E >= exponent_of(v), a finite v = M 2^(e - 1075) maps to
// X = (M << 4) >> (E - e) = v 2^(1079 - E) truncated toward zero in magnitude,
// |X| < 2^57, so that 32 of them add within 62 bits.
CGP_HD inline int64_t image64(double v, int E) {
  const uint64_t b = dbits(v);
  const int eb = (int)((b >> 52) & 0x7FF);
  const uint64_t M = (b & ((1ull << 52) - 1)) | (eb ? (1ull << 52) : 0ull);
  int sh = E - (eb ? eb : 1);
  if (sh > 63) sh = 63;
  const int64_t X = (int64_t)((M << 4) >> sh);
  return (b >> 63) ? -X : X;
}

// Tagged slot: one block's partial X (exponent E, |X| < 2^117 for a block of
// <= 1024 threads) of reduction `red` in one 128-bit word that says by itself
// whether it holds that reduction:
//   lo = m[0:56) << 8 | tag8,  hi = m[56:80) | E << 24 | tag24 << 40,
// m = X >> kTagShift (80 signed bits).  tag24 = 2^23 | (red mod 2^23) is
// never 0 (a zeroed slot) nor all ones; tag8 repeats red in the low word, so
// a word whose halves come from two different stores fails the check.  The
// value of a slot is m * 2^(kTagShift + E - 1075 - kFrac).
constexpr int kTagShift = 38;
CGP_HD inline uint64_t tag24(int red) { return 0x800000ull | ((unsigned)red & 0x7FFFFFu); }
CGP_HD inline uint64_t tag8(int red) { return ((unsigned)red & 0xFFu) ^ 0xA5u; }

// shift: bits of X dropped before packing (kTagShift for a 128-bit partial;
// 0 for a 64-bit one, whose |X| < 2^62 fits the 80-bit field as it is).
CGP_HD inline void pack_tagged(I128 x, int E, int red, uint64_t& lo, uint64_t& hi, int shift = kTagShift) {
  const I128 m = E < kBadExp ? sar(x, shift) : (I128)0;
  lo = ((uint64_t)m << 8) | tag8(red);
  hi = ((uint64_t)(m >> 56) & 0xFFFFFFull) | ((uint64_t)(E & 0xFFFF) << 24) | (tag24(red) << 40);
}
CGP_HD inline bool tagged_current(uint64_t lo, uint64_t hi, int red) {
  return (hi >> 40) == tag24(red) && (lo & 0xFFull) == tag8(red);
}
CGP_HD inline int tagged_exponent(uint64_t hi) { return (int)((hi >> 24) & 0xFFFFull); }
CGP_HD inline I128 tagged_mantissa(uint64_t lo, uint64_t hi) {
  const int64_t mh = ((int64_t)(hi << 40)) >> 40;  // m[56:80), sign-extended
  return ((I128)mh << 56) | (I128)(lo >> 8);
}

}  // namespace fx
}  // namespace cgp

// int64 fixed-point -> float64 with integer operations only.
//
// The split-precision product ends with one signed 64-bit fixed-point sum per
// output, to be scaled by a power of two.  Converting it with the float64
// unit costs one float64-pipe instruction per output, and the float64 pipe of
// this part issues about one and a half per clock per SM; with integer
// operations (leading-zero count, shifts, one rounding step) the conversion
// runs on the integer pipes instead.  The result is the IEEE round-to-nearest
// (ties to even) value of acc, as a (double) cast gives, with the exponent
// then moved by E.  The body compiles as CUDA device code and as plain C++
// (the host test checks it against the cast).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define QMLGB_HD __host__ __device__ __forceinline__
#else
#define QMLGB_HD inline
#endif

namespace qmlgb {

QMLGB_HD int clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

// Bit pattern of round(acc) 2^E (round to nearest, ties to even), sign
// flipped when neg.  False when the result would not be a normal float64 (the
// caller then scales another way); acc = 0 gives a signed zero.
QMLGB_HD bool fixed_to_double_bits(int64_t acc, int E, bool neg, uint64_t &bits) {
  const uint64_t flip = neg ? 0x8000000000000000ull : 0ull;
  if (acc == 0) {
    bits = flip;
    return true;
  }
  const uint64_t sgn = acc < 0 ? 0x8000000000000000ull : 0ull;
  const uint64_t u = acc < 0 ? (uint64_t)0 - (uint64_t)acc : (uint64_t)acc;
  const int lz = clz64(u);
  const uint64_t m = u << lz;   // leading one at bit 63
  uint64_t mant = m >> 11;      // 53 significant bits
  const uint64_t rem = m & 0x7FFull;
  int e2 = 63 - lz;             // u lies in [2^e2, 2^(e2 + 1))
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {  // rounded up to the next power of two
      mant >>= 1;
      ++e2;
    }
  }
  const int bexp = e2 + 1023 + E;
  if (bexp <= 0 || bexp >= 2047) return false;
  bits = (sgn ^ flip) | ((uint64_t)bexp << 52) | (mant & 0xFFFFFFFFFFFFFull);
  return true;
}

}  // namespace qmlgb

// Conversion of FP64 input values to the storage types, shared by the host analyser and
// the device re-pack kernel so both produce the same bits. Plain arithmetic only.
#ifndef CB_ROUND_H_
#define CB_ROUND_H_
#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define CB_HD __host__ __device__
#else
#define CB_HD
#endif

namespace cb {

// v rounded to the nearest number of a binary floating-point format with p significand
// bits (implicit bit included), smallest normal exponent emin and largest exponent emax;
// ties go to the even significand, magnitudes beyond the largest finite number become
// infinities, below the smallest normal the quantum stays 2^(emin - p + 1) (gradual
// underflow); NaN and signed zeros pass through (IEEE 754 roundTiesToEven). The result
// is exact in double.
CB_HD inline double round_to_format(double v, int p, int emin, int emax) {
  if (!isfinite(v) || v == 0.0) return v;
  int e = ilogb(v);                              // floor(log2 |v|)
  if (e > emax) return copysign(INFINITY, v);
  if (e < emin) e = emin;
  const int q = e - (p - 1);                     // exponent of the quantum
  const double r = nearbyint(ldexp(v, -q));      // the default mode rounds ties to even
  const double out = ldexp(r, q);
  if (ilogb(out) > emax) return copysign(INFINITY, v);
  return out;
}

// IEEE binary16 bits of a double that is exactly representable in binary16 (or +-inf, NaN).
CB_HD inline uint16_t half_bits(double h) {
  const uint16_t sign = signbit(h) ? 0x8000u : 0u;
  if (isnan(h)) return 0x7e00u;
  if (isinf(h)) return sign | 0x7c00u;
  const double a = fabs(h);
  if (a == 0.0) return sign;
  const int e = ilogb(a);
  if (e < -14) return (uint16_t)(sign | (uint16_t)ldexp(a, 24));          // subnormal: a / 2^-24
  const uint32_t mant = (uint32_t)ldexp(a, 10 - e) - 1024u;               // 10 fraction bits
  return (uint16_t)(sign | (uint16_t)((uint32_t)(e + 15) << 10) | (uint16_t)mant);
}

// The stored bits of v in storage type dtype (0 FP64, 1 FP32, 2 BF16, 3 FP16), rounded to
// nearest (ties to even) directly from FP64; returned in the low bytes.
CB_HD inline uint64_t storage_bits(double v, int dtype) {
  if (dtype == 0) {
    uint64_t b;
    memcpy(&b, &v, 8);
    return b;
  }
  if (dtype == 1) {
    const float f = (float)round_to_format(v, 24, -126, 127);
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
  }
  if (dtype == 2) {
    const float f = (float)round_to_format(v, 8, -126, 127);   // exact in binary32
    uint32_t b;
    memcpy(&b, &f, 4);
    return isnan(f) ? 0x7fc0u : (b >> 16);
  }
  return half_bits(round_to_format(v, 11, -14, 15));
}

}  // namespace cb
#endif

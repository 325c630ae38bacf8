// Host-side rounding of filter weights to the tensor cores' operand formats (plan creation).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

namespace rapro {

inline float tf32_round_host(float x) {
  // Round to nearest (ties away) at 10 explicit mantissa bits, as cvt.rna.tf32.f32.
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;
  u = (u + 0x1000u) & 0xffffe000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// Round to nearest even at FP16 (10 explicit mantissa bits, subnormals below 2^-14,
// overflow to infinity).
inline uint16_t f16_round_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  const uint32_t sign = (u >> 16) & 0x8000u, a = u & 0x7fffffffu;
  if (a > 0x7f800000u) return uint16_t(sign | 0x7e00u);               // NaN
  if (a >= 0x47800000u) return uint16_t(sign | 0x7c00u);              // |x| >= 65536: inf
  if (a < 0x38800000u) {                                               // |x| < 2^-14
    float f;
    std::memcpy(&f, &a, 4);
    return uint16_t(sign | uint32_t(std::nearbyint(f * 16777216.0f)));   // units of 2^-24, ties even
  }
  uint32_t h = (a - 0x38000000u) >> 13;                                // rebias 127 -> 15
  const uint32_t rem = a & 0x1fffu;
  if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;              // may carry into the exponent
  return uint16_t(sign | (h >= 0x7c00u ? 0x7c00u : h));
}

inline uint16_t bf16_round_host(float x) {
  // Round to nearest even at 7 explicit mantissa bits (finite inputs).
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  return uint16_t(u >> 16);
}

}  // namespace rapro

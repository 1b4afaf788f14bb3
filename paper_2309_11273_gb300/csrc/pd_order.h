// Break test d >= t (Eq 1.30 in the sqrt-free form xi.du >= s0 |xi|^2) on the bit patterns of two
// doubles, for a positive finite threshold t.
//
// Read as unsigned 64-bit integers, the non-negative doubles are ordered as their values, +inf is
// 0x7ff0000000000000 and every positive NaN lies above it; negative values, -0 and negative NaNs
// have the sign bit set and lie above all of them.  So d >= t holds exactly when the pattern of d
// lies in [pattern(t), pattern(+inf)], which one wrapping subtraction and one unsigned comparison
// decide: a NaN of either sign, like any negative value, does not break the bond, as IEEE
// comparison (and the oracle's s >= s0) has it.  The test runs on the integer pipe.
//
// Host and device share this file so that a host test checks the same code.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define PD_HD __host__ __device__ __forceinline__
#else
#define PD_HD inline
#endif

PD_HD uint64_t pd_double_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, sizeof(u));
  return u;
#endif
}

// d >= t for t > 0 finite; false when d is NaN.
PD_HD bool pd_ge_threshold(double d, double t) {
  const uint64_t db = pd_double_bits(d), tb = pd_double_bits(t);
  return db - tb <= 0x7ff0000000000000ull - tb;
}

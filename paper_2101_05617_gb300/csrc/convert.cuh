// FP64 <-> FP32 conversions of the complex64-bulk form on the integer pipe,
// shared by the tangent kernels (dfr_tangent.cuh, dfr_tile.cu) and the
// orthogonalisation pass that keeps the FP32 copy of the Krylov basis
// (krylov.cu).
#pragma once

#include <cuda_runtime.h>

namespace swepi {

// Conversions between the FP64 Krylov vectors and the FP32 arithmetic of the
// complex64-bulk form are done on the IEEE-754 bit fields with integer
// operations, so that none of them occupies the FP64 pipe (on this GPU a
// fraction of the FP32 rate).  binary64 -> binary32 rounds the significand to
// nearest, ties to even (an unbiased rounding matters: a systematic one, as
// truncation, scales every Krylov matvec the same way, and the stiff
// exponential amplifies that), carries into the exponent as the packed
// integer increments, maps magnitudes below the binary32 normal range to
// signed zero and above it to infinity, and NaN to NaN; binary32 -> binary64
// is exact for normal numbers, zero, infinities and NaN (binary32 subnormals
// become zero).
__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  const unsigned int sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;                  // binary32 biased exponent
  const unsigned int mant = ((hi & 0xfffffu) << 3) | (lo >> 29);   // top 23 significand bits
  unsigned int r = ((unsigned int)e << 23) | mant;
  const unsigned int round = (lo >> 28) & 1u, sticky = (lo & 0x0fffffffu) != 0u;
  r += round & (sticky | (r & 1u));                                // nearest, ties to even
  r |= sign;
  r = (e <= 0) ? sign : r;
  r = (e >= 255 || (r & 0x7f800000u) == 0x7f800000u) ? (sign | 0x7f800000u) : r;
  const bool nan = ((hi & 0x7ff00000u) == 0x7ff00000u) && (((hi & 0xfffffu) | lo) != 0u);
  return __uint_as_float(nan ? 0x7fc00000u : r);
}
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned int hi = sign | ((e + 896u) << 20) | (m >> 3);
  unsigned int lo = m << 29;
  hi = (e == 0u) ? sign : hi;
  lo = (e == 0u) ? 0u : lo;
  hi = (e == 255u) ? (sign | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u)) : hi;
  return __hiloint2double((int)hi, (int)lo);
}
template <typename T>
__device__ __forceinline__ T from_f64(double x) {
  if constexpr (sizeof(T) == 4) return f64_to_f32_bits(x);
  else return x;
}
template <typename T>
__device__ __forceinline__ double to_f64(T x) {
  if constexpr (sizeof(T) == 4) return f32_to_f64_bits(x);
  else return x;
}

}  // namespace swepi

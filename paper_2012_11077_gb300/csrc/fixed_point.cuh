// Conversions between FP32 and the 64-bit fixed-point values of the
// summed-area tables.
//
// The hardware float <-> 64-bit integer conversions execute on the FP64
// pipe, which on this GPU retires about 0.6 T conversions/s for the whole
// chip: they were the bottleneck of every table and CFAR kernel. These
// routines use only 32-bit conversions (about 4 T/s, on the XU and ALU
// pipes) and FP32 arithmetic:
//   q_from_f32: round-to-nearest-even of v * 2^s through a magic-number
//               rounding of the part above 2^31 (one FMA) and a 32-bit
//               conversion of the exact remainder;
//   f32_from_q: the integer split into a signed high and low 32-bit word,
//               each converted, recombined with one FMA.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rcfar {

// round(v * scale) to nearest, ties to even, as a 64-bit integer; scale is a
// power of two and |v * scale| < 2^52 (the table scale guarantees this for
// every in-range value). Equals __float2ll_rn(v * scale).
__device__ __forceinline__ long long q_from_f32(float v, float scale) {
  const float x = v * scale;  // exact: scaling by a power of two
  // 1.5 * 2^23 + RNE(x / 2^31): the sum's unit in the last place is 1, so the
  // add rounds x / 2^31 to an integer (|x / 2^31| < 2^21)
  const float t = fmaf(x, 4.656612873077392578125e-10f, 12582912.0f);
  const int h = __float_as_int(t) - 0x4B400000;
  // x - h * 2^31: exact (|.| <= 2^30, representable in 24 bits)
  const float rem = fmaf(t - 12582912.0f, -2147483648.0f, x);
  return (long long)h * 2147483648LL + (long long)__float2int_rn(rem);
}

// The same rounding for |v * scale| < 2^62 (sums of many cells): the part
// above 2^42 is split off first, exactly, the same way.
__device__ __forceinline__ long long q_from_f32_wide(float v, float scale) {
  const float x = v * scale;
  const float t = fmaf(x, 2.2737367544323206e-13f, 12582912.0f);  // 1.5 * 2^23 + RNE(x / 2^42)
  const int a = __float_as_int(t) - 0x4B400000;
  const float r = fmaf(t - 12582912.0f, -4398046511104.0f, x);   // x - a * 2^42, exact, |.| <= 2^41
  return (long long)a * 4398046511104LL + q_from_f32(r, 1.0f);
}

// FP32 value of a 64-bit integer, within one unit in the last place: x =
// hi * 2^32 + lo with lo the signed low word (|lo| <= 2^31), so the two
// terms never cancel beyond |x| >= 2^31 >= |lo|.
__device__ __forceinline__ float f32_from_q(long long x) {
  const unsigned long long u = (unsigned long long)x;
  const int lo = (int)(unsigned)u;
  const int hi = (int)(unsigned)(u >> 32) + (int)((unsigned)lo >> 31);
  return fmaf(__int2float_rn(hi), 4294967296.0f, __int2float_rn(lo));
}

}  // namespace rcfar

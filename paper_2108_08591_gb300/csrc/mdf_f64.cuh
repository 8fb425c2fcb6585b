// Exact FP32 -> FP64 widening built from the IEEE-754 binary32 / binary64
// bit layouts on the integer pipe.  Every binary32 value (zero, subnormal,
// normal, infinity, NaN with its payload) has an exact binary64 image:
// sign kept, exponent re-biased (+1023 - 127), fraction shifted left by 29;
// subnormals are normalised first.  Used where fields leave the kernels as
// FP64: a native FP32 -> FP64 conversion runs on the FP64 pipe, which on
// this GPU processes a few lanes per clock per SM.
#pragma once

namespace mdf {

__device__ __forceinline__ double widen_f32(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xffu;
  unsigned m = b & 0x7fffffu;
  unsigned be;  // biased binary64 exponent
  if (e == 0xffu) {
    be = 0x7ffu;
  } else if (e != 0u) {
    be = e + 896u;
  } else if (m == 0u) {
    be = 0u;
  } else {  // subnormal: m * 2^-149 with the leading one at bit 31 - clz(m)
    const int sh = __clz((int)m) - 8;
    m = (m << sh) & 0x7fffffu;
    be = 897u - (unsigned)sh;
  }
  return __hiloint2double((int)(sign | (be << 20) | (m >> 3)), (int)(m << 29));
}
__device__ __forceinline__ double widen_f32(double d) { return d; }

}  // namespace mdf

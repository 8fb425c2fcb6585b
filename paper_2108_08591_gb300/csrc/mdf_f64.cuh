// FP32 <-> FP64 conversions built from the IEEE-754 binary32 / binary64 bit
// layouts on the integer pipe.  A native conversion runs on the FP64 pipe,
// which on this GPU processes a few lanes per clock per SM; these are used
// where fields leave the kernels as FP64 and where FP64 inputs enter them.
//
// Widening is exact for every binary32 value (zero, subnormal, normal,
// infinity, NaN with its payload): sign kept, exponent re-biased
// (+1023 - 127), fraction shifted left by 29; subnormals are normalised
// first.
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

// FP64 -> FP32 with round-to-nearest-even on the integer pipe wherever the
// result is a normal float (or zero); other inputs (float subnormals, values
// rounding to infinity, infinities, NaN) take the native conversion.  The
// 29 dropped fraction bits round through the carry of
// magnitude + (2^28 - 1) + (lowest kept bit), which also carries into the
// exponent; the exponent is then re-biased (-1023 + 127).
__device__ __forceinline__ float narrow_f64(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned long long mag = b & 0x7fffffffffffffffull;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  if (mag == 0ull) return __uint_as_float(sign);
  // [2^-126, largest float]: the rounded result is a normal float
  if (mag >= 0x3810000000000000ull && mag <= 0x47efffffe0000000ull) {
    const unsigned long long r = mag + 0x0fffffffull + ((mag >> 29) & 1ull);
    return __uint_as_float(((unsigned)(r >> 29) - (896u << 23)) | sign);
  }
  return __double2float_rn(d);
}

template <class T> __device__ __forceinline__ T narrow_to(double d);
template <> __device__ __forceinline__ float narrow_to<float>(double d) { return narrow_f64(d); }
template <> __device__ __forceinline__ double narrow_to<double>(double d) { return d; }

}  // namespace mdf

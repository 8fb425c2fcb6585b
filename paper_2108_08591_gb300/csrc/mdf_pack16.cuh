// Packed 16-bit population loads shared by the 16-bit update kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace mdf {

// VX consecutive 16-bit values in one load (2, 4, 8 or 16 bytes), with the
// element bits, the pairs as FP32 lanes and the words the x-neighbours need.
template <class TS> __device__ __forceinline__ float bits_to_float(unsigned b);
template <> __device__ __forceinline__ float bits_to_float<__half>(unsigned b) {
  return __half2float(__ushort_as_half((unsigned short)b));
}
template <> __device__ __forceinline__ float bits_to_float<__nv_bfloat16>(unsigned b) {
  return __uint_as_float(b << 16);
}
template <class TS> __device__ __forceinline__ unsigned ldg_bits16(const TS *p) {
  return __ldg(reinterpret_cast<const unsigned short *>(p));
}
template <class TS> __device__ __forceinline__ float2 word_to_f2(unsigned w);
template <> __device__ __forceinline__ float2 word_to_f2<__half>(unsigned w) {
  return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
template <> __device__ __forceinline__ float2 word_to_f2<__nv_bfloat16>(unsigned w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <class TS, int VX> struct Packed16;
template <class TS> struct Packed16<TS, 1> {
  using W = unsigned short;
  static __device__ __forceinline__ W load(const TS *p) { return __ldg(reinterpret_cast<const W *>(p)); }
  static __device__ __forceinline__ unsigned bits(W w, int) { return w; }
  static __device__ __forceinline__ unsigned last_word(W w) { return w; }
  static __device__ __forceinline__ unsigned first_word(W w) { return w; }
  static __device__ __forceinline__ float lanes(W w, int) { return bits_to_float<TS>(w); }
};
template <class TS> struct Packed16<TS, 2> {
  using W = unsigned;
  static __device__ __forceinline__ W load(const TS *p) { return __ldg(reinterpret_cast<const W *>(p)); }
  static __device__ __forceinline__ unsigned bits(W w, int j) { return j ? w >> 16 : w & 0xffffu; }
  static __device__ __forceinline__ unsigned last_word(W w) { return w; }
  static __device__ __forceinline__ unsigned first_word(W w) { return w; }
  static __device__ __forceinline__ float2 lanes(W w, int) { return word_to_f2<TS>(w); }
};
template <class TS> struct Packed16<TS, 4> {
  using W = uint2;
  static __device__ __forceinline__ W load(const TS *p) { return __ldg(reinterpret_cast<const W *>(p)); }
  static __device__ __forceinline__ unsigned bits(W w, int j) {
    const unsigned v = j < 2 ? w.x : w.y;
    return (j & 1) ? v >> 16 : v & 0xffffu;
  }
  static __device__ __forceinline__ unsigned last_word(W w) { return w.y; }
  static __device__ __forceinline__ unsigned first_word(W w) { return w.x; }
  static __device__ __forceinline__ float2 lanes(W w, int q) { return word_to_f2<TS>(q ? w.y : w.x); }
};
template <class TS> struct Packed16<TS, 8> {
  using W = uint4;
  static __device__ __forceinline__ W load(const TS *p) { return __ldg(reinterpret_cast<const W *>(p)); }
  static __device__ __forceinline__ unsigned bits(W w, int j) {
    const unsigned v = j < 2 ? w.x : j < 4 ? w.y : j < 6 ? w.z : w.w;
    return (j & 1) ? v >> 16 : v & 0xffffu;
  }
  static __device__ __forceinline__ unsigned last_word(W w) { return w.w; }
  static __device__ __forceinline__ unsigned first_word(W w) { return w.x; }
  static __device__ __forceinline__ float2 lanes(W w, int q) {
    return word_to_f2<TS>(q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w);
  }
};

}  // namespace mdf

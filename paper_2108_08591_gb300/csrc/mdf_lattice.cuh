// Lattice traits, storage codecs and the per-node MRT collision of the
// MDF-LBM (Chai, Shi & Zhan, arXiv 2108.08591) for the GPU kernels.
//
// Populations are stored shifted by the rest state f_rest = f^eq(P0=1, u=0):
//   g_{i,a} = f_{i,a} - w_i [delta_{a0} rho0 + c_{i,a} P0 / c_s^2].
// The collision is linear in f once f^eq is fixed, so it acts on g exactly as
// on f with every equilibrium moment shifted the same way (P -> P' = P - P0,
// ubar_0 -> rho' = ubar_0 - rho0).  Lattice units: dx = dt = c = 1.
//
// Rounding.  Each relax() forms the change of every population, delta_i =
// -(M^-1 S (M g - m^eq))_i + w_i F, at the small scale of the
// non-equilibrium part and adds it to g_i once, so a post-collision value
// carries one rounding at the scale of g (~U).  With FP32 storage that one
// rounding, repeated on a nearly steady field every step, is the same
// rounding at every step: its errors add up coherently into the slow,
// large-scale modes (the pressure fluctuation P' ~ U^2 first).  The FP32
// kernels therefore round that add stochastically: a uniform offset in
// (-1/2, 1/2) ulp of g_i, drawn from a counter-based hash of (node, time
// step, set, direction), goes into delta_i before the add, which makes the
// expected stored value the exact one (dithered rounding).  The draw depends
// only on the node's global index and the step, so every kernel (vector,
// scalar, in-place, batched, slab) stores the same bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace mdf {

// ---------------------------------------------------------------------------
// Storage codecs: populations are held as T in HBM and computed in TC.
// ---------------------------------------------------------------------------
template <class T> struct Codec;
template <> struct Codec<float> {
  static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
  static __device__ __forceinline__ void store(float *p, float v) { __stcs(p, v); }
  static __device__ __forceinline__ float enc(double v) { return (float)v; }
};
template <> struct Codec<double> {
  static __device__ __forceinline__ double load(const double *p) { return __ldg(p); }
  static __device__ __forceinline__ void store(double *p, double v) { __stcs(p, v); }
  static __device__ __forceinline__ double enc(double v) { return v; }
};
template <> struct Codec<__half> {
  static __device__ __forceinline__ float load(const __half *p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void store(__half *p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ __half enc(double v) { return __float2half_rn((float)v); }
};
template <> struct Codec<__nv_bfloat16> {
  static __device__ __forceinline__ float load(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ void store(__nv_bfloat16 *p, float v) {
    *p = __float2bfloat16_rn(v);
  }
  static __device__ __forceinline__ __nv_bfloat16 enc(double v) {
    return __float2bfloat16_rn((float)v);
  }
};

// ---------------------------------------------------------------------------
// Dithered rounding of the FP32 populations (see the header comment).
// ---------------------------------------------------------------------------
// 32-bit integer mixer: xor-shift / odd-multiply rounds with the constants of
// the "lowbias32" mixer from C. Wellons' public hash-prospector search.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
// Random word of node n (global index; its low 32 bits) at time step t.
__device__ __forceinline__ uint32_t step_key(int t) { return mix32((uint32_t)t * 0x9e3779b9u + 0x632be5abu); }
__device__ __forceinline__ uint32_t node_key(long long n, int t) { return mix32((uint32_t)n ^ step_key(t)); }
// Random words of one node for its draws: word 0 is the node key, word k
// its product with a distinct odd constant (a bijection, so every byte of a
// word is uniform when the key is).
__device__ __forceinline__ uint32_t rand_word(uint32_t key, int k) {
  return k == 0 ? key : key * (0x9e3779b9u + 2u * (uint32_t)k);
}
// Byte j (0..3) of a random word as the FP32 number 2^-23 (1 + b/256), made
// by placing the byte in mantissa bits 15..22 under the exponent of 2^-23.
__device__ __forceinline__ float rand_scale(uint32_t w, int j) {
  const int sh = 8 * j - 15;
  const uint32_t m = (sh >= 0 ? w >> sh : w << -sh) & 0x7f8000u;
  return __uint_as_float(m | (104u << 23));
}
// The change dl of a population v with its dither: dl + (b - 127.5)/256
// ulp(v), where ulp(v) = 2^(E - 23) for v in [2^E, 2^(E+1)): 2^E is v's
// exponent bits alone (0 for v = 0 or subnormal), and r = rand_scale(...).
// Uniform in (-1/2, 1/2) ulp with 8-bit resolution (residual bias below
// ulp/512); the two FMAs round at the scale of dl.
__device__ __forceinline__ float dithered_change(float dl, float v, float r) {
  const float p2 = __int_as_float(__float_as_int(v) & 0x7f800000);
  return __fmaf_rn(r, p2, __fmaf_rn(-1.498046875f * 0x1p-23f, p2, dl));
}

// g <- g + dl: the change of a population added once, dithered for FP32
// storage (DZ) with the random scale rz[i].
template <bool DZ, class TC>
__device__ __forceinline__ void add_change(TC &g, TC dl, const float *rz, int i) {
  if constexpr (DZ) g = g + dithered_change(dl, g, rz[i]);
  else g = g + dl;
}
// Round-to-nearest storage (16-bit rest-shifted, FP64): the change of each
// population is added term by term, g - h1 - ... + w F, in the order that
// keeps fewest values live; the stored rounding dominates there.

// ---------------------------------------------------------------------------
// D2Q5 (Sec. 2.2): c_0..c_4 = (0,0),(1,0),(0,1),(-1,0),(0,-1);
// w_0 = 1/3, w_1..4 = 1/6; c_s^2 = 1/3.  MRT basis of Eq. 4-2 (c = 1):
//   m0 = sum g, m1 = g1 - g3, m2 = g2 - g4, m3 = g1 - g2 + g3 - g4,
//   m4 = -4 g0 + g1 + g2 + g3 + g4;  S_d = diag(s0, s1, s1, s2, s2) (Eq. 4-3).
// Rows of M are orthogonal with squared norms (5, 2, 2, 4, 20), so
// M^-1 = M^T diag(1/5, 1/2, 1/2, 1/4, 1/20).
// Equilibrium moments (Eq. 2-4 with Eq. 3-7a): m3eq = 0, m4eq = -(2/3) m0.
// ---------------------------------------------------------------------------
struct D2Q5 {
  static constexpr int D = 2, Q = 5;
  static constexpr int REST = 0;  // index of the rest direction
  static constexpr double CS2 = 1.0 / 3.0;
  __host__ __device__ static constexpr int c(int i, int b) {
    return b == 0 ? (i == 1 ? 1 : i == 3 ? -1 : 0) : b == 1 ? (i == 2 ? 1 : i == 4 ? -1 : 0) : 0;
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : i == 1 ? 3 : i == 2 ? 4 : i == 3 ? 1 : 2;
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
  // direction that points through the + face of the last axis (the lid)
  static constexpr int UP = 2;

  // In-place MRT relaxation of one set: g <- g - M^-1 S (M g - m^eq) + w F.
  // jeq[b]: equilibrium first moment (shifted); F: source Fbar_alpha; rz:
  // random scales (rand_scale) dithering each change before it meets g (DZ,
  // FP32 only).
  template <bool DZ = false, class TC>
  static __device__ __forceinline__ void relax(TC g[Q], const TC jeq[D], TC s1, TC s2, TC F,
                                               const float *rz = nullptr) {
    const TC m0 = g[0] + g[1] + g[2] + g[3] + g[4];
    const TC d1 = s1 * ((g[1] - g[3]) - jeq[0]);
    const TC d2 = s1 * ((g[2] - g[4]) - jeq[1]);
    const TC d3 = s2 * ((g[1] + g[3]) - (g[2] + g[4]));
    const TC d4 = s2 * ((g[1] + g[2] + g[3] + g[4]) - TC(4) * g[0] + TC(2.0 / 3.0) * m0);
    const TC h1 = TC(0.5) * d1, h2 = TC(0.5) * d2, q3 = TC(0.25) * d3, e4 = TC(0.05) * d4;
    const TC Fw = F * TC(1.0 / 6.0);
    if constexpr (DZ) {
      add_change<DZ>(g[0], TC(0.2) * d4 + F * TC(1.0 / 3.0), rz, 0);
      add_change<DZ>(g[1], ((Fw - h1) - q3) - e4, rz, 1);
      add_change<DZ>(g[2], ((Fw - h2) + q3) - e4, rz, 2);
      add_change<DZ>(g[3], ((Fw + h1) - q3) - e4, rz, 3);
      add_change<DZ>(g[4], ((Fw + h2) + q3) - e4, rz, 4);
    } else {
      g[0] = g[0] + TC(0.2) * d4 + F * TC(1.0 / 3.0);
      g[1] = g[1] - h1 - q3 - e4 + Fw;
      g[2] = g[2] - h2 + q3 - e4 + Fw;
      g[3] = g[3] + h1 - q3 - e4 + Fw;
      g[4] = g[4] + h2 + q3 - e4 + Fw;
    }
  }
};

// ---------------------------------------------------------------------------
// D3Q7 (Sec. 2.2): c_0 = 0, c_1,2 = +-x, c_3,4 = +-y, c_5,6 = +-z;
// w_0 = 1/4, w_1..6 = 1/8; c_s^2 = 1/4.  The paper prints M for D2Q5 only;
// the analogous orthogonal basis used here is
//   m0 = sum g, m1..3 = first moments, m4 = 7|c|^2 - 6 (-6 g0 + sum_{i>0} g),
//   m5 = 2cx^2 - cy^2 - cz^2, m6 = cy^2 - cz^2;  S_d = diag(s0, s1 x3, s2 x3),
// squared row norms (7, 2, 2, 2, 42, 12, 4); m4eq = -(3/4) m0, m5eq = m6eq = 0.
// ---------------------------------------------------------------------------
struct D3Q7 {
  static constexpr int D = 3, Q = 7;
  static constexpr int REST = 0;
  static constexpr double CS2 = 0.25;
  __host__ __device__ static constexpr int c(int i, int b) {
    return b == 0 ? (i == 1 ? 1 : i == 2 ? -1 : 0)
         : b == 1 ? (i == 3 ? 1 : i == 4 ? -1 : 0)
                  : (i == 5 ? 1 : i == 6 ? -1 : 0);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i & 1) ? i + 1 : i - 1;
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 0.25 : 0.125; }
  static constexpr int UP = 5;

  template <bool DZ = false, class TC>
  static __device__ __forceinline__ void relax(TC g[Q], const TC jeq[D], TC s1, TC s2, TC F,
                                               const float *rz = nullptr) {
    const TC sx = g[1] + g[2], sy = g[3] + g[4], sz = g[5] + g[6];
    const TC m0 = g[0] + sx + sy + sz;
    const TC d1 = s1 * ((g[1] - g[2]) - jeq[0]);
    const TC d2 = s1 * ((g[3] - g[4]) - jeq[1]);
    const TC d3 = s1 * ((g[5] - g[6]) - jeq[2]);
    const TC d4 = s2 * ((sx + sy + sz) - TC(6) * g[0] + TC(0.75) * m0);
    const TC d5 = s2 * (TC(2) * sx - sy - sz);
    const TC d6 = s2 * (sy - sz);
    const TC h1 = TC(0.5) * d1, h2 = TC(0.5) * d2, h3 = TC(0.5) * d3;
    const TC e4 = d4 * TC(1.0 / 42.0);
    const TC ex = d5 * TC(1.0 / 6.0), eo = d5 * TC(1.0 / 12.0), q6 = TC(0.25) * d6;
    const TC Fw = F * TC(0.125);
    if constexpr (DZ) {
      add_change<DZ>(g[0], d4 * TC(1.0 / 7.0) + F * TC(0.25), rz, 0);
      add_change<DZ>(g[1], ((Fw - h1) - e4) - ex, rz, 1);
      add_change<DZ>(g[2], ((Fw + h1) - e4) - ex, rz, 2);
      add_change<DZ>(g[3], (((Fw - h2) - e4) + eo) - q6, rz, 3);
      add_change<DZ>(g[4], (((Fw + h2) - e4) + eo) - q6, rz, 4);
      add_change<DZ>(g[5], (((Fw - h3) - e4) + eo) + q6, rz, 5);
      add_change<DZ>(g[6], (((Fw + h3) - e4) + eo) + q6, rz, 6);
    } else {
      g[0] = g[0] + d4 * TC(1.0 / 7.0) + F * TC(0.25);
      g[1] = g[1] - h1 - e4 - ex + Fw;
      g[2] = g[2] + h1 - e4 - ex + Fw;
      g[3] = g[3] - h2 - e4 + eo - q6 + Fw;
      g[4] = g[4] + h2 - e4 + eo - q6 + Fw;
      g[5] = g[5] - h3 - e4 + eo + q6 + Fw;
      g[6] = g[6] + h3 - e4 + eo + q6 + Fw;
    }
  }
};

// ---------------------------------------------------------------------------
// Lattices without a rest direction (Sec. 2.2), in the paper's order.
// D2Q4: c_0..c_3 = (1,0),(0,1),(-1,0),(0,-1); w_i = 1/4; c_s^2 = 1/2.
// The paper prints no M for it; the basis used is the conserved row, the two
// first moments and the traceless second moment:
//   m0 = sum g, m1 = g0 - g2, m2 = g1 - g3, m3 = g0 - g1 + g2 - g3,
// squared norms (4, 2, 2, 4), S_d = diag(s0, s1, s1, s2); m3eq = 0, and
// w_i F has no m3 part.
// ---------------------------------------------------------------------------
struct D2Q4 {
  static constexpr int D = 2, Q = 4;
  static constexpr int REST = -1;
  static constexpr double CS2 = 0.5;
  __host__ __device__ static constexpr int c(int i, int b) {
    return b == 0 ? (i == 0 ? 1 : i == 2 ? -1 : 0) : b == 1 ? (i == 1 ? 1 : i == 3 ? -1 : 0) : 0;
  }
  __host__ __device__ static constexpr int opp(int i) { return (i + 2) & 3; }
  __host__ __device__ static constexpr double w(int) { return 0.25; }
  static constexpr int UP = 1;

  template <bool DZ = false, class TC>
  static __device__ __forceinline__ void relax(TC g[Q], const TC jeq[D], TC s1, TC s2, TC F,
                                               const float *rz = nullptr) {
    const TC d1 = s1 * ((g[0] - g[2]) - jeq[0]);
    const TC d2 = s1 * ((g[1] - g[3]) - jeq[1]);
    const TC d3 = s2 * ((g[0] + g[2]) - (g[1] + g[3]));
    const TC h1 = TC(0.5) * d1, h2 = TC(0.5) * d2, q3 = TC(0.25) * d3;
    const TC Fw = F * TC(0.25);
    if constexpr (DZ) {
      add_change<DZ>(g[0], (Fw - h1) - q3, rz, 0);
      add_change<DZ>(g[1], (Fw - h2) + q3, rz, 1);
      add_change<DZ>(g[2], (Fw + h1) - q3, rz, 2);
      add_change<DZ>(g[3], (Fw + h2) + q3, rz, 3);
    } else {
      g[0] = g[0] - h1 - q3 + Fw;
      g[1] = g[1] - h2 + q3 + Fw;
      g[2] = g[2] + h1 - q3 + Fw;
      g[3] = g[3] + h2 + q3 + Fw;
    }
  }
};

// D3Q6: c_0..c_5 = +-x, +-y, +-z; w_i = 1/6; c_s^2 = 1/3.  Basis: m0, the
// three first moments, m4 = 2cx^2 - cy^2 - cz^2 and m5 = cy^2 - cz^2,
// squared norms (6, 2, 2, 2, 12, 4), S_d = diag(s0, s1 x3, s2 x2);
// m4eq = m5eq = 0, and w_i F has no m4 or m5 part.
struct D3Q6 {
  static constexpr int D = 3, Q = 6;
  static constexpr int REST = -1;
  static constexpr double CS2 = 1.0 / 3.0;
  __host__ __device__ static constexpr int c(int i, int b) {
    return b == 0 ? (i == 0 ? 1 : i == 1 ? -1 : 0)
         : b == 1 ? (i == 2 ? 1 : i == 3 ? -1 : 0)
                  : (i == 4 ? 1 : i == 5 ? -1 : 0);
  }
  __host__ __device__ static constexpr int opp(int i) { return i ^ 1; }
  __host__ __device__ static constexpr double w(int) { return 1.0 / 6.0; }
  static constexpr int UP = 4;

  template <bool DZ = false, class TC>
  static __device__ __forceinline__ void relax(TC g[Q], const TC jeq[D], TC s1, TC s2, TC F,
                                               const float *rz = nullptr) {
    const TC sx = g[0] + g[1], sy = g[2] + g[3], sz = g[4] + g[5];
    const TC d1 = s1 * ((g[0] - g[1]) - jeq[0]);
    const TC d2 = s1 * ((g[2] - g[3]) - jeq[1]);
    const TC d3 = s1 * ((g[4] - g[5]) - jeq[2]);
    const TC d4 = s2 * (TC(2) * sx - sy - sz);
    const TC d5 = s2 * (sy - sz);
    const TC h1 = TC(0.5) * d1, h2 = TC(0.5) * d2, h3 = TC(0.5) * d3;
    const TC ex = d4 * TC(1.0 / 6.0), eo = d4 * TC(1.0 / 12.0), q5 = TC(0.25) * d5;
    const TC Fw = F * TC(1.0 / 6.0);
    if constexpr (DZ) {
      add_change<DZ>(g[0], (Fw - h1) - ex, rz, 0);
      add_change<DZ>(g[1], (Fw + h1) - ex, rz, 1);
      add_change<DZ>(g[2], ((Fw - h2) + eo) - q5, rz, 2);
      add_change<DZ>(g[3], ((Fw + h2) + eo) - q5, rz, 3);
      add_change<DZ>(g[4], ((Fw - h3) + eo) + q5, rz, 4);
      add_change<DZ>(g[5], ((Fw + h3) + eo) + q5, rz, 5);
    } else {
      g[0] = g[0] - h1 - ex + Fw;
      g[1] = g[1] + h1 - ex + Fw;
      g[2] = g[2] - h2 + eo - q5 + Fw;
      g[3] = g[3] + h2 + eo - q5 + Fw;
      g[4] = g[4] - h3 + eo + q5 + Fw;
      g[5] = g[5] + h3 + eo + q5 + Fw;
    }
  }
};

// True for a direction with a non-zero velocity (every i but the rest one).
template <class L> __host__ __device__ constexpr bool moving(int i) { return i != L::REST; }

}  // namespace mdf

// Kernel templates of the MDF-LBM stepper: fused pull-stream + moments +
// MRT collision + store (Eq. 2-7, 3-15, 2-4, 3-21), the derived-field
// epilogue (Eq. 3-16 .. 3-19), initialisation, link masks and FP64
// reductions.  Instantiated per lattice in mdf_d2q5.cu / mdf_d3q7.cu.
//
// Memory layout (structure of arrays): set a, direction i, node (x, y, z)
//   f[((a * Q + i) * plane) + (z * ny + y) * px + x],   plane = px * ny * nz,
// with px = nx rounded up to a multiple of 32 so every row starts on a
// 128-byte boundary.  Two buffers alternate (pull scheme): the current
// buffer holds post-collision populations f*(x, t - 1); an update pulls
// f_i(x, t) = f*_i(x - c_i, t - 1), collides and stores f*_i(x, t) at x in
// the other buffer, so every population is read once and written once.
// A link whose source x - c_i lies behind a wall is replaced by the
// anti-halfway bounce-back of the node's own opposite population:
//   f_i(x, t) = -f*_{opp(i)}(x, t - 1) + 2 w_i ubar_wall.
#pragma once

#include <type_traits>

#include "mdf_internal.h"
#include "mdf_lattice.cuh"
#include "mdf_f64.cuh"
#include "mdf_pack16.cuh"

namespace mdf {

template <class TS> struct ComputeOf { using T = float; };
template <> struct ComputeOf<double> { using T = double; };

// A relaxation rate in the compute type (the FP32 copy is rounded on the
// host, so no kernel converts from FP64).
template <class TC> __device__ __forceinline__ TC rate(double d, float f) {
  if constexpr (std::is_same<TC, double>::value) return d;
  else return f;
}

// FP32 storage takes the dithered (stochastic) rounding of the collision
// (mdf_lattice.cuh); the other storage types round to nearest.
template <class TS> constexpr bool dithered() { return std::is_same<TS, float>::value; }

// Time step of this launch for the dither draws: the lattice's step counter
// as set on the device before the launch group, plus the launch's offset in
// the group (launches captured in a CUDA graph read the counter afresh on
// every replay).
__device__ __forceinline__ int launch_step(const DevArgs &A) {
  return (A.clock ? __ldg(A.clock) : 0) + A.tk;
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Index of the node x - c_i (periodic wrap on every axis; walls are masked).
template <class L>
__device__ __forceinline__ long long pull_src(const DevArgs &A, int x, int y, int z, int i) {
  const int sx = wrap(x - L::c(i, 0), A.nx);
  const int sy = wrap(y - L::c(i, 1), A.ny);
  const int sz = L::D == 3 ? wrap(z - L::c(i, 2), A.nz) : z;
  return ((long long)sz * A.ny + sy) * A.px + sx;
}

// Pull the Q populations of one set (carrying alpha, stored from `base` with
// direction stride `stride`) arriving at node idx.
template <class L, class TS, bool WALLS>
__device__ __forceinline__ void pull_set_p(const TS *__restrict__ base, long long stride,
                                           int alpha, long long idx,
                                           const long long (&src)[L::Q], uint8_t m,
                                           const double (&lid_u)[3],
                                           typename ComputeOf<TS>::T (&g)[L::Q]) {
  using TC = typename ComputeOf<TS>::T;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    if (WALLS && moving<L>(i) && ((m >> L::opp(i)) & 1)) {
      // anti-halfway bounce-back; in shifted storage the alpha = 0 wall value
      // rho0 and the rest shift cancel, leaving -g*_opp + 2 w_i u_wall(alpha)
      TC v = -TC(Codec<TS>::load(base + (long long)L::opp(i) * stride + idx));
      if (alpha >= 1 && i == L::opp(L::UP) && (m & 0x80u))
        v += TC(2.0 * L::w(i) * lid_u[alpha - 1]);
      g[i] = v;
    } else {
      g[i] = Codec<TS>::load(base + (long long)i * stride + src[i]);
    }
  }
}

// Pull the Q populations of set `a` (carrying alpha) arriving at node idx.
template <class L, class TS, bool WALLS>
__device__ __forceinline__ void pull_set(const DevArgs &A, const TS *__restrict__ fin, int a,
                                         int alpha, long long idx, const long long (&src)[L::Q],
                                         uint8_t m, typename ComputeOf<TS>::T (&g)[L::Q]) {
  pull_set_p<L, TS, WALLS>(fin + (long long)a * L::Q * A.plane, A.plane, alpha, idx, src, m,
                           A.lid_u, g);
}

// Derived fields of Eq. 2-7, 3-15 .. 3-19 at one node from the pulled
// (pre-collision) shifted populations, computed in the compute type TC and
// written as FP64.  gv: the d velocity sets; h: the alpha = 0 set (ignored
// unless with_rho).  FP32 suffices here: the populations are rest-shifted,
// so J (~u^2) and u u + P' carry absolute rounding ~1e-7 |J| while the
// first moment of f^ne they differ by is ~1e-3..1e-1 |J| at the workloads'
// sizes; the FP32 storage rounding of g dominates the error.  (GB300's FP64
// throughput is too low for FP64 arithmetic here to stay HBM-bound; the
// widening to FP64 is built on the integer pipe, leaving two FP64 adds.)
template <class L, class TC>
__device__ __forceinline__ void write_fields(const DevArgs &A, long long n, long long N,
                                             const TC (&gv)[L::D][L::Q], const TC (&h)[L::Q],
                                             const TC (&F)[L::D]) {
  constexpr int D = L::D, Q = L::Q;
  TC u[D], J[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    TC s = TC(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) s += gv[a][i];
    u[a] = A.scheme2 ? s + TC(0.5) * F[a] : s;  // Eq. 2-7a under Scheme II
#pragma unroll
    for (int b = 0; b < D; ++b) {
      TC t = TC(0);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (L::c(i, b) > 0) t += gv[a][i];
        if (L::c(i, b) < 0) t -= gv[a][i];
      }
      J[a][b] = t;  // sum_i c_{i,b} g_{i,a}
    }
  }
  TC tr = TC(0), usq = TC(0);
#pragma unroll
  for (int a = 0; a < D; ++a) { tr += J[a][a]; usq += u[a] * u[a]; }
  const TC Pp = (tr - usq) * TC(1.0 / D);  // Eq. 3-15, P' = P - P0, R = 0
  if (A.P) A.P[n] = 1.0 + widen_f32(Pp);
  if (A.u)
#pragma unroll
    for (int a = 0; a < D; ++a) A.u[a * N + n] = widen_f32(u[a]);
  if (A.rho && A.with_rho) {
    TC s = TC(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) s += h[i];
    A.rho[n] = 1.0 + widen_f32(s);
  }
  if (!(A.G || A.div || A.S || A.sigma || A.omega)) return;
  // first moment of f^ne: sum_i c_{i,b} (f - f^eq)_{i,a} = J - u_a u_b - P' delta_ab
  // (under Scheme II f = fbar + F/2, whose first moment is fbar's)
  TC mne[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int b = 0; b < D; ++b) mne[a][b] = J[a][b] - u[a] * u[b] - (a == b ? Pp : TC(0));
  const TC pref = TC(-A.s1 / L::CS2);  // Eq. 3-16 with dt = 1
  if (A.G)
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) A.G[(a * D + b) * N + n] = widen_f32(pref * mne[a][b]);
  if (A.div) {
    TC s = TC(0);
#pragma unroll
    for (int a = 0; a < D; ++a) s += mne[a][a];
    A.div[n] = widen_f32(pref * s);  // Eq. 3-16a
  }
  if (A.S || A.sigma) {
    int k = 0;
    const TC sig = TC(-(1.0 - 0.5 * A.s1));  // Eq. 3-17a with rho0 = 1
    const TC half_pref = TC(0.5) * pref;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = a; b < D; ++b, ++k) {
        const TC sym = mne[a][b] + mne[b][a];
        if (A.S) A.S[k * N + n] = widen_f32(half_pref * sym);  // Eq. 3-17
        if (A.sigma) A.sigma[k * N + n] = widen_f32(sig * sym);
      }
  }
  if (A.omega) {  // Eq. 3-18, 3-19: omega = curl u
    if (D == 2) {
      A.omega[n] = widen_f32(pref * (mne[1][0] - mne[0][1]));
    } else {
      A.omega[n] = widen_f32(pref * (mne[2][1] - mne[1][2]));
      A.omega[N + n] = widen_f32(pref * (mne[0][2] - mne[2][0]));
      A.omega[2 * N + n] = widen_f32(pref * (mne[1][0] - mne[0][1]));
    }
  }
}

// Eq. 2-7, 3-15, 2-4 (moments of Eq. 3-7a) and 3-21 at one node, in place
// on its pulled populations: g (the d velocity sets) and h (the alpha = 0
// set) become the post-collision populations.  F: Fbar_alpha, alpha = 1..d.
//
// S2 (Scheme II): g holds fbar = f - F/2 and the update is Eq. 2-3c with ubar from
// Eq. 2-7a.  In moment space (M has orthogonal rows, m = M fbar, F_m = M F):
//   row 0:    m0 - s0 (m0 - ubar) + (1 - s0/2) Fbar = m0 + Fbar, as
//             m0 - ubar = -Fbar/2, so s0 drops out;
//   rows b:   m_b - s1 (m_b - ubar_a ubar_b - P' delta_ab), F_m = 0;
//   m4 row:   with k = sum_i w_i M4_i, m4eq = k ubar = k (m0 + Fbar/2), and
//             the s2 (Fbar/2) terms cancel: k (m0 + Fbar) + (1 - s2)(m4 - k m0);
//   other rows carry no equilibrium or force part.
// So Scheme II is the Eq. 3-21 relaxation below with the equilibrium first
// moments built from ubar (m4 relaxes towards k m0 there already) and the
// same w_i Fbar source.
//
// DITHER (FP32 storage): the velocity sets' post-collision values are
// rounded stochastically, with the offsets drawn from `key` (node_key of
// the node's global index and the time step; see mdf_lattice.cuh).
template <class L, class TC, bool S2 = false>
__device__ __forceinline__ void node_moments(const TC (&g)[L::D][L::Q], const TC (&F)[L::D],
                                             TC (&u)[L::D], TC &Pp) {
  constexpr int D = L::D, Q = L::Q;
  // Eq. 2-7: u_alpha = sum_i f_{i,alpha} (the rest shift has zero sum);
  // Eq. 3-15: P' = (1/d)(sum_alpha sum_i c_{i,alpha} g_{i,alpha} - |u|^2).
  TC tr = TC(0), usq = TC(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    TC s = TC(0), t = TC(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      s += g[a][i];
      if (L::c(i, a) > 0) t += g[a][i];
      if (L::c(i, a) < 0) t -= g[a][i];
    }
    if constexpr (S2) u[a] = s + TC(0.5) * F[a];  // Eq. 2-7a
    else u[a] = s;
    tr += t;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) usq += u[a] * u[a];
  Pp = (tr - usq) * TC(1.0 / D);
}

// Relaxation of velocity set a (alpha = a + 1) of one node from its moments.
template <class L, class TC, bool DITHER = false>
__device__ __forceinline__ void relax_velocity_set(TC (&ga)[L::Q], int a, const TC (&u)[L::D], TC Pp,
                                                   TC s1, TC s2, TC Fa, uint32_t key) {
  constexpr int D = L::D, Q = L::Q;
  TC jeq[D];  // Eq. 3-7a: sum_i c_i f^eq = u_alpha u + P E_alpha (shifted: P')
#pragma unroll
  for (int b = 0; b < D; ++b) jeq[b] = u[a] * u[b] + (a == b ? Pp : TC(0));
  if constexpr (DITHER) {  // population k = a Q + i draws byte k & 3 of word k >> 2
    float rz[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int k = a * Q + i;
      rz[i] = rand_scale(rand_word(key, k >> 2), k & 3);
    }
    L::template relax<true>(ga, jeq, s1, s2, Fa, rz);
  } else {
    L::relax(ga, jeq, s1, s2, Fa);
  }
}

// Relaxation of the alpha = 0 set of one node (ubar_0 = rho0 + rho'); r
// receives rho'.
template <class L, class TC>
__device__ __forceinline__ void relax_rho_set(TC (&h)[L::Q], const TC (&u)[L::D], TC s1, TC s2, TC &r) {
  constexpr int D = L::D, Q = L::Q;
  r = TC(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) r += h[i];
  TC jeq[D];  // ubar_0 u
#pragma unroll
  for (int b = 0; b < D; ++b) jeq[b] = (TC(1) + r) * u[b];
  L::relax(h, jeq, s1, s2, TC(0));
}

template <class L, class TC, bool S2 = false, bool DITHER = false>
__device__ __forceinline__ void collide_node(TC (&g)[L::D][L::Q], TC (&h)[L::Q], bool with_rho,
                                             const TC (&F)[L::D], TC s1, TC s2,
                                             TC (&M)[L::D + 2], uint32_t key = 0u) {
  constexpr int D = L::D;
  TC u[D], Pp;
  node_moments<L, TC, S2>(g, F, u, Pp);
#pragma unroll
  for (int a = 0; a < D; ++a) M[a] = u[a];
  M[D] = Pp;
  M[D + 1] = TC(0);
#pragma unroll
  for (int a = 0; a < D; ++a) relax_velocity_set<L, TC, DITHER>(g[a], a, u, Pp, s1, s2, F[a], key);
  if (with_rho) {
    TC r;
    relax_rho_set<L, TC>(h, u, s1, s2, r);
    M[D + 1] = r;
  }
}

// One lattice update per thread-node: pull, moments, (fields), collide, store.
// Used for every grid; the vector kernel below covers x extents divisible by
// its width.
template <class L, class TS, int MODE, bool WALLS>
__global__ void __launch_bounds__(kMaxBlock) k_update(const DevArgs A) {
  using TC = typename ComputeOf<TS>::T;
  constexpr int D = L::D, Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= A.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long idx = ((long long)z * A.ny + y) * A.px + x;
  long long src[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) src[i] = pull_src<L>(A, x, y, z, i);
  const uint8_t m = WALLS ? A.mask[idx] : uint8_t(0);
  const TS *__restrict__ fin = static_cast<const TS *>(A.fin);
  const int a1 = A.with_rho;  // set index of alpha = 1

  TC g[D][Q], h[Q];
#pragma unroll
  for (int al = 1; al <= D; ++al) pull_set<L, TS, WALLS>(A, fin, a1 + al - 1, al, idx, src, m, g[al - 1]);
  if (A.with_rho) pull_set<L, TS, WALLS>(A, fin, 0, 0, idx, src, m, h);

  TC F[D];
#pragma unroll
  for (int a = 0; a < D; ++a)
    F[a] = A.force ? __ldg(static_cast<const TC *>(A.force) + a * A.plane + idx) : TC(0);
  if (MODE != MODE_STEP) {
    const long long N = (long long)A.nx * A.ny * A.nz;
    const long long n = ((long long)z * A.ny + y) * A.nx + x;
    write_fields<L, TC>(A, n, N, g, h, F);
    if (MODE == MODE_FIELDS) return;
  }

  TC M[D + 2];
  constexpr bool DZ = dithered<TS>();
  uint32_t key = 0u;
  if constexpr (DZ) key = node_key(A.key_base + ((long long)z * A.ny + y) * A.nx + x, launch_step(A));
  if (A.scheme2) collide_node<L, TC, true, DZ>(g, h, A.with_rho != 0, F, rate<TC>(A.s1, A.s1f), rate<TC>(A.s2, A.s2f), M, key);
  else collide_node<L, TC, false, DZ>(g, h, A.with_rho != 0, F, rate<TC>(A.s1, A.s1f), rate<TC>(A.s2, A.s2f), M, key);

  TS *__restrict__ fout = static_cast<TS *>(A.fout);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    TS *base = fout + (long long)(a1 + a) * Q * A.plane + idx;
#pragma unroll
    for (int i = 0; i < Q; ++i) Codec<TS>::store(base + (long long)i * A.plane, g[a][i]);
  }
  if (A.with_rho) {
    TS *base = fout + idx;
#pragma unroll
    for (int i = 0; i < Q; ++i) Codec<TS>::store(base + (long long)i * A.plane, h[i]);
  }
}

// ---------------------------------------------------------------------------
// Vector update: each thread owns VX consecutive x-nodes (x0 .. x0+VX-1) and
// moves them with one 8/16-byte access per population array.  The two
// x-shifted pulls take the missing end value from the neighbouring lane
// (warp shuffle) or, at a warp or row edge, with one scalar load.  All lanes
// stay alive through the shuffles (threads past the row end clamp their
// reads into the row and skip every store).  Node offsets are 32-bit.
// Per node the arithmetic is the scalar kernel's, so both produce the same
// bits.
// ---------------------------------------------------------------------------
template <class TS, int VX> struct VecIO;
template <> struct VecIO<float, 4> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  static __device__ __forceinline__ void store(float *p, const float (&v)[4]) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
  }
};
template <> struct VecIO<float, 2> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[2]) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    v[0] = t.x; v[1] = t.y;
  }
  static __device__ __forceinline__ void store(float *p, const float (&v)[2]) {
    __stcs(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
  }
};
template <> struct VecIO<float, 8> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
};
template <> struct VecIO<double, 2> {
  static __device__ __forceinline__ void load(const double *p, double (&v)[2]) {
    const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    v[0] = t.x; v[1] = t.y;
  }
  static __device__ __forceinline__ void store(double *p, const double (&v)[2]) {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
  }
};
// 16-bit storage: VX/2 packed pairs per access (VX = 4: 8 bytes, VX = 8: 16).
template <class H2> struct Pair;
template <> struct Pair<__half2> {
  static __device__ __forceinline__ float2 to_f2(__half2 v) { return __half22float2(v); }
  static __device__ __forceinline__ __half2 from(float a, float b) { return __floats2half2_rn(a, b); }
};
template <> struct Pair<__nv_bfloat162> {
  static __device__ __forceinline__ float2 to_f2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ __nv_bfloat162 from(float a, float b) {
    return __floats2bfloat162_rn(a, b);
  }
};
template <class T16, class H2, int VX> struct VecIO16 {
  static_assert(VX == 2 || VX == 4 || VX == 8, "16-bit vectors of 2, 4 or 8");
  using Raw = typename std::conditional<VX == 2, uint32_t,
              typename std::conditional<VX == 4, uint2, uint4>::type>::type;
  static __device__ __forceinline__ void load(const T16 *p, float (&v)[VX]) {
    const Raw r = __ldg(reinterpret_cast<const Raw *>(p));
    const uint32_t *w = reinterpret_cast<const uint32_t *>(&r);
#pragma unroll
    for (int k = 0; k < VX / 2; ++k) {
      const float2 f = Pair<H2>::to_f2(*reinterpret_cast<const H2 *>(&w[k]));
      v[2 * k] = f.x;
      v[2 * k + 1] = f.y;
    }
  }
  static __device__ __forceinline__ void store(T16 *p, const float (&v)[VX]) {
    Raw r;
    uint32_t *w = reinterpret_cast<uint32_t *>(&r);
#pragma unroll
    for (int k = 0; k < VX / 2; ++k) {
      const H2 hv = Pair<H2>::from(v[2 * k], v[2 * k + 1]);
      w[k] = *reinterpret_cast<const uint32_t *>(&hv);
    }
    *reinterpret_cast<Raw *>(p) = r;
  }
};
// one element: the scalar codec
template <class T16, class H2> struct VecIO16<T16, H2, 1> {
  static __device__ __forceinline__ void load(const T16 *p, float (&v)[1]) { v[0] = Codec<T16>::load(p); }
  static __device__ __forceinline__ void store(T16 *p, const float (&v)[1]) { Codec<T16>::store(p, v[0]); }
};
template <> struct VecIO<float, 1> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[1]) { v[0] = __ldg(p); }
  static __device__ __forceinline__ void store(float *p, const float (&v)[1]) { __stcs(p, v[0]); }
};
template <int VX> struct VecIO<__half, VX> : VecIO16<__half, __half2, VX> {};
template <int VX> struct VecIO<__nv_bfloat16, VX> : VecIO16<__nv_bfloat16, __nv_bfloat162, VX> {};

struct VecRows {
  int row0, row_ym, row_yp, row_zm, row_zp;  // row offsets of the pull sources
  int x0, xl, xr;                            // first x, wrapped x0 - 1 and x0 + VX
  bool ledge, redge;                         // x - 1 / x + VX not held by a neighbour lane
};

// Anti-halfway bounce-back on the wall links of VX nodes of one set (see
// pull_set): the pulled value is minus the node's own opposite population,
// plus the lid term on the lid.
template <class L, class TS, int VX>
__device__ __forceinline__ void bounce_back_vec(const DevArgs &A, const TS *__restrict__ base, int alpha,
                                                const VecRows &R, const uint8_t (&m)[VX],
                                                typename ComputeOf<TS>::T (&v)[L::Q][VX]) {
  using TC = typename ComputeOf<TS>::T;
#pragma unroll
  for (int i = 0; i < L::Q; ++i)
#pragma unroll
    for (int j = 0; j < VX; ++j)
      if (moving<L>(i) && ((m[j] >> L::opp(i)) & 1)) {
        TC w = -TC(Codec<TS>::load(base + (long long)L::opp(i) * A.plane + R.row0 + R.x0 + j));
        if (alpha >= 1 && i == L::opp(L::UP) && (m[j] & 0x80u))
          w += TC(2.0 * L::w(i) * A.lid_u[alpha - 1]);
        v[i][j] = w;
      }
}

// Pull VX consecutive nodes of one set (carrying alpha) into v[i][j].
template <class L, class TS, int VX, bool WALLS>
__device__ __forceinline__ void pull_set_vec(const DevArgs &A, const TS *__restrict__ base,
                                             int alpha, const VecRows &R, const uint8_t (&m)[VX],
                                             typename ComputeOf<TS>::T (&v)[L::Q][VX]) {
  using TC = typename ComputeOf<TS>::T;
  constexpr int Q = L::Q;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const TS *p = base + (long long)i * A.plane;
    if (L::c(i, 0) == 1) {  // pulls from x - 1
      TC own[VX];
      VecIO<TS, VX>::load(p + R.row0 + R.x0, own);
      TC pv = __shfl_up_sync(0xffffffffu, own[VX - 1], 1);
      if (R.ledge) pv = Codec<TS>::load(p + R.row0 + R.xl);
      v[i][0] = pv;
#pragma unroll
      for (int j = 1; j < VX; ++j) v[i][j] = own[j - 1];
    } else if (L::c(i, 0) == -1) {  // pulls from x + 1
      TC own[VX];
      VecIO<TS, VX>::load(p + R.row0 + R.x0, own);
      TC nv = __shfl_down_sync(0xffffffffu, own[0], 1);
      if (R.redge) nv = Codec<TS>::load(p + R.row0 + R.xr);
#pragma unroll
      for (int j = 0; j < VX - 1; ++j) v[i][j] = own[j + 1];
      v[i][VX - 1] = nv;
    } else {
      const int r = L::c(i, 1) == 1 ? R.row_ym : L::c(i, 1) == -1 ? R.row_yp
                  : L::c(i, 2) == 1 ? R.row_zm : L::c(i, 2) == -1 ? R.row_zp : R.row0;
      VecIO<TS, VX>::load(p + r + R.x0, v[i]);
    }
  }
  if (WALLS) bounce_back_vec<L, TS, VX>(A, base, alpha, R, m, v);
}

// 16-bit storage, all sets: every population word of the VX nodes is loaded
// before any is converted, so all of a thread's reads are in flight
// together; then the x-shifted pulls take their end values from the
// neighbouring lanes (or, at a warp or row edge, the scalar loads issued
// with the words), and the wall links bounce back.  Same values as
// pull_set_vec.
template <class L, class TS, int VX, bool WALLS>
__device__ __forceinline__ void pull_all_vec16(const DevArgs &A, const TS *__restrict__ fin,
                                               const VecRows &R, const uint8_t (&m)[VX],
                                               float (&g)[L::D][L::Q][VX], float (&h)[L::Q][VX]) {
  constexpr int D = L::D, Q = L::Q;
  using PK = Packed16<TS, VX>;
  typename PK::W wv[D + 1][Q];
  unsigned edge[D + 1][2];
  const int a1 = A.with_rho;
#pragma unroll
  for (int s = 0; s <= D; ++s) {  // velocity sets first, the continuity set last
    if (s == D && !A.with_rho) break;
    const TS *base = fin + (long long)(s < D ? a1 + s : 0) * Q * A.plane;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const TS *p = base + (long long)i * A.plane;
      const int r = L::c(i, 1) == 1 ? R.row_ym : L::c(i, 1) == -1 ? R.row_yp
                  : L::c(i, 2) == 1 ? R.row_zm : L::c(i, 2) == -1 ? R.row_zp : R.row0;
      wv[s][i] = PK::load(p + r + R.x0);
      if (L::c(i, 0) == 1) edge[s][0] = R.ledge ? ldg_bits16(p + R.row0 + R.xl) : 0u;
      if (L::c(i, 0) == -1) edge[s][1] = R.redge ? ldg_bits16(p + R.row0 + R.xr) : 0u;
    }
  }
#pragma unroll
  for (int s = 0; s <= D; ++s) {
    if (s == D && !A.with_rho) break;
    float(&v)[Q][VX] = s < D ? g[s < D ? s : 0] : h;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const typename PK::W w = wv[s][i];
      if (L::c(i, 0) == 1) {  // from x - 1: v[0] from the lane to the left
        unsigned nb = __shfl_up_sync(0xffffffffu, PK::last_word(w), 1);
        nb = R.ledge ? edge[s][0] : (VX == 1 ? nb : nb >> 16);
        v[i][0] = bits_to_float<TS>(nb);
#pragma unroll
        for (int j = 1; j < VX; ++j) v[i][j] = bits_to_float<TS>(PK::bits(w, j - 1));
      } else if (L::c(i, 0) == -1) {  // from x + 1: v[VX - 1] from the lane to the right
        unsigned nb = __shfl_down_sync(0xffffffffu, PK::first_word(w), 1);
        nb = R.redge ? edge[s][1] : (nb & 0xffffu);
#pragma unroll
        for (int j = 0; j < VX - 1; ++j) v[i][j] = bits_to_float<TS>(PK::bits(w, j + 1));
        v[i][VX - 1] = bits_to_float<TS>(nb);
      } else {
#pragma unroll
        for (int q = 0; q < VX / 2; ++q) {
          const float2 f = PK::lanes(w, q);
          v[i][2 * q] = f.x;
          v[i][2 * q + 1] = f.y;
        }
      }
    }
    if (WALLS)
      bounce_back_vec<L, TS, VX>(A, fin + (long long)(s < D ? a1 + s : 0) * Q * A.plane, s < D ? s + 1 : 0,
                                 R, m, v);
  }
}

// Register budget of the FP32 vector kernel with 4 nodes per thread, which
// sets its resident warps at the 128-thread launch (the other widths and
// types take the compiler's choice).
constexpr int kVecF32x4Regs = 96;

template <class L, class TS, int VX, int MODE, bool WALLS, bool S2>
__device__ __forceinline__ void update_vec_body(const DevArgs &A);

template <class L, class TS, int VX, int MODE, bool WALLS, bool S2>
__global__ void __launch_bounds__(kMaxBlock) k_update_vec(const DevArgs A) {
  update_vec_body<L, TS, VX, MODE, WALLS, S2>(A);
}
template <class L, int MODE, bool WALLS, bool S2>
__global__ void __maxnreg__(kVecF32x4Regs) k_update_vec_f32x4(const DevArgs A) {
  update_vec_body<L, float, 4, MODE, WALLS, S2>(A);
}

template <class L, class TS, int VX, int MODE, bool WALLS, bool S2>
__device__ __forceinline__ void update_vec_body(const DevArgs &A) {
  using TC = typename ComputeOf<TS>::T;
  constexpr int D = L::D, Q = L::Q;
  const int lane = threadIdx.x & 31;
  int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * VX;
  const bool active = x0 < A.nx;
  if (!active) x0 = A.nx - VX;
  const int y = blockIdx.y, z = blockIdx.z;
  const int row0 = (z * A.ny + y) * A.px;
  // rows the y- and z-directed pulls come from
  const int row_ym = (z * A.ny + wrap(y - 1, A.ny)) * A.px;  // source of c_y = +1
  const int row_yp = (z * A.ny + wrap(y + 1, A.ny)) * A.px;  // source of c_y = -1
  const int row_zm = D == 3 ? (wrap(z - 1, A.nz) * A.ny + y) * A.px : row0;
  const int row_zp = D == 3 ? (wrap(z + 1, A.nz) * A.ny + y) * A.px : row0;
  const bool ledge = lane == 0 || x0 == 0;
  const bool redge = lane == 31 || x0 + VX >= A.nx;
  const int xl = x0 == 0 ? A.nx - 1 : x0 - 1;
  const int xr = x0 + VX >= A.nx ? 0 : x0 + VX;
  const TS *__restrict__ fin = static_cast<const TS *>(A.fin);
  const int a1 = A.with_rho;
  uint8_t m[VX];
  if (WALLS) {
#pragma unroll
    for (int j = 0; j < VX; ++j) m[j] = A.mask[row0 + x0 + j];
  }

  const VecRows rows{row0, row_ym, row_yp, row_zm, row_zp, x0, xl, xr, ledge, redge};
  TC g[D][Q][VX], h[Q][VX];
  if constexpr (sizeof(TS) == 2) {
    pull_all_vec16<L, TS, VX, WALLS>(A, fin, rows, m, g, h);
  } else {
#pragma unroll
    for (int al = 1; al <= D; ++al)
      pull_set_vec<L, TS, VX, WALLS>(A, fin + (long long)(a1 + al - 1) * Q * A.plane, al, rows, m,
                                     g[al - 1]);
    if (A.with_rho) pull_set_vec<L, TS, VX, WALLS>(A, fin, 0, rows, m, h);
  }

  const long long N = (long long)A.nx * A.ny * A.nz;
  const long long n0 = ((long long)z * A.ny + y) * A.nx + x0;
  TC F[D][VX];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (A.force) {
      VecIO<TC, VX>::load(static_cast<const TC *>(A.force) + a * A.plane + row0 + x0, F[a]);
    } else {
#pragma unroll
      for (int j = 0; j < VX; ++j) F[a][j] = TC(0);
    }
  }
  const TC s1 = rate<TC>(A.s1, A.s1f), s2 = rate<TC>(A.s2, A.s2f);
  constexpr bool DZ = dithered<TS>();
  if (MODE != MODE_STEP) {  // fields of the pulled state, node by node
#pragma unroll
    for (int j = 0; j < VX; ++j) {
      TC gn[D][Q], hn[Q], Fn[D];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
#pragma unroll
        for (int a = 0; a < D; ++a) gn[a][i] = g[a][i][j];
        hn[i] = h[i][j];
      }
#pragma unroll
      for (int a = 0; a < D; ++a) Fn[a] = F[a][j];
      if (active) write_fields<L, TC>(A, n0 + j, N, gn, hn, Fn);
    }
    if (MODE == MODE_FIELDS) return;
  }
  TS *__restrict__ fout = static_cast<TS *>(A.fout);
  if constexpr (!DZ) {  // node by node, then every population array stored
#pragma unroll
    for (int j = 0; j < VX; ++j) {
      TC gn[D][Q], hn[Q], Fn[D];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
#pragma unroll
        for (int a = 0; a < D; ++a) gn[a][i] = g[a][i][j];
        hn[i] = h[i][j];
      }
#pragma unroll
      for (int a = 0; a < D; ++a) Fn[a] = F[a][j];
      TC M[D + 2];
      collide_node<L, TC, S2>(gn, hn, A.with_rho != 0, Fn, s1, s2, M);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
#pragma unroll
        for (int a = 0; a < D; ++a) g[a][i][j] = gn[a][i];
        h[i][j] = hn[i];
      }
    }
    if (!active) return;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int i = 0; i < Q; ++i)
        VecIO<TS, VX>::store(fout + ((long long)(a1 + a) * Q + i) * A.plane + row0 + x0, g[a][i]);
    if (A.with_rho)
#pragma unroll
      for (int i = 0; i < Q; ++i) VecIO<TS, VX>::store(fout + (long long)i * A.plane + row0 + x0, h[i]);
    return;
  }
  // With the dither draws (FP32): set by set, with the per-node arithmetic
  // of collide_node.  The moments of every node first, then each set
  // relaxed for every node and stored, so that its registers are free for
  // the next set (the node-by-node order needs ~145 registers here).
  TC u[VX][D], Pp[VX];
  uint32_t key[VX];
  const int tstep = DZ ? launch_step(A) : 0;
#pragma unroll
  for (int j = 0; j < VX; ++j) {
    TC gn[D][Q], Fn[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      Fn[a] = F[a][j];
#pragma unroll
      for (int i = 0; i < Q; ++i) gn[a][i] = g[a][i][j];
    }
    node_moments<L, TC, S2>(gn, Fn, u[j], Pp[j]);
    key[j] = DZ ? node_key(A.key_base + n0 + j, tstep) : 0u;
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
#pragma unroll
    for (int j = 0; j < VX; ++j) {
      TC ga[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) ga[i] = g[a][i][j];
      relax_velocity_set<L, TC, DZ>(ga, a, u[j], Pp[j], s1, s2, F[a][j], key[j]);
#pragma unroll
      for (int i = 0; i < Q; ++i) g[a][i][j] = ga[i];
    }
    if (active)
#pragma unroll
      for (int i = 0; i < Q; ++i)
        VecIO<TS, VX>::store(fout + ((long long)(a1 + a) * Q + i) * A.plane + row0 + x0, g[a][i]);
  }
  if (A.with_rho) {
#pragma unroll
    for (int j = 0; j < VX; ++j) {
      TC hn[Q], r;
#pragma unroll
      for (int i = 0; i < Q; ++i) hn[i] = h[i][j];
      relax_rho_set<L, TC>(hn, u[j], s1, s2, r);
#pragma unroll
      for (int i = 0; i < Q; ++i) h[i][j] = hn[i];
    }
    if (active)
#pragma unroll
      for (int i = 0; i < Q; ++i) VecIO<TS, VX>::store(fout + (long long)i * A.plane + row0 + x0, h[i]);
  }
}

// Seed (u, P' = P - 1) of node n in the compute type TC: P' is formed in
// FP64 (P ~ 1), then both are rounded to TC (narrow_to: integer pipe).
template <class L, class TC>
__device__ __forceinline__ void seed_at(const DevArgs &A, long long N, long long n, TC (&u)[L::D],
                                        TC &Pp) {
#pragma unroll
  for (int b = 0; b < L::D; ++b) u[b] = narrow_to<TC>(A.uin[b * N + n]);
  Pp = narrow_to<TC>(A.Pin[n] - 1.0);
}

// Shifted equilibrium g^eq_i of set alpha (Eq. 2-4 minus the rest state)
// from a node's (u, P'): alpha >= 1: w_i [u_a + (c_i.u u_a + c_{i,a} P') /
// c_s^2]; alpha = 0 (ubar_0 = rho0 = 1): w_i c_i.u / c_s^2.
template <class L, class TC>
__device__ __forceinline__ TC geq_v(int alpha, int i, const TC (&u)[L::D], TC Pp) {
  TC cu = TC(0);
#pragma unroll
  for (int b = 0; b < L::D; ++b) {
    if (L::c(i, b) > 0) cu += u[b];
    if (L::c(i, b) < 0) cu -= u[b];
  }
  const TC wi = TC(L::w(i)), ics2 = TC(1.0 / L::CS2);
  if (alpha == 0) return wi * cu * ics2;
  const TC ua = u[alpha - 1];
  const TC cP = L::c(i, alpha - 1) > 0 ? Pp : (L::c(i, alpha - 1) < 0 ? -Pp : TC(0));
  return wi * (ua + (cu * ua + cP) * ics2);
}

// First-order non-equilibrium part of set alpha along c_i at node n from
// the seed gradient Gin[a][b] = du_a/dx_b: -(w_i / s1) c_i . (G_alpha -
// tr G / d e_alpha), the inverse of Eq. 3-16 (its first moment is
// -(c_s^2 / s1) times the traceless gradient; the trace would read as
// pressure in Eq. 3-15).  Zero without a gradient, for alpha = 0 and for
// the rest direction.
template <class L>
__device__ __forceinline__ double fne_at(const DevArgs &A, long long N, long long n, int alpha, int i) {
  constexpr int D = L::D;
  if (!A.Gin || alpha == 0 || !moving<L>(i)) return 0.0;
  const int b = L::c(i, 0) != 0 ? 0 : L::c(i, 1) != 0 ? 1 : 2;
  const int sg = L::c(i, b);
  double g = A.Gin[((long long)(alpha - 1) * D + b) * N + n];
  if (alpha - 1 == b) {
    double tr = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) tr += A.Gin[((long long)a * D + a) * N + n];
    g -= tr / D;
  }
  return -(L::w(i) / A.s1) * sg * g;
}

template <class L, class TC>
__device__ __forceinline__ TC geq(const DevArgs &A, long long N, long long n, int alpha, int i) {
  TC u[L::D], Pp;
  seed_at<L, TC>(A, N, n, u, Pp);
  return geq_v<L, TC>(alpha, i, u, Pp);
}

// v rounded to the storage type and back (exact for FP32 and FP64).
template <class TS> __device__ __forceinline__ typename ComputeOf<TS>::T round_to(typename ComputeOf<TS>::T v) {
  if constexpr (std::is_same<TS, __half>::value) return __half2float(__float2half_rn(v));
  else if constexpr (std::is_same<TS, __nv_bfloat16>::value) return __bfloat162float(__float2bfloat16_rn(v));
  else return v;
}

// Initial state f = f^eq(P, u) written in pull form, pushed from each node:
// the population arriving at x along c_i is stored where the first update
// pulls it from, at x - c_i, or, when that link comes through a wall, in the
// slot of the opposite direction at x, whose bounce-back returns it.  Every
// slot is written once, and a node reads only its own seed.  With a seed
// gradient the population is f^eq + f^ne (fne_at); under Scheme II it is
// fbar = f - w_i Fbar_alpha / 2.  The seed is rounded once per node.  For
// the in-place AA pattern (A.aa) the state starts in the even layout, where
// each node's slots hold its own arriving populations.
template <class L, class TS, bool WALLS>
__global__ void __launch_bounds__(kMaxBlock) k_init(const DevArgs A) {
  using TC = typename ComputeOf<TS>::T;
  constexpr int D = L::D, Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= A.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long idx = ((long long)z * A.ny + y) * A.px + x;
  const long long N = (long long)A.nx * A.ny * A.nz;
  const long long n = ((long long)z * A.ny + y) * A.nx + x;
  const uint8_t m = WALLS ? A.mask[idx] : uint8_t(0);
  TC u[D], Pp;
  seed_at<L, TC>(A, N, n, u, Pp);
  TS *fout = static_cast<TS *>(A.fout);
  const int nsets = D + A.with_rho;
  for (int a = 0; a < nsets; ++a) {
    const int alpha = a + 1 - A.with_rho;
    const TC Fa = (A.scheme2 && alpha >= 1)
                      ? __ldg(static_cast<const TC *>(A.force) + (alpha - 1) * A.plane + idx) : TC(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int o = L::opp(i);
      const bool wall = WALLS && moving<L>(i) && ((m >> o) & 1);  // arrives through a wall
      TC v;
      long long dst;
      const bool lid = WALLS && wall && alpha >= 1 && o == L::UP && (m & 0x80u);
      if (A.aa && !lid) {  // in-place AA, even layout: slot i of x holds the arriving f_i(x)
        v = geq_v<L, TC>(alpha, i, u, Pp);
        if (A.Gin) v += narrow_to<TC>(fne_at<L>(A, N, n, alpha, i));
        if (A.scheme2 && alpha >= 1) v = v - TC(0.5 * L::w(i)) * Fa;
        dst = ((long long)a * Q + i) * A.plane + idx;
      } else if (wall) {  // stored in slot o at x, negated by the bounce-back
        v = -geq_v<L, TC>(alpha, i, u, Pp);
        if (A.Gin) v -= narrow_to<TC>(fne_at<L>(A, N, n, alpha, i));
        if (lid) v += TC(2.0 * L::w(o) * A.lid_u[alpha - 1]);
        if (A.scheme2 && alpha >= 1) v = v + TC(0.5 * L::w(o)) * Fa;
        dst = ((long long)a * Q + o) * A.plane + idx;
        if (A.aa) {
          // the value the pull stream's first bounce-back delivers (the lid
          // term does not cancel exactly in rounded arithmetic), so that
          // both layouts start from the same state
          v = -round_to<TS>(v) + TC(2.0 * L::w(i) * A.lid_u[alpha - 1]);
          dst = ((long long)a * Q + i) * A.plane + idx;
        }
      } else {  // stored in slot i at x - c_i
        v = geq_v<L, TC>(alpha, i, u, Pp);
        if (A.Gin) v += narrow_to<TC>(fne_at<L>(A, N, n, alpha, i));
        if (A.scheme2 && alpha >= 1) v = v - TC(0.5 * L::w(i)) * Fa;
        dst = ((long long)a * Q + i) * A.plane + pull_src<L>(A, x, y, z, i);
      }
      Codec<TS>::store(fout + dst, v);
    }
  }
}

// Block-wide FP64 sum of k values (fixed order: deterministic).
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *out) {
  __shared__ double sh[K][kReduceThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int w = 0; w < kReduceThreads / 32; ++w) s += sh[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
}

// Grid-stride FP64 reduction over all nodes.
//   RED_SUMS:     partial[k] = sum_x ubar_k (k over carried sets, Eq. 2-7)
//   RED_RESIDUAL: partial[0] = sum |u - uprev|^2, partial[1] = sum |u|^2, uprev <- u
template <class L, class TS, bool WALLS, int KIND>
__global__ void __launch_bounds__(kReduceThreads) k_reduce(const DevArgs A) {
  using TC = typename ComputeOf<TS>::T;
  constexpr int D = L::D, Q = L::Q;
  const long long N = (long long)A.nx * A.ny * A.nz;
  const TS *__restrict__ fin = static_cast<const TS *>(A.fin);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  bool bad = false;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % A.nx);
    const int y = (int)((n / A.nx) % A.ny);
    const int z = (int)(n / ((long long)A.nx * A.ny));
    const long long idx = ((long long)z * A.ny + y) * A.px + x;
    long long src[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) src[i] = pull_src<L>(A, x, y, z, i);
    const uint8_t m = WALLS ? A.mask[idx] : uint8_t(0);
    const int nsets = D + A.with_rho;
#pragma unroll
    for (int a = 0; a < D + 1; ++a) {
      if (a >= nsets) break;
      const int alpha = a + 1 - A.with_rho;
      TC g[Q];
      pull_set<L, TS, WALLS>(A, fin, a, alpha, idx, src, m, g);
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) s += (double)g[i];
      if (alpha == 0) s += 1.0;  // the rest shift of the alpha = 0 set sums to rho0
      if (A.scheme2 && alpha >= 1)  // Eq. 2-7a
        s += 0.5 * (double)__ldg(static_cast<const TC *>(A.force) + (alpha - 1) * A.plane + idx);
      bad |= !isfinite(s);
      if (KIND == RED_SUMS) {
        acc[a] += s;
      } else if (alpha >= 1) {
        double *up = A.uprev + (long long)(alpha - 1) * N + n;
        const double dlt = s - *up;
        acc[0] += dlt * dlt;
        acc[1] += s * s;
        *up = s;
      }
    }
  }
  block_sum<4>(acc, A.partials + (long long)blockIdx.x * 4);
  if (bad) atomicExch(A.nonfinite, 1);
}

template <class L>
__global__ void k_mask(const DevArgs A, int wx, int wy, int wz, int lid, uint8_t *mask) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= A.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const int pos[3] = {x, y, z}, ext[3] = {A.nx, A.ny, A.nz}, wall[3] = {wx, wy, wz};
  uint8_t m = 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
#pragma unroll
    for (int b = 0; b < L::D; ++b) {
      const int t = pos[b] + L::c(i, b);  // the rest direction never leaves
      if (wall[b] && (t < 0 || t >= ext[b])) {
        m |= uint8_t(1u << i);
        if (lid && b == L::D - 1 && t >= ext[b]) m |= 0x80u;
      }
    }
  }
  mask[((long long)z * A.ny + y) * A.px + x] = m;
}

}  // namespace mdf

#include "mdf_eq.cuh"
#include "mdf_aa.cuh"
#include "mdf_vec16p.cuh"

namespace mdf {

// ---------------------------------------------------------------------------
// Host-side dispatch over storage / mode / walls for one lattice.
// ---------------------------------------------------------------------------
inline dim3 node_grid(const DevArgs &a) {
  return dim3((unsigned)((a.nx + kBlockX - 1) / kBlockX), (unsigned)a.ny, (unsigned)a.nz);
}

template <class L, class TS>
cudaError_t update_scalar(int mode, bool walls, const DevArgs &a, cudaStream_t s) {
  const int bx = a.block;
  const dim3 grid((unsigned)((a.nx + bx - 1) / bx), (unsigned)a.ny, (unsigned)a.nz), block(bx);
  if (walls) {
    if (mode == MODE_STEP) k_update<L, TS, MODE_STEP, true><<<grid, block, 0, s>>>(a);
    else if (mode == MODE_STEP_FIELDS) k_update<L, TS, MODE_STEP_FIELDS, true><<<grid, block, 0, s>>>(a);
    else k_update<L, TS, MODE_FIELDS, true><<<grid, block, 0, s>>>(a);
  } else {
    if (mode == MODE_STEP) k_update<L, TS, MODE_STEP, false><<<grid, block, 0, s>>>(a);
    else if (mode == MODE_STEP_FIELDS) k_update<L, TS, MODE_STEP_FIELDS, false><<<grid, block, 0, s>>>(a);
    else k_update<L, TS, MODE_FIELDS, false><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// Plain updates only: an update that writes fields runs one node per thread
// (the same bits), whose FP64 field stores are coalesced; with VX nodes per
// thread each 8-byte store of a warp lands VX * 8 bytes from the next lane's
// and the fused step took 2.5x longer (1.49 vs 0.61 ms at 4096^2).
template <class L, class TS, int VX>
cudaError_t update_vec(int mode, bool walls, const DevArgs &a, cudaStream_t s) {
  if (mode != MODE_STEP) return cudaErrorInvalidValue;
  const int bx = a.block;
  const int threads = a.nx / VX;
  const dim3 grid((unsigned)((threads + bx - 1) / bx), (unsigned)a.ny, (unsigned)a.nz), block(bx);
  // Scheme II is a separate build: its ubar needs the force before the
  // moments, which costs the Eq. 3-21 kernel registers when decided at run time
  // 3D 16-bit: populations kept packed in registers (the FP32 copies of
  // 28 x VX values do not fit; in 2D the FP32 form is the faster one)
  if constexpr (sizeof(TS) == 2 && L::D == 3) {
    if (a.scheme2) {
      if (walls) k_update_vec16p<L, TS, VX, true, true><<<grid, block, 0, s>>>(a);
      else k_update_vec16p<L, TS, VX, false, true><<<grid, block, 0, s>>>(a);
    } else {
      if (walls) k_update_vec16p<L, TS, VX, true, false><<<grid, block, 0, s>>>(a);
      else k_update_vec16p<L, TS, VX, false, false><<<grid, block, 0, s>>>(a);
    }
  } else if constexpr (std::is_same<TS, float>::value && VX == 4) {  // the register-budgeted build
    if (a.scheme2) {
      if (walls) k_update_vec_f32x4<L, MODE_STEP, true, true><<<grid, block, 0, s>>>(a);
      else k_update_vec_f32x4<L, MODE_STEP, false, true><<<grid, block, 0, s>>>(a);
    } else {
      if (walls) k_update_vec_f32x4<L, MODE_STEP, true, false><<<grid, block, 0, s>>>(a);
      else k_update_vec_f32x4<L, MODE_STEP, false, false><<<grid, block, 0, s>>>(a);
    }
  } else {
    if (a.scheme2) {
      if (walls) k_update_vec<L, TS, VX, MODE_STEP, true, true><<<grid, block, 0, s>>>(a);
      else k_update_vec<L, TS, VX, MODE_STEP, false, true><<<grid, block, 0, s>>>(a);
    } else {
      if (walls) k_update_vec<L, TS, VX, MODE_STEP, true, false><<<grid, block, 0, s>>>(a);
      else k_update_vec<L, TS, VX, MODE_STEP, false, false><<<grid, block, 0, s>>>(a);
    }
  }
  return cudaGetLastError();
}

// Vector widths built per storage type: FP32 2 or 4 (2 only in 3D, where
// 4 nodes spill registers), 16-bit 4 or 8 (4 only in 3D, where 8 nodes of
// 28 populations spill registers), FP64 2.  A
// field-writing update, any other width, an x extent not divisible by the
// width, or a plane beyond 32-bit offsets runs the scalar kernel.
template <class L, class TS>
cudaError_t update_t(int mode, bool walls, const DevArgs &a, cudaStream_t s) {
  const bool ok = mode == MODE_STEP && a.vx > 1 && a.nx % a.vx == 0 && a.plane < (1LL << 31) - 64;
  if (ok) {
    if constexpr (sizeof(TS) == 4) {
      if constexpr (L::D == 2) {
        if (a.vx == 4) return update_vec<L, TS, 4>(mode, walls, a, s);
      }
      if (a.vx == 2) return update_vec<L, TS, 2>(mode, walls, a, s);
    } else if constexpr (sizeof(TS) == 2) {
      if constexpr (L::D == 2) {
        if (a.vx == 8) return update_vec<L, TS, 8>(mode, walls, a, s);
      }
      if (a.vx == 4) return update_vec<L, TS, 4>(mode, walls, a, s);
    } else {
      if (a.vx == 2) return update_vec<L, TS, 2>(mode, walls, a, s);
    }
  }
  return update_scalar<L, TS>(mode, walls, a, s);
}

template <class L, class TS, int VX>
cudaError_t update_eq_vx(int mode, bool walls, const DevArgs &a, cudaStream_t s) {
  const int bx = a.block;
  const int threads = a.nx / VX;
  const dim3 grid((unsigned)((threads + bx - 1) / bx), (unsigned)a.ny, (unsigned)a.nz), block(bx);
  if constexpr (VX > 1) {  // plain updates only (see update_vec)
    if (mode != MODE_STEP) return cudaErrorInvalidValue;
    if (walls) k_update_eq<L, TS, VX, MODE_STEP, true><<<grid, block, 0, s>>>(a);
    else k_update_eq<L, TS, VX, MODE_STEP, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
  }
  if (walls) {
    if (mode == MODE_STEP) k_update_eq<L, TS, VX, MODE_STEP, true><<<grid, block, 0, s>>>(a);
    else if (mode == MODE_STEP_FIELDS) k_update_eq<L, TS, VX, MODE_STEP_FIELDS, true><<<grid, block, 0, s>>>(a);
    else k_update_eq<L, TS, VX, MODE_FIELDS, true><<<grid, block, 0, s>>>(a);
  } else {
    if (mode == MODE_STEP) k_update_eq<L, TS, VX, MODE_STEP, false><<<grid, block, 0, s>>>(a);
    else if (mode == MODE_STEP_FIELDS) k_update_eq<L, TS, VX, MODE_STEP_FIELDS, false><<<grid, block, 0, s>>>(a);
    else k_update_eq<L, TS, VX, MODE_FIELDS, false><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// Equilibrium-shifted storage: widths 1, 2 or 4 for plain updates (a width
// that does not divide nx runs with 1); field-writing updates run with 1.
template <class L, class TS>
cudaError_t update_eq_t(int mode, bool walls, const DevArgs &a, cudaStream_t s) {
  if constexpr (L::D == 2) {  // 3D: 4 nodes of 28 populations spill registers
    if (mode == MODE_STEP && a.vx == 4 && a.nx % 4 == 0) return update_eq_vx<L, TS, 4>(mode, walls, a, s);
  }
  if (mode == MODE_STEP && a.vx == 2 && a.nx % 2 == 0) return update_eq_vx<L, TS, 2>(mode, walls, a, s);
  return update_eq_vx<L, TS, 1>(mode, walls, a, s);
}

// Lattices without a rest direction have the rest-shifted codecs only (the
// equilibrium-shifted kernels are written for D2Q5 and D3Q7).
template <class L>
cudaError_t update_lattice(int storage, int mode, bool walls, const DevArgs &a, cudaStream_t s) {
  switch (storage) {
    case ST_F16EQ:
      if constexpr (L::REST == 0) return update_eq_t<L, __half>(mode, walls, a, s);
      return cudaErrorInvalidValue;
    case ST_BF16EQ:
      if constexpr (L::REST == 0) return update_eq_t<L, __nv_bfloat16>(mode, walls, a, s);
      return cudaErrorInvalidValue;
    case ST_F32: return a.aa ? update_aa_t<L, float>(mode, walls, a, s) : update_t<L, float>(mode, walls, a, s);
    case ST_F16: return a.aa ? update_aa_t<L, __half>(mode, walls, a, s) : update_t<L, __half>(mode, walls, a, s);
    case ST_BF16:
      return a.aa ? update_aa_t<L, __nv_bfloat16>(mode, walls, a, s) : update_t<L, __nv_bfloat16>(mode, walls, a, s);
    case ST_F64: return a.aa ? update_aa_t<L, double>(mode, walls, a, s) : update_t<L, double>(mode, walls, a, s);
  }
  return cudaErrorInvalidValue;
}

template <class L, class TS>
cudaError_t init_t(bool walls, const DevArgs &a, cudaStream_t s) {
  if (walls) k_init<L, TS, true><<<node_grid(a), kBlockX, 0, s>>>(a);
  else k_init<L, TS, false><<<node_grid(a), kBlockX, 0, s>>>(a);
  return cudaGetLastError();
}

template <class L, class TS>
cudaError_t init_eq_t(bool walls, const DevArgs &a, cudaStream_t s) {
  if (walls) k_init_eq<L, TS, true><<<node_grid(a), kBlockX, 0, s>>>(a);
  else k_init_eq<L, TS, false><<<node_grid(a), kBlockX, 0, s>>>(a);
  return cudaGetLastError();
}

template <class L>
cudaError_t init_lattice(int storage, bool walls, const DevArgs &a, cudaStream_t s) {
  switch (storage) {
    case ST_F16EQ:
      if constexpr (L::REST == 0) return init_eq_t<L, __half>(walls, a, s);
      return cudaErrorInvalidValue;
    case ST_BF16EQ:
      if constexpr (L::REST == 0) return init_eq_t<L, __nv_bfloat16>(walls, a, s);
      return cudaErrorInvalidValue;
    case ST_F32: return init_t<L, float>(walls, a, s);
    case ST_F16: return init_t<L, __half>(walls, a, s);
    case ST_BF16: return init_t<L, __nv_bfloat16>(walls, a, s);
    case ST_F64: return init_t<L, double>(walls, a, s);
  }
  return cudaErrorInvalidValue;
}

template <class L, class TS>
cudaError_t reduce_t(bool walls, int kind, const DevArgs &a, cudaStream_t s) {
  const int nb = kReduceBlocks;
  if (kind == RED_SUMS) {
    if (walls) k_reduce<L, TS, true, RED_SUMS><<<nb, kReduceThreads, 0, s>>>(a);
    else k_reduce<L, TS, false, RED_SUMS><<<nb, kReduceThreads, 0, s>>>(a);
  } else {
    if (walls) k_reduce<L, TS, true, RED_RESIDUAL><<<nb, kReduceThreads, 0, s>>>(a);
    else k_reduce<L, TS, false, RED_RESIDUAL><<<nb, kReduceThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <class L, class TS>
cudaError_t reduce_eq_t(bool walls, int kind, const DevArgs &a, cudaStream_t s) {
  const int nb = kReduceBlocks;
  if (kind == RED_SUMS) {
    if (walls) k_reduce_eq<L, TS, true, RED_SUMS><<<nb, kReduceThreads, 0, s>>>(a);
    else k_reduce_eq<L, TS, false, RED_SUMS><<<nb, kReduceThreads, 0, s>>>(a);
  } else {
    if (walls) k_reduce_eq<L, TS, true, RED_RESIDUAL><<<nb, kReduceThreads, 0, s>>>(a);
    else k_reduce_eq<L, TS, false, RED_RESIDUAL><<<nb, kReduceThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <class L>
cudaError_t reduce_lattice(int storage, bool walls, int kind, const DevArgs &a, cudaStream_t s) {
  switch (storage) {
    case ST_F16EQ:
      if constexpr (L::REST == 0) return reduce_eq_t<L, __half>(walls, kind, a, s);
      return cudaErrorInvalidValue;
    case ST_BF16EQ:
      if constexpr (L::REST == 0) return reduce_eq_t<L, __nv_bfloat16>(walls, kind, a, s);
      return cudaErrorInvalidValue;
    case ST_F32: return a.aa ? reduce_aa_t<L, float>(walls, kind, a, s) : reduce_t<L, float>(walls, kind, a, s);
    case ST_F16: return a.aa ? reduce_aa_t<L, __half>(walls, kind, a, s) : reduce_t<L, __half>(walls, kind, a, s);
    case ST_BF16:
      return a.aa ? reduce_aa_t<L, __nv_bfloat16>(walls, kind, a, s) : reduce_t<L, __nv_bfloat16>(walls, kind, a, s);
    case ST_F64: return a.aa ? reduce_aa_t<L, double>(walls, kind, a, s) : reduce_t<L, double>(walls, kind, a, s);
  }
  return cudaErrorInvalidValue;
}

template <class L>
cudaError_t mask_lattice(const int wall[3], int lid, const DevArgs &a, uint8_t *mask,
                         cudaStream_t s) {
  k_mask<L><<<node_grid(a), kBlockX, 0, s>>>(a, wall[0], wall[1], wall[2], lid, mask);
  return cudaGetLastError();
}

}  // namespace mdf

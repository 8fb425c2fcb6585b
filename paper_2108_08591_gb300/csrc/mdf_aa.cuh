// In-place AA-pattern update: one population buffer instead of two.
//
// The stream of Eq. 3-21 moves each post-collision population one link; the
// AA pattern (Bailey et al., 2009) folds that move into alternating access
// orders so that every update reads and writes the same locations:
//   even layout: slot i of node x holds f_i(x), the population arriving at x;
//   even update: read slot i at x, collide, write f*_i(x) to slot opp(i) at
//                x, which leaves the odd layout, in which f_i(y) sits in slot
//                opp(i) of node y - c_i;
//   odd update:  read f_i(y) from slot opp(i) at y - c_i, collide, write
//                f*_i(y) to slot i at y + c_i, which is slot i of the node it
//                arrives at: the even layout again.
// Each node reads and writes one fixed set of locations, read completely
// before any is written, so threads never touch each other's data.  Wall
// links (anti-halfway bounce-back) stay inside the node: in the odd layout
// a population that arrives at y through a wall is minus the one that
// left y, f*_opp(i)(y), found in slot i of y (plus the lid term); the odd
// update writes a population leaving through a wall, bounced, into slot
// opp(i) of its own node, so the even layout holds arrived populations
// only.  The per-node arithmetic is the pull kernel's (collide_node,
// write_fields), so both give the same bits.
//
// The buffer is read and written through one pointer with plain loads (no
// read-only cache path and no restrict qualifiers: the locations alias).
#pragma once

#include <type_traits>

#include "mdf_vec16p.cuh"  // packed 16-bit words (Words, set_bits, f2bits)

namespace mdf {

template <class T> struct CodecRW;
template <> struct CodecRW<float> {
  static __device__ __forceinline__ float load(const float *p) { return *p; }
};
template <> struct CodecRW<double> {
  static __device__ __forceinline__ double load(const double *p) { return *p; }
};
template <> struct CodecRW<__half> {
  static __device__ __forceinline__ float load(const __half *p) { return __half2float(*p); }
};
template <> struct CodecRW<__nv_bfloat16> {
  static __device__ __forceinline__ float load(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
};

// Padded index of x + c_i (periodic wrap; wall links never use it).
template <class L>
__device__ __forceinline__ long long push_dst(const DevArgs &A, int x, int y, int z, int i) {
  const int tx = wrap(x + L::c(i, 0), A.nx);
  const int ty = wrap(y + L::c(i, 1), A.ny);
  const int tz = L::D == 3 ? wrap(z + L::c(i, 2), A.nz) : z;
  return ((long long)tz * A.ny + ty) * A.px + tx;
}

// f_i arriving at node idx, for every i of one set, in the layout of the phase.
template <class L, class TS, bool ODD, bool WALLS>
__device__ __forceinline__ void aa_read_set(const DevArgs &A, const TS *base, int alpha, int x, int y,
                                            int z, long long idx, uint8_t m,
                                            typename ComputeOf<TS>::T (&g)[L::Q]) {
  using TC = typename ComputeOf<TS>::T;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    if (!ODD) {
      g[i] = CodecRW<TS>::load(base + (long long)i * A.plane + idx);
    } else if (WALLS && moving<L>(i) && ((m >> L::opp(i)) & 1)) {
      TC v = -TC(CodecRW<TS>::load(base + (long long)i * A.plane + idx));
      if (alpha >= 1 && i == L::opp(L::UP) && (m & 0x80u)) v += TC(2.0 * L::w(i) * A.lid_u[alpha - 1]);
      g[i] = v;
    } else {
      g[i] = CodecRW<TS>::load(base + (long long)L::opp(i) * A.plane + pull_src<L>(A, x, y, z, i));
    }
  }
}

// f*_i leaving node idx, for every i of one set, in the layout the phase leaves.
template <class L, class TS, bool ODD, bool WALLS>
__device__ __forceinline__ void aa_write_set(const DevArgs &A, TS *base, int alpha, int x, int y, int z,
                                             long long idx, uint8_t m,
                                             const typename ComputeOf<TS>::T (&g)[L::Q]) {
  using TC = typename ComputeOf<TS>::T;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    if (!ODD) {
      Codec<TS>::store(base + (long long)L::opp(i) * A.plane + idx, g[i]);
    } else if (WALLS && moving<L>(i) && ((m >> i) & 1)) {
      // bounced: arrives back at this node as f_opp(i)
      TC v = -g[i];
      if (alpha >= 1 && i == L::UP && (m & 0x80u)) v += TC(2.0 * L::w(i) * A.lid_u[alpha - 1]);
      Codec<TS>::store(base + (long long)L::opp(i) * A.plane + idx, v);
    } else {
      Codec<TS>::store(base + (long long)i * A.plane + push_dst<L>(A, x, y, z, i), g[i]);
    }
  }
}

template <class L, class TS, bool ODD, int MODE, bool WALLS>
__global__ void __launch_bounds__(kMaxBlock) k_update_aa(const DevArgs A) {
  using TC = typename ComputeOf<TS>::T;
  constexpr int D = L::D, Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= A.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long idx = ((long long)z * A.ny + y) * A.px + x;
  const uint8_t m = WALLS ? A.mask[idx] : uint8_t(0);
  TS *f = static_cast<TS *>(A.fout);  // == A.fin
  const int a1 = A.with_rho;

  TC g[D][Q], h[Q];
#pragma unroll
  for (int al = 1; al <= D; ++al)
    aa_read_set<L, TS, ODD, WALLS>(A, f + (long long)(a1 + al - 1) * Q * A.plane, al, x, y, z, idx, m,
                                   g[al - 1]);
  if (A.with_rho) aa_read_set<L, TS, ODD, WALLS>(A, f, 0, x, y, z, idx, m, h);
  else
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = TC(0);

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

#pragma unroll
  for (int a = 0; a < D; ++a)
    aa_write_set<L, TS, ODD, WALLS>(A, f + (long long)(a1 + a) * Q * A.plane, a + 1, x, y, z, idx, m, g[a]);
  if (A.with_rho) aa_write_set<L, TS, ODD, WALLS>(A, f, 0, x, y, z, idx, m, h);
}

// ---------------------------------------------------------------------------
// Vector AA update: VX consecutive x-nodes per thread (plain updates).  The
// even phase touches the thread's own VX nodes only, with one vector access
// per slot.  The odd phase pulls and pushes along x: a slot's VX values
// shift by one node, the end value crossing to the neighbouring lane by a
// warp shuffle; at a warp or row edge that value is loaded or stored with
// one scalar access by the thread owning the node, so every location is
// still read and written by one thread only.  A wall link (only the row's
// end nodes along x; whole rows along y and z) takes the per-node path.
// ---------------------------------------------------------------------------
template <class TS, int VX> struct VecRW;  // coherent vector loads (the buffer is written too)
template <int VX> struct VecRW<float, VX> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[VX]) {
    if constexpr (VX == 4) {
      const float4 t = *reinterpret_cast<const float4 *>(p);
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
      static_assert(VX == 2, "FP32 vectors of 2 or 4");
      const float2 t = *reinterpret_cast<const float2 *>(p);
      v[0] = t.x; v[1] = t.y;
    }
  }
};
template <> struct VecRW<double, 2> {
  static __device__ __forceinline__ void load(const double *p, double (&v)[2]) {
    const double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = t.x; v[1] = t.y;
  }
};
template <class T16, int VX> struct VecRW16 {
  static_assert(VX == 4 || VX == 8, "16-bit vectors of 4 or 8");
  using Raw = typename std::conditional<VX == 4, uint2, uint4>::type;
  static __device__ __forceinline__ void load(const T16 *p, float (&v)[VX]) {
    const Raw r = *reinterpret_cast<const Raw *>(p);
    const unsigned *w = reinterpret_cast<const unsigned *>(&r);
#pragma unroll
    for (int k = 0; k < VX / 2; ++k) {
      const float2 f = word_to_f2<T16>(w[k]);
      v[2 * k] = f.x;
      v[2 * k + 1] = f.y;
    }
  }
};
template <int VX> struct VecRW<__half, VX> : VecRW16<__half, VX> {};
template <int VX> struct VecRW<__nv_bfloat16, VX> : VecRW16<__nv_bfloat16, VX> {};

// Source row of the pull along c_i (the node's own row for x and the rest).
template <class L>
__device__ __forceinline__ int source_row(const VecRows &R, int i) {
  return L::c(i, 1) == 1 ? R.row_ym : L::c(i, 1) == -1 ? R.row_yp
       : L::c(i, 2) == 1 ? R.row_zm : L::c(i, 2) == -1 ? R.row_zp : R.row0;
}

// The VX nodes' arriving populations of every set, in the layout of the
// phase: every load of the thread is issued first (the odd phase's x-shifted
// values then cross lanes by shuffles), as in the pull kernels.  g: the d
// velocity sets, h: the continuity set (zero without it).
template <class L, class TS, int VX, bool ODD, bool WALLS>
__device__ __forceinline__ void aa_read_all_vec(const DevArgs &A, const TS *f, const VecRows &R,
                                                const uint8_t (&m)[VX],
                                                typename ComputeOf<TS>::T (&g)[L::D][L::Q][VX],
                                                typename ComputeOf<TS>::T (&h)[L::Q][VX]) {
  using TC = typename ComputeOf<TS>::T;
  constexpr int D = L::D, Q = L::Q;
  const int a1 = A.with_rho;
  auto set_base = [&](int s) { return f + (long long)(s < D ? a1 + s : 0) * Q * A.plane; };
  if constexpr (sizeof(TS) == 2) {
    using PK = Packed16<TS, VX>;
    using W = typename PK::W;
    W wv[D + 1][Q];
    unsigned edge[D + 1][2];
#pragma unroll
    for (int s = 0; s <= D; ++s) {
      if (s == D && !A.with_rho) break;
      const TS *base = set_base(s);
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const TS *p = base + (long long)(ODD ? L::opp(i) : i) * A.plane;
        wv[s][i] = *reinterpret_cast<const W *>(p + (ODD ? source_row<L>(R, i) : R.row0) + R.x0);
        if (ODD && L::c(i, 0) == 1)
          edge[s][0] = R.ledge ? *reinterpret_cast<const unsigned short *>(p + R.row0 + R.xl) : 0u;
        if (ODD && L::c(i, 0) == -1)
          edge[s][1] = R.redge ? *reinterpret_cast<const unsigned short *>(p + R.row0 + R.xr) : 0u;
      }
    }
#pragma unroll
    for (int s = 0; s <= D; ++s) {
      if (s == D && !A.with_rho) break;
      float(&v)[Q][VX] = s < D ? g[s < D ? s : 0] : h;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const W w = wv[s][i];
        if (ODD && L::c(i, 0) == 1) {  // from x - 1
          unsigned nb = __shfl_up_sync(0xffffffffu, PK::last_word(w), 1);
          nb = R.ledge ? edge[s][0] : (nb >> 16);
          v[i][0] = bits_to_float<TS>(nb);
#pragma unroll
          for (int j = 1; j < VX; ++j) v[i][j] = bits_to_float<TS>(PK::bits(w, j - 1));
        } else if (ODD && L::c(i, 0) == -1) {  // from x + 1
          unsigned nb = __shfl_down_sync(0xffffffffu, PK::first_word(w), 1);
          nb = R.redge ? edge[s][1] : (nb & 0xffffu);
#pragma unroll
          for (int j = 0; j < VX - 1; ++j) v[i][j] = bits_to_float<TS>(PK::bits(w, j + 1));
          v[i][VX - 1] = bits_to_float<TS>(nb);
        } else {
#pragma unroll
          for (int j = 0; j < VX; ++j) v[i][j] = bits_to_float<TS>(PK::bits(w, j));
        }
      }
    }
  } else {
    TC edge[D + 1][2];
#pragma unroll
    for (int s = 0; s <= D; ++s) {
      if (s == D && !A.with_rho) break;
      const TS *base = set_base(s);
      TC(&v)[Q][VX] = s < D ? g[s < D ? s : 0] : h;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const TS *p = base + (long long)(ODD ? L::opp(i) : i) * A.plane;
        VecRW<TS, VX>::load(p + (ODD ? source_row<L>(R, i) : R.row0) + R.x0, v[i]);
        if (ODD && L::c(i, 0) == 1) edge[s][0] = R.ledge ? CodecRW<TS>::load(p + R.row0 + R.xl) : TC(0);
        if (ODD && L::c(i, 0) == -1) edge[s][1] = R.redge ? CodecRW<TS>::load(p + R.row0 + R.xr) : TC(0);
      }
    }
    if (ODD) {
#pragma unroll
      for (int s = 0; s <= D; ++s) {
        if (s == D && !A.with_rho) break;
        TC(&v)[Q][VX] = s < D ? g[s < D ? s : 0] : h;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (L::c(i, 0) == 1) {  // from x - 1: shift up by one node
            TC pv = __shfl_up_sync(0xffffffffu, v[i][VX - 1], 1);
            if (R.ledge) pv = edge[s][0];
#pragma unroll
            for (int j = VX - 1; j > 0; --j) v[i][j] = v[i][j - 1];
            v[i][0] = pv;
          } else if (L::c(i, 0) == -1) {  // from x + 1: shift down by one node
            TC nv = __shfl_down_sync(0xffffffffu, v[i][0], 1);
            if (R.redge) nv = edge[s][1];
#pragma unroll
            for (int j = 0; j < VX - 1; ++j) v[i][j] = v[i][j + 1];
            v[i][VX - 1] = nv;
          }
        }
      }
    }
  }
  if (!A.with_rho)
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
      for (int j = 0; j < VX; ++j) h[i][j] = TC(0);
  if (ODD && WALLS) {  // arrived through a wall: minus the node's own leaving value
#pragma unroll
    for (int s = 0; s <= D; ++s) {
      if (s == D && !A.with_rho) break;
      const int alpha = s < D ? s + 1 : 0;
      const TS *base = set_base(s);
      TC(&v)[Q][VX] = s < D ? g[s < D ? s : 0] : h;
#pragma unroll
      for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < VX; ++j)
          if (moving<L>(i) && ((m[j] >> L::opp(i)) & 1)) {
            TC w = -TC(CodecRW<TS>::load(base + (long long)i * A.plane + R.row0 + R.x0 + j));
            if (alpha >= 1 && i == L::opp(L::UP) && (m[j] & 0x80u)) w += TC(2.0 * L::w(i) * A.lid_u[alpha - 1]);
            v[i][j] = w;
          }
    }
  }
}

// Every lane runs the shuffles; a lane past the row end (`active` false)
// stores nothing.
template <class L, class TS, int VX, bool ODD, bool WALLS>
__device__ __forceinline__ void aa_write_vec(const DevArgs &A, TS *base, int alpha, const VecRows &R,
                                             const uint8_t (&m)[VX], bool active,
                                             const typename ComputeOf<TS>::T (&v)[L::Q][VX]) {
  using TC = typename ComputeOf<TS>::T;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    if (!ODD) {
      if (active) VecIO<TS, VX>::store(base + (long long)L::opp(i) * A.plane + R.row0 + R.x0, v[i]);
      continue;
    }
    TS *p = base + (long long)i * A.plane;
    // nodes whose link along c_i leaves through a wall: bounced into slot opp(i)
    bool any_wall = false;
    if (WALLS && moving<L>(i))
#pragma unroll
      for (int j = 0; j < VX; ++j) any_wall |= ((m[j] >> i) & 1) != 0;
    auto bounce = [&](int j) {
      TC w = -v[i][j];
      if (alpha >= 1 && i == L::UP && (m[j] & 0x80u)) w += TC(2.0 * L::w(i) * A.lid_u[alpha - 1]);
      Codec<TS>::store(base + (long long)L::opp(i) * A.plane + R.row0 + R.x0 + j, w);
    };
    if (L::c(i, 0) == 1) {  // to x + 1: position x0 + j holds node x0 + j - 1
      TC out[VX];
      out[0] = __shfl_up_sync(0xffffffffu, v[i][VX - 1], 1);
#pragma unroll
      for (int j = 1; j < VX; ++j) out[j] = v[i][j - 1];
      if (!active) continue;
      if (!R.ledge) {
        VecIO<TS, VX>::store(p + R.row0 + R.x0, out);
      } else {
#pragma unroll
        for (int j = 1; j < VX; ++j) Codec<TS>::store(p + R.row0 + R.x0 + j, out[j]);
      }
      if (R.redge) {  // node x0 + VX - 1 feeds the next thread's first position
        if (any_wall && ((m[VX - 1] >> i) & 1)) bounce(VX - 1);
        else Codec<TS>::store(p + R.row0 + R.xr, v[i][VX - 1]);
      }
    } else if (L::c(i, 0) == -1) {  // to x - 1: position x0 + j holds node x0 + j + 1
      TC out[VX];
#pragma unroll
      for (int j = 0; j < VX - 1; ++j) out[j] = v[i][j + 1];
      out[VX - 1] = __shfl_down_sync(0xffffffffu, v[i][0], 1);
      if (!active) continue;
      if (!R.redge) {
        VecIO<TS, VX>::store(p + R.row0 + R.x0, out);
      } else {
#pragma unroll
        for (int j = 0; j < VX - 1; ++j) Codec<TS>::store(p + R.row0 + R.x0 + j, out[j]);
      }
      if (R.ledge) {  // node x0 feeds the previous thread's last position
        if (any_wall && ((m[0] >> i) & 1)) bounce(0);
        else Codec<TS>::store(p + R.row0 + R.xl, v[i][0]);
      }
    } else {
      if (!active) continue;
      const int r = L::c(i, 1) == 1 ? R.row_yp : L::c(i, 1) == -1 ? R.row_ym
                  : L::c(i, 2) == 1 ? R.row_zp : L::c(i, 2) == -1 ? R.row_zm : R.row0;
      if (!any_wall) {
        VecIO<TS, VX>::store(p + r + R.x0, v[i]);
      } else {
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          if ((m[j] >> i) & 1) bounce(j);
          else Codec<TS>::store(p + r + R.x0 + j, v[i][j]);
        }
      }
    }
  }
}

template <class L, class TS, int VX, bool ODD, bool WALLS, bool S2>
__global__ void __launch_bounds__(kMaxBlock) k_update_aa_vec(const DevArgs A) {
  using TC = typename ComputeOf<TS>::T;
  constexpr int D = L::D, Q = L::Q;
  const int lane = threadIdx.x & 31;
  int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * VX;
  const bool active = x0 < A.nx;
  if (!active) x0 = A.nx - VX;  // stays in the shuffles, stores nothing
  const int y = blockIdx.y, z = blockIdx.z;
  const int row0 = (z * A.ny + y) * A.px;
  const int row_ym = (z * A.ny + wrap(y - 1, A.ny)) * A.px;
  const int row_yp = (z * A.ny + wrap(y + 1, A.ny)) * A.px;
  const int row_zm = D == 3 ? (wrap(z - 1, A.nz) * A.ny + y) * A.px : row0;
  const int row_zp = D == 3 ? (wrap(z + 1, A.nz) * A.ny + y) * A.px : row0;
  const bool ledge = lane == 0 || x0 == 0;
  const bool redge = lane == 31 || x0 + VX >= A.nx;
  const int xl = x0 == 0 ? A.nx - 1 : x0 - 1;
  const int xr = x0 + VX >= A.nx ? 0 : x0 + VX;
  TS *f = static_cast<TS *>(A.fout);  // == A.fin
  const int a1 = A.with_rho;
  uint8_t m[VX];
#pragma unroll
  for (int j = 0; j < VX; ++j) m[j] = WALLS ? A.mask[row0 + x0 + j] : uint8_t(0);

  const VecRows R{row0, row_ym, row_yp, row_zm, row_zp, x0, xl, xr, ledge, redge};
  TC g[D][Q][VX], h[Q][VX];
  aa_read_all_vec<L, TS, VX, ODD, WALLS>(A, f, R, m, g, h);

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
  const int tstep = DZ ? launch_step(A) : 0;
  const long long n0 = ((long long)z * A.ny + y) * A.nx + x0;
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
    const uint32_t key = DZ ? node_key(A.key_base + n0 + j, tstep) : 0u;
    collide_node<L, TC, S2, DZ>(gn, hn, A.with_rho != 0, Fn, s1, s2, M, key);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
#pragma unroll
      for (int a = 0; a < D; ++a) g[a][i][j] = gn[a][i];
      h[i][j] = hn[i];
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a)
    aa_write_vec<L, TS, VX, ODD, WALLS>(A, f + (long long)(a1 + a) * Q * A.plane, a + 1, R, m, active, g[a]);
  if (A.with_rho) aa_write_vec<L, TS, VX, ODD, WALLS>(A, f, 0, R, m, active, h);
}

// ---------------------------------------------------------------------------
// 16-bit vector AA update with the populations packed in registers (see
// k_update_vec16p): words are loaded (and, in the odd phase, realigned along
// x) first, every node is decoded, collided and encoded back into its
// element, and the words are stored in the layout the phase leaves.  A
// population leaving through a wall is bounced in FP32 before it is encoded
// (as the one-node-per-thread kernel does) and its element is stored in the
// node's own slot.
// ---------------------------------------------------------------------------
template <class TS> __device__ __forceinline__ void st_bits16(TS *p, unsigned b) {
  *reinterpret_cast<unsigned short *>(p) = (unsigned short)b;
}

template <class L, class TS, int VX, bool ODD, bool WALLS, bool S2>
__global__ void __launch_bounds__(kMaxBlock) k_update_aa_vec16p(const DevArgs A) {
  constexpr int D = L::D, Q = L::Q;
  using PK = Packed16<TS, VX>;
  using W = typename Words<VX>::W;
  const int lane = threadIdx.x & 31;
  int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * VX;
  const bool active = x0 < A.nx;
  if (!active) x0 = A.nx - VX;  // stays in the shuffles, stores nothing
  const int y = blockIdx.y, z = blockIdx.z;
  const int row0 = (z * A.ny + y) * A.px;
  const int row_ym = (z * A.ny + wrap(y - 1, A.ny)) * A.px;
  const int row_yp = (z * A.ny + wrap(y + 1, A.ny)) * A.px;
  const int row_zm = D == 3 ? (wrap(z - 1, A.nz) * A.ny + y) * A.px : row0;
  const int row_zp = D == 3 ? (wrap(z + 1, A.nz) * A.ny + y) * A.px : row0;
  const bool ledge = lane == 0 || x0 == 0;
  const bool redge = lane == 31 || x0 + VX >= A.nx;
  const int xl = x0 == 0 ? A.nx - 1 : x0 - 1;
  const int xr = x0 + VX >= A.nx ? 0 : x0 + VX;
  const VecRows R{row0, row_ym, row_yp, row_zm, row_zp, x0, xl, xr, ledge, redge};
  TS *f = static_cast<TS *>(A.fout);  // == A.fin
  const int a1 = A.with_rho;
  uint8_t m[VX];
#pragma unroll
  for (int j = 0; j < VX; ++j) m[j] = WALLS ? A.mask[row0 + x0 + j] : uint8_t(0);
  auto set_base = [&](int s) { return f + (long long)(s < D ? a1 + s : 0) * Q * A.plane; };

  W wv[D + 1][Q];
  unsigned edge[D + 1][2];
#pragma unroll
  for (int s = 0; s <= D; ++s) {
    if (s == D && !A.with_rho) break;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const TS *p = set_base(s) + (long long)(ODD ? L::opp(i) : i) * A.plane;
      wv[s][i] = *reinterpret_cast<const W *>(p + (ODD ? source_row<L>(R, i) : row0) + x0);
      if (ODD && L::c(i, 0) == 1) edge[s][0] = ledge ? *reinterpret_cast<const unsigned short *>(p + row0 + xl) : 0u;
      if (ODD && L::c(i, 0) == -1) edge[s][1] = redge ? *reinterpret_cast<const unsigned short *>(p + row0 + xr) : 0u;
    }
  }
  if (ODD) {
#pragma unroll
    for (int s = 0; s <= D; ++s) {
      if (s == D && !A.with_rho) break;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (L::c(i, 0) == 1) {
          unsigned nb = __shfl_up_sync(0xffffffffu, PK::last_word(wv[s][i]), 1) >> 16;
          if (ledge) nb = edge[s][0];
          wv[s][i] = Words<VX>::up(wv[s][i], nb);
        } else if (L::c(i, 0) == -1) {
          unsigned nb = __shfl_down_sync(0xffffffffu, PK::first_word(wv[s][i]), 1) & 0xffffu;
          if (redge) nb = edge[s][1];
          wv[s][i] = Words<VX>::down(wv[s][i], nb);
        }
      }
    }
  }

  float F[D][VX];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (A.force) {
      VecIO<float, VX>::load(static_cast<const float *>(A.force) + a * A.plane + row0 + x0, F[a]);
    } else {
#pragma unroll
      for (int j = 0; j < VX; ++j) F[a][j] = 0.f;
    }
  }
  const float s1 = A.s1f, s2 = A.s2f;
#pragma unroll
  for (int j = 0; j < VX; ++j) {
    float gn[D][Q], hn[Q], Fn[D];
#pragma unroll
    for (int s = 0; s <= D; ++s) {
      if (s == D && !A.with_rho) break;
      const int alpha = s < D ? s + 1 : 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        float v = bits_to_float<TS>(PK::bits(wv[s][i], j));
        if (ODD && WALLS && moving<L>(i) && ((m[j] >> L::opp(i)) & 1)) {  // arrived through a wall
          v = -CodecRW<TS>::load(set_base(s) + (long long)i * A.plane + row0 + x0 + j);
          if (alpha >= 1 && i == L::opp(L::UP) && (m[j] & 0x80u)) v += float(2.0 * L::w(i) * A.lid_u[alpha - 1]);
        }
        if (s < D) gn[s < D ? s : 0][i] = v;
        else hn[i] = v;
      }
    }
    if (!A.with_rho)
#pragma unroll
      for (int i = 0; i < Q; ++i) hn[i] = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) Fn[a] = F[a][j];
    float M[D + 2];
    collide_node<L, float, S2>(gn, hn, A.with_rho != 0, Fn, s1, s2, M);
#pragma unroll
    for (int s = 0; s <= D; ++s) {
      if (s == D && !A.with_rho) break;
      const int alpha = s < D ? s + 1 : 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        float v = s < D ? gn[s < D ? s : 0][i] : hn[i];
        if (ODD && WALLS && moving<L>(i) && ((m[j] >> i) & 1)) {  // leaves through a wall: bounced
          v = -v;
          if (alpha >= 1 && i == L::UP && (m[j] & 0x80u)) v += float(2.0 * L::w(i) * A.lid_u[alpha - 1]);
        }
        set_bits<VX>(wv[s][i], j, f2bits<TS>(v));
      }
    }
  }

  // stores (every lane runs the shuffles; lanes past the row end store nothing)
#pragma unroll
  for (int s = 0; s <= D; ++s) {
    if (s == D && !A.with_rho) break;
    TS *base = set_base(s);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const W w = wv[s][i];
      if (!ODD) {
        if (active) *reinterpret_cast<W *>(base + (long long)L::opp(i) * A.plane + row0 + x0) = w;
        continue;
      }
      TS *p = base + (long long)i * A.plane;
      TS *own_opp = base + (long long)L::opp(i) * A.plane + row0 + x0;  // bounced elements
      auto leaves_wall = [&](int j) { return WALLS && moving<L>(i) && ((m[j] >> i) & 1); };
      if (L::c(i, 0) == 1) {  // to x + 1
        const unsigned nb = __shfl_up_sync(0xffffffffu, PK::last_word(w), 1) >> 16;
        if (!active) continue;
        const W out = Words<VX>::up(w, nb);
        if (!ledge) {
          *reinterpret_cast<W *>(p + row0 + x0) = out;
        } else {
#pragma unroll
          for (int j = 1; j < VX; ++j) st_bits16(p + row0 + x0 + j, PK::bits(out, j));
        }
        if (redge) {
          if (leaves_wall(VX - 1)) st_bits16(own_opp + VX - 1, PK::bits(w, VX - 1));
          else st_bits16(p + row0 + xr, PK::bits(w, VX - 1));
        }
      } else if (L::c(i, 0) == -1) {  // to x - 1
        const unsigned nb = __shfl_down_sync(0xffffffffu, PK::first_word(w), 1) & 0xffffu;
        if (!active) continue;
        const W out = Words<VX>::down(w, nb);
        if (!redge) {
          *reinterpret_cast<W *>(p + row0 + x0) = out;
        } else {
#pragma unroll
          for (int j = 0; j < VX - 1; ++j) st_bits16(p + row0 + x0 + j, PK::bits(out, j));
        }
        if (ledge) {
          if (leaves_wall(0)) st_bits16(own_opp, PK::bits(w, 0));
          else st_bits16(p + row0 + xl, PK::bits(w, 0));
        }
      } else {
        if (!active) continue;
        const int r = L::c(i, 1) == 1 ? row_yp : L::c(i, 1) == -1 ? row_ym
                    : L::c(i, 2) == 1 ? row_zp : L::c(i, 2) == -1 ? row_zm : row0;
        bool any_wall = false;
#pragma unroll
        for (int j = 0; j < VX; ++j) any_wall |= leaves_wall(j);
        if (!any_wall) {
          *reinterpret_cast<W *>(p + r + x0) = w;
        } else {
#pragma unroll
          for (int j = 0; j < VX; ++j) {
            if (leaves_wall(j)) st_bits16(own_opp + j, PK::bits(w, j));
            else st_bits16(p + r + x0 + j, PK::bits(w, j));
          }
        }
      }
    }
  }
}

// FP64 sums and residual over the in-place buffer (see k_reduce).
template <class L, class TS, bool ODD, bool WALLS, int KIND>
__global__ void __launch_bounds__(kReduceThreads) k_reduce_aa(const DevArgs A) {
  using TC = typename ComputeOf<TS>::T;
  constexpr int D = L::D, Q = L::Q;
  const long long N = (long long)A.nx * A.ny * A.nz;
  const TS *f = static_cast<const TS *>(A.fin);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  bool bad = false;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % A.nx);
    const int y = (int)((n / A.nx) % A.ny);
    const int z = (int)(n / ((long long)A.nx * A.ny));
    const long long idx = ((long long)z * A.ny + y) * A.px + x;
    const uint8_t m = WALLS ? A.mask[idx] : uint8_t(0);
    const int nsets = D + A.with_rho;
#pragma unroll
    for (int a = 0; a < D + 1; ++a) {
      if (a >= nsets) break;
      const int alpha = a + 1 - A.with_rho;
      TC g[Q];
      aa_read_set<L, TS, ODD, WALLS>(A, f + (long long)a * Q * A.plane, alpha, x, y, z, idx, m, g);
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) s += (double)g[i];
      if (alpha == 0) s += 1.0;
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

// Host dispatch: A.aa = 1 (even phase) or 2 (odd phase); one node per thread.
template <class L, class TS, bool ODD>
cudaError_t update_aa_phase(int mode, bool walls, const DevArgs &a, cudaStream_t s) {
  const int bx = a.block;
  const dim3 grid((unsigned)((a.nx + bx - 1) / bx), (unsigned)a.ny, (unsigned)a.nz), block(bx);
  if (walls) {
    if (mode == MODE_STEP) k_update_aa<L, TS, ODD, MODE_STEP, true><<<grid, block, 0, s>>>(a);
    else if (mode == MODE_STEP_FIELDS) k_update_aa<L, TS, ODD, MODE_STEP_FIELDS, true><<<grid, block, 0, s>>>(a);
    else k_update_aa<L, TS, ODD, MODE_FIELDS, true><<<grid, block, 0, s>>>(a);
  } else {
    if (mode == MODE_STEP) k_update_aa<L, TS, ODD, MODE_STEP, false><<<grid, block, 0, s>>>(a);
    else if (mode == MODE_STEP_FIELDS) k_update_aa<L, TS, ODD, MODE_STEP_FIELDS, false><<<grid, block, 0, s>>>(a);
    else k_update_aa<L, TS, ODD, MODE_FIELDS, false><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <class L, class TS, int VX, bool ODD>
cudaError_t update_aa_vec_phase(bool walls, const DevArgs &a, cudaStream_t s) {
  const int bx = a.block;
  const int threads = a.nx / VX;
  const dim3 grid((unsigned)((threads + bx - 1) / bx), (unsigned)a.ny, (unsigned)a.nz), block(bx);
  if constexpr (sizeof(TS) == 2) {  // 16-bit: populations kept packed in registers
    if (a.scheme2) {
      if (walls) k_update_aa_vec16p<L, TS, VX, ODD, true, true><<<grid, block, 0, s>>>(a);
      else k_update_aa_vec16p<L, TS, VX, ODD, false, true><<<grid, block, 0, s>>>(a);
    } else {
      if (walls) k_update_aa_vec16p<L, TS, VX, ODD, true, false><<<grid, block, 0, s>>>(a);
      else k_update_aa_vec16p<L, TS, VX, ODD, false, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
  }
  if (a.scheme2) {
    if (walls) k_update_aa_vec<L, TS, VX, ODD, true, true><<<grid, block, 0, s>>>(a);
    else k_update_aa_vec<L, TS, VX, ODD, false, true><<<grid, block, 0, s>>>(a);
  } else {
    if (walls) k_update_aa_vec<L, TS, VX, ODD, true, false><<<grid, block, 0, s>>>(a);
    else k_update_aa_vec<L, TS, VX, ODD, false, false><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <class L, class TS, int VX>
cudaError_t update_aa_vec(bool walls, const DevArgs &a, cudaStream_t s) {
  return a.aa == 2 ? update_aa_vec_phase<L, TS, VX, true>(walls, a, s)
                   : update_aa_vec_phase<L, TS, VX, false>(walls, a, s);
}

// Plain updates with a width built for the storage type that divides nx
// run the vector kernel (FP32 2 or 4, 16-bit 4 or 8, FP64 2; in 3D, where
// the wider ones spill registers, FP32 2 and 16-bit 4); everything else,
// and every field-writing update, runs one node per thread.
template <class L, class TS>
cudaError_t update_aa_t(int mode, bool walls, const DevArgs &a, cudaStream_t s) {
  const bool ok = mode == MODE_STEP && a.vx > 1 && a.nx % a.vx == 0 && a.plane < (1LL << 31) - 64;
  if (ok) {
    if constexpr (sizeof(TS) == 4) {
      if constexpr (L::D == 2) {
        if (a.vx == 4) return update_aa_vec<L, TS, 4>(walls, a, s);
      }
      if (a.vx == 2) return update_aa_vec<L, TS, 2>(walls, a, s);
    } else if constexpr (sizeof(TS) == 2) {
      if constexpr (L::D == 2) {
        if (a.vx == 8) return update_aa_vec<L, TS, 8>(walls, a, s);
      }
      if (a.vx == 4) return update_aa_vec<L, TS, 4>(walls, a, s);
    } else {
      if (a.vx == 2) return update_aa_vec<L, TS, 2>(walls, a, s);
    }
  }
  return a.aa == 2 ? update_aa_phase<L, TS, true>(mode, walls, a, s)
                   : update_aa_phase<L, TS, false>(mode, walls, a, s);
}

template <class L, class TS, bool ODD>
cudaError_t reduce_aa_phase(bool walls, int kind, const DevArgs &a, cudaStream_t s) {
  const int nb = kReduceBlocks;
  if (kind == RED_SUMS) {
    if (walls) k_reduce_aa<L, TS, ODD, true, RED_SUMS><<<nb, kReduceThreads, 0, s>>>(a);
    else k_reduce_aa<L, TS, ODD, false, RED_SUMS><<<nb, kReduceThreads, 0, s>>>(a);
  } else {
    if (walls) k_reduce_aa<L, TS, ODD, true, RED_RESIDUAL><<<nb, kReduceThreads, 0, s>>>(a);
    else k_reduce_aa<L, TS, ODD, false, RED_RESIDUAL><<<nb, kReduceThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <class L, class TS>
cudaError_t reduce_aa_t(bool walls, int kind, const DevArgs &a, cudaStream_t s) {
  return a.aa == 2 ? reduce_aa_phase<L, TS, true>(walls, kind, a, s)
                   : reduce_aa_phase<L, TS, false>(walls, kind, a, s);
}

}  // namespace mdf

// Equilibrium-shifted 16-bit population storage (MDF_F16EQ, MDF_BF16EQ).
//
// Rest-shifted 16-bit storage keeps populations of size ~U in 11 (FP16) or 8
// (BF16) significant bits, which resolves u but not the pressure
// fluctuation (~U^2) nor the first moment of f^ne (Eq. 3-16), both far below
// one ulp of the populations.  This codec stores instead, per node x and set,
// the post-collision non-equilibrium part
//     s_i(x) = SCALE * ( g*_i(x) - g^eq_i(M(x)) )
// in 16 bits, and the node's moments M(x) = (u_1..u_d, P', rho') in FP32,
// where g = f - f_rest is the rest-shifted population and M(x) are the
// moments the node's collision used.  A pull rebuilds
//     g_i(y) = s_i(x) / SCALE + g^eq_i(M(x)),  x = y - c_i,
// with the same FP32 expression the writer used, so the only loss is the
// 16-bit rounding of s, whose size is that of f^ne.  The collision itself
// (Eq. 3-21) is unchanged.  Moments are double-buffered with the
// populations.  Bytes per node update: 2*2*q*nsets + 2*4*K with
// K = d + 1 + with_rho moments.
#pragma once

namespace mdf {

// Memory layout.  x is cut into tiles of 64 nodes (the x pitch is a
// multiple of 64).  For each row (z, y) and tile, the nk arrays of the
// tile (populations: set-major, direction within set; moments: slot by
// slot) lie one after the other, 64 elements each:
//     element k of node x in row r:  ((r px/64 + x/64) nk + k) 64 + x mod 64.
// A thread's nodes share one tile, so every array it touches sits at a
// compile-time offset (k 64 elements) from a few per-row pointers, and a
// warp's 64 nodes of one array are one contiguous 128-byte (16-bit) or
// 256-byte (FP32) span.
constexpr int kEqTile = 64;
__host__ __device__ __forceinline__ long long eq_off(int px, long long row, int x, int nk) {
  return ((row * (px / kEqTile) + (x / kEqTile)) * (long long)nk) * kEqTile + (x & (kEqTile - 1));
}

// FP16 keeps |s| in its normal range (6e-5 .. 65504) for non-equilibrium
// parts between ~4e-9 and 4; BF16 has the FP32 exponent range.
template <class TS> struct EqScale;
template <> struct EqScale<__half> { static constexpr float s = 16384.f, inv = 1.f / 16384.f; };
template <> struct EqScale<__nv_bfloat16> { static constexpr float s = 1.f, inv = 1.f; };

// g^eq_i of set alpha (rest-shifted, Eq. 2-4) from the moments
// M = (u_1..u_d, P', rho'): alpha >= 1: w_i [u_a + (c_i.u u_a + c_{i,a} P')/c_s^2];
// alpha = 0: w_i [rho' + (1 + rho') c_i.u / c_s^2].
template <class L>
__device__ __forceinline__ float geq_m(int alpha, int i, const float (&M)[L::D + 2]) {
  float cu = 0.f;
#pragma unroll
  for (int b = 0; b < L::D; ++b) {
    if (L::c(i, b) > 0) cu += M[b];
    if (L::c(i, b) < 0) cu -= M[b];
  }
  const float wi = float(L::w(i)), ics2 = float(1.0 / L::CS2);
  if (alpha == 0) return wi * (M[L::D + 1] + cu * (1.f + M[L::D + 1]) * ics2);
  const float ua = M[alpha - 1];
  const float cP = L::c(i, alpha - 1) > 0 ? M[L::D] : (L::c(i, alpha - 1) < 0 ? -M[L::D] : 0.f);
  return wi * (ua + (cu * ua + cP) * ics2);
}

// The KM moment slots of VX nodes from a tile pointer (slots >= K read 0).
template <int KM, int VX>
__device__ __forceinline__ void load_moments(const float *mt, int K, float (&M)[KM][VX]) {
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    if (k < K) {
      float v[VX];
      VecIO<float, VX>::load(mt + k * kEqTile, v);
#pragma unroll
      for (int j = 0; j < VX; ++j) M[k][j] = v[j];
    } else {
#pragma unroll
      for (int j = 0; j < VX; ++j) M[k][j] = 0.f;
    }
  }
}

// Moments of the source of element j along direction i (see VecRows).
template <class L, int VX>
__device__ __forceinline__ void source_moments(int i, int j, const float (&Mo)[L::D + 2][VX],
                                               const float (&Mym)[L::D + 2][VX],
                                               const float (&Myp)[L::D + 2][VX],
                                               const float (&Mzm)[L::D + 2][VX],
                                               const float (&Mzp)[L::D + 2][VX],
                                               const float (&Mxl)[L::D + 2],
                                               const float (&Mxr)[L::D + 2],
                                               float (&Ms)[L::D + 2]) {
#pragma unroll
  for (int k = 0; k < L::D + 2; ++k) {
    float v;
    if (L::c(i, 0) == 1) v = j == 0 ? Mxl[k] : Mo[k][j - 1];
    else if (L::c(i, 0) == -1) v = j == VX - 1 ? Mxr[k] : Mo[k][j + 1];
    else if (L::c(i, 1) == 1) v = Mym[k][j];
    else if (L::c(i, 1) == -1) v = Myp[k][j];
    else if (L::c(i, 2) == 1) v = Mzm[k][j];
    else if (L::c(i, 2) == -1) v = Mzp[k][j];
    else v = Mo[k][j];
    Ms[k] = v;
  }
}

// Moment slots: u_1..u_d, P', then rho' (only stored when with_rho).
__device__ __forceinline__ int moment_slots(int D, int with_rho) { return D + 1 + with_rho; }

// ---------------------------------------------------------------------------
// Update kernel.  Arithmetic is carried in "scaled" units G = SCALE * g and
// per lane group: one float (VX = 1) or an FP32 pair (VX >= 2) handled by
// the f32x2 instructions, whose lanes round exactly like the scalar ones, so
// every VX gives the same bits.  Every operation is an explicit add / mul /
// fma, independent of compiler contraction.
//
// Pull (decode): G_i(y) = raw_i(x) + SCALE w_i e_i(M(x)), x = y - c_i, with
// g^eq_i = w_i e_i (Eq. 2-4, rest-shifted): for a velocity set alpha and a
// moving direction c_i = sg e_b, e = u_alpha (1 + sg u_b / c_s^2) +
// [alpha = b] sg P' / c_s^2; for the continuity set e = rho' + sg u_b (1 +
// rho') / c_s^2; for the rest direction e = u_alpha (rho').
//
// Collide (Eq. 3-21) and encode in one: the stored part is
//   s = SCALE (f* - f^eq(M)) = M^-1 (I - S) (m - m^eq) + SCALE w F,
// since f - f^eq = M^-1 (m - m^eq) and the conserved moment m_0 equals its
// equilibrium.  With M's orthogonal rows, M^-1 = M^T diag(1 / |row k|^2),
// so each stored value is a short signed sum of the moment deviations E_k =
// m_k - m_k^eq scaled by (1 - s_k) / |row k|^2.
// ---------------------------------------------------------------------------
template <int VX> struct Lanes {
  using T = float2;
  static constexpr int N = VX / 2, W = 2;
};
template <> struct Lanes<1> {
  using T = float;
  static constexpr int N = 1, W = 1;
};

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

#define MDF_F32X2_BINARY(name, op)                                                              \
  __device__ __forceinline__ float2 name(float2 a, float2 b) {                                  \
    float2 r;                                                                                   \
    asm("{\n .reg .b64 a, b, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n " op           \
        " d, a, b;\n mov.b64 {%0, %1}, d;\n}\n"                                                 \
        : "=f"(r.x), "=f"(r.y)                                                                  \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                              \
    return r;                                                                                   \
  }
MDF_F32X2_BINARY(vadd, "add.rn.f32x2")
MDF_F32X2_BINARY(vsub, "sub.rn.f32x2")
MDF_F32X2_BINARY(vmul, "mul.rn.f32x2")
#undef MDF_F32X2_BINARY
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n .reg .b64 a, b, c, d;\n mov.b64 a, {%2, %3};\n mov.b64 b, {%4, %5};\n"
      " mov.b64 c, {%6, %7};\n fma.rn.f32x2 d, a, b, c;\n mov.b64 {%0, %1}, d;\n}\n"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}

template <class T> __device__ __forceinline__ T splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 splat<float2>(float c) { return make_float2(c, c); }
__device__ __forceinline__ void to_lanes(float &t, const float *v) { t = v[0]; }
__device__ __forceinline__ void to_lanes(float2 &t, const float *v) { t = make_float2(v[0], v[1]); }
__device__ __forceinline__ void from_lanes(float *v, float t) { v[0] = t; }
__device__ __forceinline__ void from_lanes(float *v, float2 t) { v[0] = t.x; v[1] = t.y; }

// Moving direction i of lattice L: axis b and sign sg (sg = 0: rest).
template <class L> __host__ __device__ constexpr int dir_axis(int i) {
  return L::c(i, 0) != 0 ? 0 : L::c(i, 1) != 0 ? 1 : 2;
}
template <class L> __host__ __device__ constexpr int dir_sign(int i) {
  return L::c(i, 0) + L::c(i, 1) + (L::D == 3 ? L::c(i, 2) : 0);
}

// e_i of set alpha from source moments (u, P', rho') (see above).
template <class L, class T>
__device__ __forceinline__ T eq_inner(int alpha, int i, const T (&u)[L::D], T P, T r) {
  constexpr float ics2 = float(1.0 / L::CS2);
  if (i == 0) return alpha == 0 ? r : u[alpha - 1];
  const int b = dir_axis<L>(i);
  const float sc = dir_sign<L>(i) > 0 ? ics2 : -ics2;
  if (alpha == 0) return vfma(vmul(u[b], splat<T>(sc)), vadd(r, splat<T>(1.f)), r);
  const T t = vfma(u[b], splat<T>(sc), splat<T>(1.f));
  if (alpha - 1 == b) return vfma(u[b], t, vmul(P, splat<T>(sc)));
  return vmul(u[alpha - 1], t);
}

// Axis-b direction pair of lattice L: c = +e_b and c = -e_b.
template <class L> __host__ __device__ constexpr int dir_pos(int b) { return L::Q == 5 ? 1 + b : 1 + 2 * b; }
template <class L> __host__ __device__ constexpr int dir_neg(int b) { return L::Q == 5 ? 3 + b : 2 + 2 * b; }

// Relax-and-encode of one set: g (scaled pulled populations) -> stored s.
// Ef: first-moment deviations m_b - m_b^eq (scaled); m0: scaled zeroth
// moment; Fw, Fw0: scaled source w_i F for i > 0 and i = 0.  k: the
// (1 - s_k)/|row k|^2 factors.
template <class L, class T>
__device__ __forceinline__ void relax_encode(T (&g)[L::Q], const T (&Ef)[L::D], T m0, T Fw, T Fw0,
                                             const float (&k)[6]) {
  if constexpr (L::Q == 5) {
    // D2Q5 rows: m1 = g1 - g3, m2 = g2 - g4, m3 = g1 + g3 - g2 - g4,
    // m4 = g1 + g2 + g3 + g4 - 4 g0; |row|^2 = 2, 2, 4, 20; m4eq = -2/3 m0.
    const T p13 = vadd(g[1], g[3]), p24 = vadd(g[2], g[4]);
    const T E1 = Ef[0], E2 = Ef[1];
    const T E3 = vsub(p13, p24);
    const T E4 = vfma(splat<T>(2.f / 3.f), m0, vfma(splat<T>(-4.f), g[0], vadd(p13, p24)));
    // k = {(1-s1)/2, (1-s2)/4, (1-s2)/20, -4 (1-s2)/20}
    const T t = vfma(splat<T>(k[2]), E4, Fw);
    const T pp = vfma(splat<T>(k[1]), E3, t), nn = vfma(splat<T>(-k[1]), E3, t);
    g[0] = vfma(splat<T>(k[3]), E4, Fw0);
    g[1] = vfma(splat<T>(k[0]), E1, pp);
    g[3] = vfma(splat<T>(-k[0]), E1, pp);
    g[2] = vfma(splat<T>(k[0]), E2, nn);
    g[4] = vfma(splat<T>(-k[0]), E2, nn);
  } else {
    // D3Q7 rows: m1..3 first moments, m4 = sum_{i>0} g - 6 g0,
    // m5 = 2 sx - sy - sz, m6 = sy - sz; |row|^2 = 2, 42, 12, 4;
    // m4eq = -3/4 m0, m5eq = m6eq = 0.
    const T sx = vadd(g[1], g[2]), sy = vadd(g[3], g[4]), sz = vadd(g[5], g[6]);
    const T syz = vadd(sy, sz);
    const T E1 = Ef[0], E2 = Ef[1], E3 = Ef[2];
    const T E4 = vfma(splat<T>(0.75f), m0, vfma(splat<T>(-6.f), g[0], vadd(sx, syz)));
    const T E5 = vsub(vadd(sx, sx), syz);
    const T E6 = vsub(sy, sz);
    // k = {(1-s1)/2, (1-s2)/42, (1-s2)/6, -(1-s2)/12, (1-s2)/4, -6 (1-s2)/42}
    const T t = vfma(splat<T>(k[1]), E4, Fw);
    const T A = vfma(splat<T>(k[2]), E5, t), B = vfma(splat<T>(k[3]), E5, t);
    const T B3 = vfma(splat<T>(k[4]), E6, B), B5 = vfma(splat<T>(-k[4]), E6, B);
    g[0] = vfma(splat<T>(k[5]), E4, Fw0);
    g[1] = vfma(splat<T>(k[0]), E1, A);
    g[2] = vfma(splat<T>(-k[0]), E1, A);
    g[3] = vfma(splat<T>(k[0]), E2, B3);
    g[4] = vfma(splat<T>(-k[0]), E2, B3);
    g[5] = vfma(splat<T>(k[0]), E3, B5);
    g[6] = vfma(splat<T>(-k[0]), E3, B5);
  }
}

// Stochastic rounding of two FP32 values to a packed 16-bit pair in one
// instruction (cvt.rs, sm_100 family): lo goes to bits 15..0, hi to bits
// 31..16, and rbits[15:0] / rbits[31:16] are their random bits.
template <class TS> __device__ __forceinline__ uint32_t cvt_rs_pair(float lo, float hi, uint32_t rbits);
template <> __device__ __forceinline__ uint32_t cvt_rs_pair<__half>(float lo, float hi, uint32_t rbits) {
  uint32_t d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
template <> __device__ __forceinline__ uint32_t cvt_rs_pair<__nv_bfloat16>(float lo, float hi, uint32_t rbits) {
  uint32_t d;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
// Random word of population e of the node pair (x, x + 1), x even, from
// the key of its even node: an odd multiple, so each half is uniform.
__device__ __forceinline__ uint32_t pair_word(uint32_t key, int e) {
  return key * (0x9e3779b1u + 2u * (uint32_t)e);
}

// Moments of the x - 1 and x + VX neighbours of a thread's nodes: from the
// neighbouring lanes, or, at a warp or row edge, from the loaded El / Er.
template <int KM, int VX>
__device__ __forceinline__ void settle_edge_moments(const float (&Mo)[KM][VX], const float (&El)[KM],
                                                    const float (&Er)[KM], int K, bool ledge, bool redge,
                                                    float (&Mxl)[KM], float (&Mxr)[KM]) {
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    const float l = __shfl_up_sync(0xffffffffu, Mo[k][VX - 1], 1);
    const float r = __shfl_down_sync(0xffffffffu, Mo[k][0], 1);
    Mxl[k] = k < K ? (ledge ? El[k] : l) : 0.f;
    Mxr[k] = k < K ? (redge ? Er[k] : r) : 0.f;
  }
}

// VX consecutive 16-bit elements of population e stored with stochastic
// rounding, as one 2/4/8/16-byte access; kp[p] is the key of the even node
// of pair p.  VX = 1 (node x, x0 = x) takes its lane of its pair's word, so
// every width stores the same bits.
template <class TS, int VX>
__device__ __forceinline__ void store_sr(TS *p, const float (&v)[VX], const uint32_t (&kp)[(VX + 1) / 2],
                                         int e, int x0) {
  if constexpr (VX == 1) {
    const int odd = x0 & 1;
    const uint32_t d = cvt_rs_pair<TS>(odd ? 0.f : v[0], odd ? v[0] : 0.f, pair_word(kp[0], e));
    *reinterpret_cast<unsigned short *>(p) = (unsigned short)(odd ? d >> 16 : d);
  } else {
    using Raw = typename std::conditional<VX == 2, uint32_t,
                typename std::conditional<VX == 4, uint2, uint4>::type>::type;
    Raw raw;
    uint32_t *w = reinterpret_cast<uint32_t *>(&raw);
#pragma unroll
    for (int k = 0; k < VX / 2; ++k) w[k] = cvt_rs_pair<TS>(v[2 * k], v[2 * k + 1], pair_word(kp[k], e));
    *reinterpret_cast<Raw *>(p) = raw;
  }
}

template <class L, class TS, int VX, int MODE, bool WALLS>
__global__ void __launch_bounds__(kMaxBlock) k_update_eq(const DevArgs A) {
  constexpr int D = L::D, Q = L::Q, KM = D + 2;
  using T = typename Lanes<VX>::T;
  constexpr int NP = Lanes<VX>::N, LW = Lanes<VX>::W;
  constexpr float SC = EqScale<TS>::s, INV = EqScale<TS>::inv;
  const int lane = threadIdx.x & 31;
  int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * VX;
  const bool active = x0 < A.nx;
  if (!active) x0 = A.nx - VX;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long rc = (long long)z * A.ny + y;  // this row and the rows the pulls come from
  const long long rym = (long long)z * A.ny + wrap(y - 1, A.ny);
  const long long ryp = (long long)z * A.ny + wrap(y + 1, A.ny);
  const long long rzm = D == 3 ? (long long)wrap(z - 1, A.nz) * A.ny + y : rc;
  const long long rzp = D == 3 ? (long long)wrap(z + 1, A.nz) * A.ny + y : rc;
  const bool ledge = lane == 0 || x0 == 0;
  const bool redge = lane == 31 || x0 + VX >= A.nx;
  const int xl = x0 == 0 ? A.nx - 1 : x0 - 1;
  const int xr = x0 + VX >= A.nx ? 0 : x0 + VX;
  const int K = moment_slots(D, A.with_rho);
  const int NK = (D + A.with_rho) * Q;  // population arrays per tile
  const TS *__restrict__ fin = static_cast<const TS *>(A.fin);
  const float *__restrict__ min = static_cast<const float *>(A.min);
  const int a1 = A.with_rho;
  // tile pointers: array k of the thread's nodes (or of an x-edge node) is
  // at pointer + k * kEqTile
  const TS *Pc = fin + eq_off(A.px, rc, x0, NK), *Pym = fin + eq_off(A.px, rym, x0, NK);
  const TS *Pyp = fin + eq_off(A.px, ryp, x0, NK), *Pzm = fin + eq_off(A.px, rzm, x0, NK);
  const TS *Pzp = fin + eq_off(A.px, rzp, x0, NK);
  const TS *Pl = fin + eq_off(A.px, rc, xl, NK), *Pr = fin + eq_off(A.px, rc, xr, NK);

  uint8_t m[VX];
  if (WALLS) {
#pragma unroll
    for (int j = 0; j < VX; ++j) m[j] = A.mask[rc * A.px + x0 + j];
  }
  // ---- every load of the thread is issued before any value is used (moments
  // of the node and its pull sources, the x-edge moments, the population
  // words and their x-edge words), so that all are in flight together
  float Mo[KM][VX], Mym[KM][VX], Myp[KM][VX], Mzm[KM][VX], Mzp[KM][VX], Mxl[KM], Mxr[KM];
  load_moments<KM, VX>(min + eq_off(A.px, rc, x0, K), K, Mo);
  load_moments<KM, VX>(min + eq_off(A.px, rym, x0, K), K, Mym);
  load_moments<KM, VX>(min + eq_off(A.px, ryp, x0, K), K, Myp);
  if (D == 3) {
    load_moments<KM, VX>(min + eq_off(A.px, rzm, x0, K), K, Mzm);
    load_moments<KM, VX>(min + eq_off(A.px, rzp, x0, K), K, Mzp);
  }
  float El[KM], Er[KM];  // x - 1 and x + VX moments, read by the warp's edge lanes
  {
    const float *Ml = min + eq_off(A.px, rc, xl, K), *Mr = min + eq_off(A.px, rc, xr, K);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      El[k] = (k < K && ledge) ? __ldg(Ml + k * kEqTile) : 0.f;
      Er[k] = (k < K && redge) ? __ldg(Mr + k * kEqTile) : 0.f;
    }
  }
  // In 3D (28 words and five moment rows per thread, ~124 registers) the
  // x-neighbour moments are settled before the population words are
  // requested, which keeps fewer values live (measured faster there; so is
  // this register path against staging the moment rows in shared memory);
  // in 2D everything is requested first.
  if constexpr (D == 3) settle_edge_moments<KM, VX>(Mo, El, Er, K, ledge, redge, Mxl, Mxr);
  using PW = typename Packed16<TS, VX>::W;
  PW wv[D + 1][Q];
  unsigned edge[D + 1][2];  // per set: x - 1 value of the +x pull, x + VX value of the -x pull
#pragma unroll
  for (int s = 0; s <= D; ++s) {
    const int alpha = s == D ? 0 : s + 1;  // velocity sets first, alpha = 0 last
    if (alpha == 0 && !A.with_rho) break;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int k = ((alpha == 0 ? 0 : a1 + alpha - 1) * Q + i) * kEqTile;
      const TS *p = L::c(i, 1) == 1 ? Pym : L::c(i, 1) == -1 ? Pyp
                  : L::c(i, 2) == 1 ? Pzm : L::c(i, 2) == -1 ? Pzp : Pc;
      wv[s][i] = Packed16<TS, VX>::load(p + k);
      if (L::c(i, 0) == 1) edge[s][0] = ledge ? ldg_bits16(Pl + k) : 0u;
      if (L::c(i, 0) == -1) edge[s][1] = redge ? ldg_bits16(Pr + k) : 0u;
    }
  }
  if constexpr (D == 2) settle_edge_moments<KM, VX>(Mo, El, Er, K, ledge, redge, Mxl, Mxr);
  // ---- decode, direction by direction (source terms shared by the sets)
  T G[D + 1][Q][NP];  // [velocity sets 0..D-1, continuity set D][i][lane group]
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    T su[NP][D], sP[NP], sr[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      float e[KM][LW];
#pragma unroll
      for (int q = 0; q < LW; ++q) {
        float Ms[KM];
        source_moments<L, VX>(i, LW * p + q, Mo, Mym, Myp, Mzm, Mzp, Mxl, Mxr, Ms);
#pragma unroll
        for (int k = 0; k < KM; ++k) e[k][q] = Ms[k];
      }
#pragma unroll
      for (int b = 0; b < D; ++b) to_lanes(su[p][b], e[b]);
      to_lanes(sP[p], e[D]);
      to_lanes(sr[p], e[D + 1]);
    }
    const float sw = float(SC * L::w(i));
#pragma unroll
    for (int s = 0; s <= D; ++s) {
      const int alpha = s == D ? 0 : s + 1;
      if (alpha == 0 && !A.with_rho) break;
      const PW w = wv[s][i];
      T rv[NP];
      if (L::c(i, 0) == 1) {  // raw[0] from the lane to the left, raw[j] = own[j - 1]
        unsigned nb = __shfl_up_sync(0xffffffffu, Packed16<TS, VX>::last_word(w), 1);
        nb = ledge ? edge[s][0] : (VX == 1 ? nb : nb >> 16);
        float raw[VX];
        raw[0] = bits_to_float<TS>(nb);
#pragma unroll
        for (int j = 1; j < VX; ++j) raw[j] = bits_to_float<TS>(Packed16<TS, VX>::bits(w, j - 1));
#pragma unroll
        for (int q = 0; q < NP; ++q) to_lanes(rv[q], raw + LW * q);
      } else if (L::c(i, 0) == -1) {  // raw[j] = own[j + 1], raw[VX - 1] from the right
        unsigned nb = __shfl_down_sync(0xffffffffu, Packed16<TS, VX>::first_word(w), 1);
        nb = redge ? edge[s][1] : (nb & 0xffffu);
        float raw[VX];
#pragma unroll
        for (int j = 0; j < VX - 1; ++j) raw[j] = bits_to_float<TS>(Packed16<TS, VX>::bits(w, j + 1));
        raw[VX - 1] = bits_to_float<TS>(nb);
#pragma unroll
        for (int q = 0; q < NP; ++q) to_lanes(rv[q], raw + LW * q);
      } else {
#pragma unroll
        for (int q = 0; q < NP; ++q) rv[q] = Packed16<TS, VX>::lanes(w, q);
      }
#pragma unroll
      for (int q = 0; q < NP; ++q)
        G[s][i][q] = vfma(eq_inner<L, T>(alpha, i, su[q], sP[q], sr[q]), splat<T>(sw), rv[q]);
    }
  }
  if (WALLS) {  // anti-halfway bounce-back from the node's own opposite population
#pragma unroll
    for (int s = 0; s <= D; ++s) {
      const int alpha = s == D ? 0 : s + 1;
      if (alpha == 0 && !A.with_rho) break;
      const TS *base = Pc + (alpha == 0 ? 0 : a1 + alpha - 1) * Q * kEqTile;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int o = L::opp(i);
        const float swo = float(SC * L::w(o));
        const float lid = alpha >= 1 ? float(SC * 2.0 * L::w(i) * A.lid_u[alpha - 1]) : 0.f;
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          if ((m[j] >> o) & 1) {
            float un[D];
#pragma unroll
            for (int b = 0; b < D; ++b) un[b] = Mo[b][j];
            const float own = Codec<TS>::load(base + o * kEqTile + j);
            float w = -vfma(eq_inner<L, float>(alpha, o, un, Mo[D][j], Mo[D + 1][j]), swo, own);
            if (alpha >= 1 && i == L::opp(L::UP) && (m[j] & 0x80u)) w = vadd(w, lid);
            float v[LW];
            from_lanes(v, G[s][i][j / LW]);
            v[j % LW] = w;
            to_lanes(G[s][i][j / LW], v);
          }
        }
      }
    }
  }

  const long long N = (long long)A.nx * A.ny * A.nz;
  const long long n0 = ((long long)z * A.ny + y) * A.nx + x0;
  float Fr[D][VX];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (A.force) {
      VecIO<float, VX>::load(static_cast<const float *>(A.force) + a * A.plane + rc * A.px + x0, Fr[a]);
    } else {
#pragma unroll
      for (int j = 0; j < VX; ++j) Fr[a][j] = 0.f;
    }
  }
  if (MODE != MODE_STEP && active) {  // derived fields of the pulled state (FP32, unscaled)
#pragma unroll
    for (int j = 0; j < VX; ++j) {
      float gn[D][Q], hn[Q], Fn[D];
#pragma unroll
      for (int a = 0; a < D; ++a) Fn[a] = Fr[a][j];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        float v[LW];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          from_lanes(v, G[a][i][j / LW]);
          gn[a][i] = vmul(v[j % LW], INV);
        }
        from_lanes(v, G[D][i][j / LW]);
        hn[i] = A.with_rho ? vmul(v[j % LW], INV) : 0.f;
      }
      write_fields<L, float>(A, n0 + j, N, gn, hn, Fn);
    }
  }
  if (MODE == MODE_FIELDS || !active) return;

  // ---- collide + encode
  const float s1 = A.s1f, s2 = A.s2f;
  float kf[6];
  if constexpr (Q == 5) {
    kf[0] = (1.f - s1) * 0.5f;
    kf[1] = (1.f - s2) * 0.25f;
    kf[2] = (1.f - s2) * 0.05f;
    kf[3] = (1.f - s2) * -0.2f;
    kf[4] = kf[5] = 0.f;
  } else {
    kf[0] = (1.f - s1) * 0.5f;
    kf[1] = (1.f - s2) * float(1.0 / 42.0);
    kf[2] = (1.f - s2) * float(1.0 / 6.0);
    kf[3] = (1.f - s2) * float(-1.0 / 12.0);
    kf[4] = (1.f - s2) * 0.25f;
    kf[5] = (1.f - s2) * float(-1.0 / 7.0);
  }
  // Scheme II (Eq. 2-3c): G holds SCALE fbar; ubar = sum fbar + Fbar/2
  // (Eq. 2-7a) builds the equilibrium first moments and the stored moments,
  // m4 relaxes towards k sum fbar, and the stored deviation from
  // g^eq(ubar) carries w_i Fbar / 2 (the zeroth and m4 parts of the
  // (I - S/2) source less the Fbar/2 in g^eq; the s0 and s2 terms cancel).
  const float fw_scale = A.scheme2 ? 0.5f : 1.f;
  T Mn[KM][NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    // Every product that meets a sum is one fma (nothing is left for the
    // compiler to contract, so scalar and pair lanes give the same bits).
    T us[D], ub[D], u[D], un[D], Fs[D], dif[D + 1][D], tr = splat<T>(0.f), usqS = splat<T>(0.f);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float fl[LW];
#pragma unroll
      for (int e = 0; e < LW; ++e) fl[e] = Fr[a][LW * q + e];
      to_lanes(Fs[a], fl);
      Fs[a] = vmul(Fs[a], splat<T>(SC));
      T sm = G[a][0][q];
#pragma unroll
      for (int i = 1; i < Q; ++i) sm = vadd(sm, G[a][i][q]);
      us[a] = sm;
      ub[a] = A.scheme2 ? vfma(Fs[a], splat<T>(0.5f), sm) : sm;
      u[a] = SC == 1.f ? ub[a] : vmul(ub[a], splat<T>(INV));
      un[a] = vsub(splat<T>(0.f), u[a]);
    }
#pragma unroll
    for (int a = 0; a <= D; ++a) {
      if (a == D && !A.with_rho) break;
#pragma unroll
      for (int b = 0; b < D; ++b) dif[a][b] = vsub(G[a][dir_pos<L>(b)][q], G[a][dir_neg<L>(b)][q]);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {  // sum_i c_{i,a} G_{i,a} and SCALE |u|^2
      tr = vadd(tr, dif[a][a]);
      usqS = vfma(ub[a], u[a], usqS);
    }
    // Eq. 3-15 (scaled): SCALE P' = (SCALE tr - SCALE |u|^2) / d
    const T PS = vmul(vsub(tr, usqS), splat<T>(float(1.0 / D)));
    const T P = SC == 1.f ? PS : vmul(PS, splat<T>(INV));
#pragma unroll
    for (int a = 0; a < D; ++a) {
      // m_b - m_b^eq with m_b^eq = SCALE (u_a u_b + [a = b] P') (Eq. 3-7a)
      T Ef[D];
#pragma unroll
      for (int b = 0; b < D; ++b)
        Ef[b] = a == b ? vsub(dif[a][b], vfma(ub[a], u[b], PS)) : vfma(ub[a], un[b], dif[a][b]);
      const T Fw = vmul(Fs[a], splat<T>(fw_scale * float(L::w(1))));
      const T Fw0 = vmul(Fs[a], splat<T>(fw_scale * float(L::w(0))));
      T gq[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) gq[i] = G[a][i][q];
      relax_encode<L, T>(gq, Ef, us[a], Fw, Fw0, kf);
#pragma unroll
      for (int i = 0; i < Q; ++i) G[a][i][q] = gq[i];
    }
    T rr = splat<T>(0.f);
    if (A.with_rho) {
      T sm = G[D][0][q];
#pragma unroll
      for (int i = 1; i < Q; ++i) sm = vadd(sm, G[D][i][q]);
      rr = SC == 1.f ? sm : vmul(sm, splat<T>(INV));
      const T rs = vadd(sm, splat<T>(SC));  // SCALE (1 + rho'): m_b^eq = rs u_b
      T Ef[D];
#pragma unroll
      for (int b = 0; b < D; ++b) Ef[b] = vfma(rs, un[b], dif[D][b]);
      T gq[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) gq[i] = G[D][i][q];
      relax_encode<L, T>(gq, Ef, sm, splat<T>(0.f), splat<T>(0.f), kf);
#pragma unroll
      for (int i = 0; i < Q; ++i) G[D][i][q] = gq[i];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) Mn[a][q] = u[a];
    Mn[D][q] = P;
    Mn[D + 1][q] = rr;
  }

  TS *__restrict__ fout = static_cast<TS *>(A.fout);
  float *__restrict__ mout = static_cast<float *>(A.mout);
  // stochastic rounding of the stored 16-bit parts: the random bits of a
  // node pair (x, x + 1), x even, come from its even node's key of (global
  // index, time step)
  uint32_t kp[(VX + 1) / 2];
  {
    const int tstep = launch_step(A);
#pragma unroll
    for (int p = 0; p < (VX + 1) / 2; ++p)
      kp[p] = node_key(A.key_base + n0 + 2 * p - (VX == 1 ? (x0 & 1) : 0), tstep);
  }
#pragma unroll
  for (int s = 0; s <= D; ++s) {
    const int alpha = s == D ? 0 : s + 1;
    if (alpha == 0 && !A.with_rho) break;
    TS *base = fout + eq_off(A.px, rc, x0, NK) + (alpha == 0 ? 0 : a1 + alpha - 1) * Q * kEqTile;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float v[VX];
#pragma unroll
      for (int q = 0; q < NP; ++q) from_lanes(v + LW * q, G[s][i][q]);
      store_sr<TS, VX>(base + i * kEqTile, v, kp, s * Q + i, x0);
    }
  }
  float *mo = mout + eq_off(A.px, rc, x0, K);
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    if (k < K) {
      float v[VX];
#pragma unroll
      for (int q = 0; q < NP; ++q) from_lanes(v + LW * q, Mn[k][q]);
      VecIO<float, VX>::store(mo + k * kEqTile, v);
    }
  }
}

// Initial state f = f^eq(P, u) in pull form for this codec: moments
// M0 = (u, P - 1, 0) at every node, and s_i(x) such that the first pull
// rebuilds g^eq_i(M0(x + c_i)) at x + c_i (or, on a wall link, the value
// whose bounce-back returns g^eq_opp(M0(x)) at x).  A seed gradient adds
// f^ne (fne_at); under Scheme II the rebuilt value is fbar = f - w_i Fbar / 2
// (its ubar is still u).
template <class L>
__device__ __forceinline__ void init_moments(const DevArgs &A, long long N, long long n,
                                             float (&M)[L::D + 2]) {
#pragma unroll
  for (int b = 0; b < L::D; ++b) M[b] = narrow_f64(A.uin[b * N + n]);
  M[L::D] = narrow_f64(A.Pin[n] - 1.0);
  M[L::D + 1] = 0.f;
}

template <class L, class TS, bool WALLS>
__global__ void __launch_bounds__(kMaxBlock) k_init_eq(const DevArgs A) {
  constexpr int D = L::D, Q = L::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= A.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long idx = ((long long)z * A.ny + y) * A.px + x;
  const long long N = (long long)A.nx * A.ny * A.nz;
  const long long n = ((long long)z * A.ny + y) * A.nx + x;
  const uint8_t m = WALLS ? A.mask[idx] : uint8_t(0);
  float M0[D + 2];
  init_moments<L>(A, N, n, M0);
  float *mout = static_cast<float *>(A.mout);
  const int K = moment_slots(D, A.with_rho);
  const long long row = (long long)z * A.ny + y;
  for (int k = 0; k < K; ++k) mout[eq_off(A.px, row, x, K) + k * kEqTile] = M0[k];
  TS *fout = static_cast<TS *>(A.fout);
  const int nsets = D + A.with_rho;
  TS *fn = fout + eq_off(A.px, row, x, nsets * Q);
  for (int a = 0; a < nsets; ++a) {
    const int alpha = a + 1 - A.with_rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float target;
      const bool half = A.scheme2 && alpha >= 1;
      const float *Fa = half ? static_cast<const float *>(A.force) + (alpha - 1) * A.plane : nullptr;
      if (WALLS && i != 0 && ((m >> i) & 1)) {
        target = -geq_m<L>(alpha, L::opp(i), M0);
        if (A.Gin) target -= narrow_f64(fne_at<L>(A, N, n, alpha, L::opp(i)));
        if (alpha >= 1 && i == L::UP && (m & 0x80u)) target += float(2.0 * L::w(i) * A.lid_u[alpha - 1]);
        if (half) target += float(0.5 * L::w(i)) * __ldg(Fa + idx);  // negated by the bounce-back
      } else {
        const int tx = wrap(x + L::c(i, 0), A.nx);
        const int ty = wrap(y + L::c(i, 1), A.ny);
        const int tz = D == 3 ? wrap(z + L::c(i, 2), A.nz) : z;
        const long long tn = ((long long)tz * A.ny + ty) * A.nx + tx;
        float Mt[D + 2];
        init_moments<L>(A, N, tn, Mt);
        target = geq_m<L>(alpha, i, Mt);
        if (A.Gin) target += narrow_f64(fne_at<L>(A, N, tn, alpha, i));
        if (half) target -= float(0.5 * L::w(i)) * __ldg(Fa + ((long long)tz * A.ny + ty) * A.px + tx);
      }
      Codec<TS>::store(fn + (a * Q + i) * kEqTile, (target - geq_m<L>(alpha, i, M0)) * EqScale<TS>::s);
    }
  }
}

// Scalar pull of every set at one node for the reductions.
template <class L, class TS, bool WALLS>
__device__ __forceinline__ void pull_node_eq(const DevArgs &A, int x, int y, int z,
                                             float (&g)[L::D + 1][L::Q]) {
  constexpr int D = L::D, Q = L::Q;
  const long long idx = ((long long)z * A.ny + y) * A.px + x;
  const uint8_t m = WALLS ? A.mask[idx] : uint8_t(0);
  const int K = moment_slots(D, A.with_rho);
  const float *min = static_cast<const float *>(A.min);
  const TS *fin = static_cast<const TS *>(A.fin);
  const int nsets = D + A.with_rho;
  const long long row = (long long)z * A.ny + y;
  float Mo[D + 2];
#pragma unroll
  for (int k = 0; k < D + 2; ++k) Mo[k] = k < K ? __ldg(min + eq_off(A.px, row, x, K) + k * kEqTile) : 0.f;
  for (int a = 0; a < nsets; ++a) {
    const int alpha = a + 1 - A.with_rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (WALLS && i != 0 && ((m >> L::opp(i)) & 1)) {
        float w = -(Codec<TS>::load(fin + eq_off(A.px, row, x, nsets * Q) + (a * Q + L::opp(i)) * kEqTile) *
                        EqScale<TS>::inv +
                    geq_m<L>(alpha, L::opp(i), Mo));
        if (alpha >= 1 && i == L::opp(L::UP) && (m & 0x80u)) w += float(2.0 * L::w(i) * A.lid_u[alpha - 1]);
        g[a][i] = w;
      } else {  // from the node x - c_i (periodic wrap)
        const int sx = wrap(x - L::c(i, 0), A.nx);
        const int sy = wrap(y - L::c(i, 1), A.ny);
        const int sz = D == 3 ? wrap(z - L::c(i, 2), A.nz) : z;
        const long long srow = (long long)sz * A.ny + sy;
        float Ms[D + 2];
#pragma unroll
        for (int k = 0; k < D + 2; ++k) Ms[k] = k < K ? __ldg(min + eq_off(A.px, srow, sx, K) + k * kEqTile) : 0.f;
        g[a][i] = Codec<TS>::load(fin + eq_off(A.px, srow, sx, nsets * Q) + (a * Q + i) * kEqTile) *
                      EqScale<TS>::inv +
                  geq_m<L>(alpha, i, Ms);
      }
    }
  }
}

template <class L, class TS, bool WALLS, int KIND>
__global__ void __launch_bounds__(kReduceThreads) k_reduce_eq(const DevArgs A) {
  constexpr int D = L::D, Q = L::Q;
  const long long N = (long long)A.nx * A.ny * A.nz;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  bool bad = false;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % A.nx);
    const int y = (int)((n / A.nx) % A.ny);
    const int z = (int)(n / ((long long)A.nx * A.ny));
    float g[D + 1][Q];
    pull_node_eq<L, TS, WALLS>(A, x, y, z, g);
    const int nsets = D + A.with_rho;
#pragma unroll
    for (int a = 0; a < D + 1; ++a) {
      if (a >= nsets) break;
      const int alpha = a + 1 - A.with_rho;
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) s += (double)g[a][i];
      if (alpha == 0) s += 1.0;
      if (A.scheme2 && alpha >= 1)  // Eq. 2-7a
        s += 0.5 * (double)__ldg(static_cast<const float *>(A.force) + (alpha - 1) * A.plane +
                                 ((long long)z * A.ny + y) * A.px + x);
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

}  // namespace mdf

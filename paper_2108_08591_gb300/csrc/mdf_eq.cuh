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

template <int KM, int VX>
__device__ __forceinline__ void load_moments(const DevArgs &A, int K, int off,
                                             float (&M)[KM][VX]) {
  const float *min = static_cast<const float *>(A.min);
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    if (k < K) {
      float v[VX];
      VecIO<float, VX>::load(min + (long long)k * A.plane + off, v);
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

template <class L, class TS, int VX, int MODE, bool WALLS>
__global__ void __launch_bounds__(kMaxBlock) k_update_eq(const DevArgs A) {
  constexpr int D = L::D, Q = L::Q;
  const float scale = EqScale<TS>::s, inv = EqScale<TS>::inv;
  const int lane = threadIdx.x & 31;
  int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * VX;
  const bool active = x0 < A.nx;
  if (!active) x0 = A.nx - VX;
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
  const int K = moment_slots(D, A.with_rho);
  const TS *__restrict__ fin = static_cast<const TS *>(A.fin);
  const float *__restrict__ min = static_cast<const float *>(A.min);

  uint8_t m[VX];
  if (WALLS) {
#pragma unroll
    for (int j = 0; j < VX; ++j) m[j] = A.mask[row0 + x0 + j];
  }
  // moments of this row's nodes, the y/z neighbour rows and the two x ends
  constexpr int KM = D + 2;
  float Mo[KM][VX], Mym[KM][VX], Myp[KM][VX], Mzm[KM][VX], Mzp[KM][VX], Mxl[KM], Mxr[KM];
  load_moments<KM, VX>(A, K, row0 + x0, Mo);
  load_moments<KM, VX>(A, K, row_ym + x0, Mym);
  load_moments<KM, VX>(A, K, row_yp + x0, Myp);
  if (D == 3) {
    load_moments<KM, VX>(A, K, row_zm + x0, Mzm);
    load_moments<KM, VX>(A, K, row_zp + x0, Mzp);
  }
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    float l = __shfl_up_sync(0xffffffffu, Mo[k][VX - 1], 1);
    float r = __shfl_down_sync(0xffffffffu, Mo[k][0], 1);
    if (k < K) {
      if (ledge) l = __ldg(min + (long long)k * A.plane + row0 + xl);
      if (redge) r = __ldg(min + (long long)k * A.plane + row0 + xr);
    } else {
      l = r = 0.f;
    }
    Mxl[k] = l;
    Mxr[k] = r;
  }

  float g[D][Q][VX], h[Q][VX];
  const int a1 = A.with_rho;
#pragma unroll
  for (int s = 0; s <= D; ++s) {
    const int alpha = s == D ? 0 : s + 1;  // velocity sets first, alpha = 0 last
    if (alpha == 0 && !A.with_rho) break;
    const TS *base = fin + (long long)(alpha == 0 ? 0 : a1 + alpha - 1) * Q * A.plane;
    float(&v)[Q][VX] = s == D ? h : g[s < D ? s : 0];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const TS *p = base + (long long)i * A.plane;
      float raw[VX];
      if (L::c(i, 0) == 1) {
        float own[VX];
        VecIO<TS, VX>::load(p + row0 + x0, own);
        float pv = __shfl_up_sync(0xffffffffu, own[VX - 1], 1);
        if (ledge) pv = Codec<TS>::load(p + row0 + xl);
        raw[0] = pv;
#pragma unroll
        for (int j = 1; j < VX; ++j) raw[j] = own[j - 1];
      } else if (L::c(i, 0) == -1) {
        float own[VX];
        VecIO<TS, VX>::load(p + row0 + x0, own);
        float nv = __shfl_down_sync(0xffffffffu, own[0], 1);
        if (redge) nv = Codec<TS>::load(p + row0 + xr);
#pragma unroll
        for (int j = 0; j < VX - 1; ++j) raw[j] = own[j + 1];
        raw[VX - 1] = nv;
      } else {
        const int r = L::c(i, 1) == 1 ? row_ym : L::c(i, 1) == -1 ? row_yp
                    : L::c(i, 2) == 1 ? row_zm : L::c(i, 2) == -1 ? row_zp : row0;
        VecIO<TS, VX>::load(p + r + x0, raw);
      }
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        float Ms[D + 2];
        source_moments<L, VX>(i, j, Mo, Mym, Myp, Mzm, Mzp, Mxl, Mxr, Ms);
        v[i][j] = raw[j] * inv + geq_m<L>(alpha, i, Ms);
      }
    }
    if (WALLS) {  // anti-halfway bounce-back from the node's own opposite population
#pragma unroll
      for (int i = 1; i < Q; ++i)
#pragma unroll
        for (int j = 0; j < VX; ++j)
          if ((m[j] >> L::opp(i)) & 1) {
            float Mn[D + 2];
#pragma unroll
            for (int k = 0; k < D + 2; ++k) Mn[k] = Mo[k][j];
            const float own = Codec<TS>::load(base + (long long)L::opp(i) * A.plane + row0 + x0 + j);
            float w = -(own * inv + geq_m<L>(alpha, L::opp(i), Mn));
            if (alpha >= 1 && i == L::opp(L::UP) && (m[j] & 0x80u))
              w += float(2.0 * L::w(i) * A.lid_u[alpha - 1]);
            v[i][j] = w;
          }
    }
  }

  const long long N = (long long)A.nx * A.ny * A.nz;
  const long long n0 = ((long long)z * A.ny + y) * A.nx + x0;
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
  const float s1 = float(A.s1), s2 = float(A.s2);
  float Mnew[D + 2][VX];
#pragma unroll
  for (int j = 0; j < VX; ++j) {
    float gn[D][Q], hn[Q], Fn[D], M[D + 2];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
#pragma unroll
      for (int a = 0; a < D; ++a) gn[a][i] = g[a][i][j];
      hn[i] = h[i][j];
    }
    if (MODE != MODE_STEP && active) write_fields<L, float>(A, n0 + j, N, gn, hn);
    if (MODE == MODE_FIELDS) continue;
#pragma unroll
    for (int a = 0; a < D; ++a) Fn[a] = F[a][j];
    collide_node<L, float>(gn, hn, A.with_rho != 0, Fn, s1, s2, M);
    // store the non-equilibrium part against the moments just used
#pragma unroll
    for (int i = 0; i < Q; ++i) {
#pragma unroll
      for (int a = 0; a < D; ++a) g[a][i][j] = (gn[a][i] - geq_m<L>(a + 1, i, M)) * scale;
      h[i][j] = (hn[i] - geq_m<L>(0, i, M)) * scale;
    }
#pragma unroll
    for (int k = 0; k < D + 2; ++k) Mnew[k][j] = M[k];
  }
  if (MODE == MODE_FIELDS || !active) return;
  TS *__restrict__ fout = static_cast<TS *>(A.fout);
  float *__restrict__ mout = static_cast<float *>(A.mout);
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int i = 0; i < Q; ++i)
      VecIO<TS, VX>::store(fout + ((long long)(a1 + a) * Q + i) * A.plane + row0 + x0, g[a][i]);
  if (A.with_rho)
#pragma unroll
    for (int i = 0; i < Q; ++i) VecIO<TS, VX>::store(fout + (long long)i * A.plane + row0 + x0, h[i]);
#pragma unroll
  for (int k = 0; k < D + 2; ++k)
    if (k < K) VecIO<float, VX>::store(mout + (long long)k * A.plane + row0 + x0, Mnew[k]);
}

// Initial state f = f^eq(P, u) in pull form for this codec: moments
// M0 = (u, P - 1, 0) at every node, and s_i(x) such that the first pull
// rebuilds g^eq_i(M0(x + c_i)) at x + c_i (or, on a wall link, the value
// whose bounce-back returns g^eq_opp(M0(x)) at x).
template <class L>
__device__ __forceinline__ void init_moments(const DevArgs &A, long long N, long long n,
                                             float (&M)[L::D + 2]) {
#pragma unroll
  for (int b = 0; b < L::D; ++b) M[b] = float(A.uin[b * N + n]);
  M[L::D] = float(A.Pin[n] - 1.0);
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
  for (int k = 0; k < K; ++k) mout[k * A.plane + idx] = M0[k];
  TS *fout = static_cast<TS *>(A.fout);
  const int nsets = D + A.with_rho;
  for (int a = 0; a < nsets; ++a) {
    const int alpha = a + 1 - A.with_rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float target;
      if (WALLS && i != 0 && ((m >> i) & 1)) {
        target = -geq_m<L>(alpha, L::opp(i), M0);
        if (alpha >= 1 && i == L::UP && (m & 0x80u)) target += float(2.0 * L::w(i) * A.lid_u[alpha - 1]);
      } else {
        const int tx = wrap(x + L::c(i, 0), A.nx);
        const int ty = wrap(y + L::c(i, 1), A.ny);
        const int tz = D == 3 ? wrap(z + L::c(i, 2), A.nz) : z;
        float Mt[D + 2];
        init_moments<L>(A, N, ((long long)tz * A.ny + ty) * A.nx + tx, Mt);
        target = geq_m<L>(alpha, i, Mt);
      }
      Codec<TS>::store(fout + ((long long)a * Q + i) * A.plane + idx,
                       (target - geq_m<L>(alpha, i, M0)) * EqScale<TS>::s);
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
  float Mo[D + 2];
#pragma unroll
  for (int k = 0; k < D + 2; ++k) Mo[k] = k < K ? __ldg(min + k * A.plane + idx) : 0.f;
  const int nsets = D + A.with_rho;
  for (int a = 0; a < nsets; ++a) {
    const int alpha = a + 1 - A.with_rho;
    const TS *base = fin + (long long)a * Q * A.plane;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (WALLS && i != 0 && ((m >> L::opp(i)) & 1)) {
        float w = -(Codec<TS>::load(base + (long long)L::opp(i) * A.plane + idx) * EqScale<TS>::inv +
                    geq_m<L>(alpha, L::opp(i), Mo));
        if (alpha >= 1 && i == L::opp(L::UP) && (m & 0x80u)) w += float(2.0 * L::w(i) * A.lid_u[alpha - 1]);
        g[a][i] = w;
      } else {
        const long long src = pull_src<L>(A, x, y, z, i);
        float Ms[D + 2];
#pragma unroll
        for (int k = 0; k < D + 2; ++k) Ms[k] = k < K ? __ldg(min + k * A.plane + src) : 0.f;
        g[a][i] = Codec<TS>::load(base + (long long)i * A.plane + src) * EqScale<TS>::inv +
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

// Rest-shifted 16-bit update with the populations held packed in registers.
//
// With VX nodes per thread the vector kernel keeps Q x (d + 1) x VX FP32
// values live between its loads and its stores (224 for D3Q7 x 4 with 8
// nodes), more than the register file holds.  Here every population stays
// in its 16-bit word from the load to the store:
//   1. every packed word of the thread's nodes (and the x-edge values) is
//      loaded first;
//   2. the x-shifted slots are realigned inside the word (a funnel shift by
//      one element, the end element from the neighbouring lane or the edge
//      load), so element j of every word is the population arriving at node
//      x0 + j;
//   3. node by node, its elements are converted to FP32, collided
//      (collide_node, the other kernels' arithmetic) and converted back to
//      16 bits into the same element;
//   4. the words are stored as they are.
// A population that arrives through a wall is taken, in FP32, from the
// node's own opposite population as in the other kernels, so the bits are
// those of the one-node-per-thread kernel.  Plain updates only.
#pragma once

namespace mdf {

template <class TS> __device__ __forceinline__ unsigned f2bits(float v);
template <> __device__ __forceinline__ unsigned f2bits<__half>(float v) {
  return __half_as_ushort(__float2half_rn(v));
}
template <> __device__ __forceinline__ unsigned f2bits<__nv_bfloat16>(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Words of VX 16-bit elements (element j in half j & 1 of 32-bit word j / 2).
template <int VX> struct Words;
template <> struct Words<4> {
  using W = uint2;
  static __device__ __forceinline__ unsigned &word(W &w, int k) { return k == 0 ? w.x : w.y; }
  // element j <- element j - 1, element 0 <- in
  static __device__ __forceinline__ W up(W w, unsigned in) {
    return make_uint2((w.x << 16) | (in & 0xffffu), __funnelshift_l(w.x, w.y, 16));
  }
  // element j <- element j + 1, element VX - 1 <- in
  static __device__ __forceinline__ W down(W w, unsigned in) {
    return make_uint2(__funnelshift_r(w.x, w.y, 16), (w.y >> 16) | (in << 16));
  }
};
template <> struct Words<8> {
  using W = uint4;
  static __device__ __forceinline__ unsigned &word(W &w, int k) {
    return k == 0 ? w.x : k == 1 ? w.y : k == 2 ? w.z : w.w;
  }
  static __device__ __forceinline__ W up(W w, unsigned in) {
    return make_uint4((w.x << 16) | (in & 0xffffu), __funnelshift_l(w.x, w.y, 16),
                      __funnelshift_l(w.y, w.z, 16), __funnelshift_l(w.z, w.w, 16));
  }
  static __device__ __forceinline__ W down(W w, unsigned in) {
    return make_uint4(__funnelshift_r(w.x, w.y, 16), __funnelshift_r(w.y, w.z, 16),
                      __funnelshift_r(w.z, w.w, 16), (w.w >> 16) | (in << 16));
  }
};

template <int VX>
__device__ __forceinline__ void set_bits(typename Words<VX>::W &w, int j, unsigned b) {
  unsigned &v = Words<VX>::word(w, j >> 1);
  v = (j & 1) ? ((v & 0xffffu) | (b << 16)) : ((v & 0xffff0000u) | (b & 0xffffu));
}

template <class L, class TS, int VX, bool WALLS, bool S2>
__global__ void __launch_bounds__(kMaxBlock) k_update_vec16p(const DevArgs A) {
  static_assert(VX == 4 || VX == 8, "packed words of 4 or 8 elements");
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
  const TS *__restrict__ fin = static_cast<const TS *>(A.fin);
  const int a1 = A.with_rho;
  uint8_t m[VX];
#pragma unroll
  for (int j = 0; j < VX; ++j) m[j] = WALLS ? A.mask[row0 + x0 + j] : uint8_t(0);
  // set s: velocity sets alpha = s + 1 at array index a1 + s, the continuity set last
  auto set_index = [&](int s) { return s < D ? a1 + s : 0; };

  W wv[D + 1][Q];
  unsigned edge[D + 1][2];
#pragma unroll
  for (int s = 0; s <= D; ++s) {
    if (s == D && !A.with_rho) break;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const TS *p = fin + ((long long)set_index(s) * Q + i) * A.plane;
      const int r = L::c(i, 1) == 1 ? row_ym : L::c(i, 1) == -1 ? row_yp
                  : L::c(i, 2) == 1 ? row_zm : L::c(i, 2) == -1 ? row_zp : row0;
      wv[s][i] = PK::load(p + r + x0);
      if (L::c(i, 0) == 1) edge[s][0] = ledge ? ldg_bits16(p + row0 + xl) : 0u;
      if (L::c(i, 0) == -1) edge[s][1] = redge ? ldg_bits16(p + row0 + xr) : 0u;
    }
  }
#pragma unroll
  for (int s = 0; s <= D; ++s) {
    if (s == D && !A.with_rho) break;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (L::c(i, 0) == 1) {  // from x - 1
        unsigned nb = __shfl_up_sync(0xffffffffu, PK::last_word(wv[s][i]), 1) >> 16;
        if (ledge) nb = edge[s][0];
        wv[s][i] = Words<VX>::up(wv[s][i], nb);
      } else if (L::c(i, 0) == -1) {  // from x + 1
        unsigned nb = __shfl_down_sync(0xffffffffu, PK::first_word(wv[s][i]), 1) & 0xffffu;
        if (redge) nb = edge[s][1];
        wv[s][i] = Words<VX>::down(wv[s][i], nb);
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
        if (WALLS && moving<L>(i) && ((m[j] >> L::opp(i)) & 1)) {  // anti-halfway bounce-back
          v = -Codec<TS>::load(fin + ((long long)set_index(s) * Q + L::opp(i)) * A.plane + row0 + x0 + j);
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
#pragma unroll
      for (int i = 0; i < Q; ++i) set_bits<VX>(wv[s][i], j, f2bits<TS>(s < D ? gn[s < D ? s : 0][i] : hn[i]));
    }
  }
  if (!active) return;
  TS *__restrict__ fout = static_cast<TS *>(A.fout);
#pragma unroll
  for (int s = 0; s <= D; ++s) {
    if (s == D && !A.with_rho) break;
#pragma unroll
    for (int i = 0; i < Q; ++i)
      *reinterpret_cast<W *>(fout + ((long long)set_index(s) * Q + i) * A.plane + row0 + x0) = wv[s][i];
  }
}

}  // namespace mdf

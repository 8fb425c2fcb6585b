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
  if (A.scheme2) collide_node<L, TC, true>(g, h, A.with_rho != 0, F, TC(A.s1), TC(A.s2), M);
  else collide_node<L, TC, false>(g, h, A.with_rho != 0, F, TC(A.s1), TC(A.s2), M);

#pragma unroll
  for (int a = 0; a < D; ++a)
    aa_write_set<L, TS, ODD, WALLS>(A, f + (long long)(a1 + a) * Q * A.plane, a + 1, x, y, z, idx, m, g[a]);
  if (A.with_rho) aa_write_set<L, TS, ODD, WALLS>(A, f, 0, x, y, z, idx, m, h);
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

template <class L, class TS>
cudaError_t update_aa_t(int mode, bool walls, const DevArgs &a, cudaStream_t s) {
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

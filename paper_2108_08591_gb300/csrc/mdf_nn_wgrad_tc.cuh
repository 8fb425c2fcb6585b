// Weight gradient of the 3x3 convolution on the 5th-generation tensor cores.
//
// dW[o][t][ci] = sum_p dz[p][o] x[p + s_t][ci]: for every tap t a GEMM over
// pixel positions p (the K dimension) with M = output channels o and N =
// input channels ci.  Pixels are taken in the padded column-strip positions
// of the forward halo kernel (strip width <= 64, pitch P = width + 2), so
// tap (kh, kw) of position p reads x at position p + kh P + kw: one staged
// x halo per chunk of KP positions serves all nine taps as start offsets.
//
// Both operands come straight from NHWC memory with the pixel index
// outermost, i.e. MN-major: rows of 16 bytes (8 channels of one position),
// consecutive positions 16 bytes apart inside an 8-channel column.  Staged
// as such, a K step of 16 positions is a 256-byte advance of the start
// address, and the tap shift a 16-byte one.  dz rows of the discarded pad
// columns (and of positions past the image) are zero, so their x values do
// not contribute.  Nine FP32 accumulators (one per tap, BN columns each)
// live in TMEM; M is 128 output channels (rows past Cout stay zero).  The
// pixel chunks are split over CTAs; each writes its partial sums to
// part[split][Cout][9 Cin] for the split reduction.
//
// Warp-specialised like the forward kernels: warps 0-3 load with cp.async
// and signal a stage's `full` mbarrier, one lane of warp 4 issues the
// 9 x KP / 16 MMAs of a chunk and commits them to the stage's `empty`
// mbarrier; warps 0-3 then read TMEM and store the partial sums.  Every wait
// is bounded; a time-out raises the error flag and the CTA still drains its
// copies and MMAs before freeing TMEM.
#pragma once

#include "mdf_nn_halo.cuh"

namespace mdfnn {

constexpr int WG_KP = 64;  // pixel positions per chunk (K per stage)
constexpr int WG_RB = ((WG_KP + 2 * 66 + 2) + 7) & ~7;  // x-halo rows per 8-channel column

struct WgradTcArgs {
  const bf16 *x;   // [B][H][W][Cin]
  const bf16 *dz;  // [B][H][W][Cout]
  float *part;     // [splits][Cout][9 Cin]
  int B, H, W, Cin, Cout;
  int splits;
};

template <int BN, int S>
constexpr size_t wgrad_tc_smem_bytes() {
  return (size_t)S * (16 * WG_KP * 16 + (BN / 8) * WG_RB * 16) + (2 * S + 1) * 8 + 16;
}

template <int BN, int S>
__global__ void __launch_bounds__(HX_THREADS) k_conv_wgrad_tc(WgradTcArgs a, int *err) {
  static_assert(BN == 16 || BN == 32, "N tile");
  constexpr int LAG = S >= 3 ? S - 1 : 1;  // copy groups in flight
  static_assert(LAG >= 1 && LAG < S, "look-ahead");
  constexpr int A_BYTES = 16 * WG_KP * 16;      // 128 output channels x KP positions
  constexpr int NCB = BN / 8;                   // 8-channel columns of the x halo
  constexpr int B_BYTES = NCB * WG_RB * 16;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t TCOLS = 9 * BN <= 256 ? 256 : 512;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + S * STAGE);
  uint64_t *empty = full + S;
  uint64_t *done = empty + S;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const HaloGeom g = halo_geom(a.H, a.W, 1);
  const int tiles = (a.H * g.P + WG_KP - 1) / WG_KP;
  const long long NQ = (long long)a.B * g.strips * tiles;
  const int split = blockIdx.z;
  const long long q0 = NQ * split / a.splits, q1 = NQ * (split + 1) / a.splits;
  const int NL = (int)(q1 - q0);  // chunks of this CTA (>= 1)
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * 128;
  const int mcores = min(16, (a.Cout - m0) / 8);  // real 8-channel columns of dz
  const int R = WG_KP + 2 * g.P + 2;
  const long long limit = 2000000000LL;

  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int k = 0; k < S; ++k) {
      mbar_init(&full[k], 128);
      mbar_init(&empty[k], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // dz columns past Cout are zero in every stage and never rewritten
  for (int k = tid; k < S * (16 - mcores) * WG_KP; k += blockDim.x) {
    const int st = k / ((16 - mcores) * WG_KP), rem = k - st * ((16 - mcores) * WG_KP);
    const int core = mcores + rem / WG_KP, row = rem - (rem / WG_KP) * WG_KP;
    *reinterpret_cast<uint4 *>(smem + st * STAGE + core * (WG_KP * 16) + row * 16) = make_uint4(0, 0, 0, 0);
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  if (warp < 4) {
    // ---------------- producers
    const int rr = tid & 7;
    const int acore = tid >> 3;  // dz: 16 columns x 8 rows per pass
    const int bcore = (tid >> 3) % NCB, brg = (tid >> 3) / NCB;
    constexpr int BROWS = 8 * (16 / NCB);  // x-halo rows per pass
    for (int i = 0; i < NL; ++i) {
      const int s = i % S;
      if (i >= S && !mbar_wait(&empty[s], (uint32_t)((i / S - 1) & 1), limit)) {
        ok = false;
        break;
      }
      const long long qq = q0 + i;
      const int kt = (int)(qq % tiles);
      const long long bs = qq / tiles;
      const int strip = (int)(bs % g.strips), b = (int)(bs / g.strips);
      const int o0 = kt * WG_KP, col0 = strip * g.TW, TWs = min(g.TW, a.W - col0);
      uint8_t *sa = smem + s * STAGE, *sb = sa + A_BYTES;
      if (acore < mcores) {  // dz rows: positions o0 + row, zero outside the image or in pad columns
        int pr = (o0 + rr) / g.P, pc = (o0 + rr) - pr * g.P;
        for (int row = rr; row < WG_KP; row += 8) {
          const bool v = pr < a.H && pc < TWs;
          const bf16 *src = v ? a.dz + (((size_t)b * a.H + pr) * a.W + col0 + pc) * a.Cout + m0 + acore * 8 : a.dz;
          cp_async16(sa + acore * (WG_KP * 16) + row * 16, src, v);
          pc += 8;
          while (pc >= g.P) {
            pc -= g.P;
            ++pr;
          }
        }
      }
      {  // x halo rows: padded positions o0 + row
        const int r0 = brg * 8 + rr;
        int pr = (o0 + r0) / g.P, pc = (o0 + r0) - pr * g.P;
        const int ci = n0 + bcore * 8;
        for (int row = r0; row < R; row += BROWS) {
          const int h = pr - 1, w = col0 + pc - 1;
          const bool v = ci < a.Cin && (unsigned)h < (unsigned)a.H && (unsigned)w < (unsigned)a.W;
          const bf16 *src = v ? a.x + (((size_t)b * a.H + h) * a.W + w) * a.Cin + ci : a.x;
          cp_async16(sb + bcore * (WG_RB * 16) + row * 16, src, v);
          pc += BROWS;
          while (pc >= g.P) {
            pc -= g.P;
            ++pr;
          }
        }
      }
      cp_async_commit();
      if (i >= LAG) {
        cp_async_wait<LAG>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive(&full[(i - LAG) % S]);
      }
    }
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (ok)
      for (int u = NL > LAG ? NL - LAG : 0; u < NL; ++u) mbar_arrive(&full[u % S]);
    // ---------------- epilogue: lane = output channel, 9 BN columns
    if (!mbar_wait(done, 0u, limit)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (__all_sync(0xffffffffu, ok)) {
      const int o = m0 + warp * 32 + lane;
      float *dst0 = a.part + ((size_t)split * a.Cout + o) * 9 * a.Cin + n0;
#pragma unroll 1
      for (int t = 0; t < 9; ++t) {
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
          float v[16];
          tc_ld<16>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * BN + c0), v);
          if (o < a.Cout && n0 + c0 < a.Cin) {
            float4 *d = reinterpret_cast<float4 *>(dst0 + t * a.Cin + c0);
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
          }
        }
      }
    }
  } else if (lane == 0) {
    // ---------------- MMA issuer: A = dz (MN-major, M = output channels),
    // B = x halo (MN-major, N = input channels), K = positions
    const uint32_t idesc = umma_idesc_bf16(128, BN) | (1u << 15) | (1u << 16);
    // leading byte offset: K-adjacent core matrices (8 positions) 128 B
    // apart; stride byte offset: MN-adjacent core matrices, dz columns KP x
    // 16 B apart, halo columns RB x 16 B apart
    const uint32_t k_st = 128, a_mn = WG_KP * 16, b_mn = WG_RB * 16;
    for (int i = 0; i < NL; ++i) {
      const int s = i % S;
      if (!mbar_wait(&full[s], (uint32_t)((i / S) & 1), limit)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      // descriptors of the stage, advanced through their start-address field
      // (address / 16; shared memory stays below 256 KB, so no carry)
      const uint32_t sa = smem_u32(smem + s * STAGE), sb = sa + A_BYTES;
      const uint64_t da = umma_smem_desc(sa, k_st, a_mn), db = umma_smem_desc(sb, k_st, b_mn);
#pragma unroll 1
      for (int t = 0; t < 9; ++t) {
        const int kh = t / 3, kw = t - 3 * (t / 3);
        const uint64_t dbt = db + (uint64_t)(kh * g.P + kw);  // tap shift: rows of 16 B
#pragma unroll
        for (int ks = 0; ks < WG_KP / 16; ++ks)
          tc_mma(tmem + (uint32_t)(t * BN), da + (uint64_t)(ks * 16), dbt + (uint64_t)(ks * 16), idesc,
                 (i > 0 || ks > 0) ? 1u : 0u);
      }
      tc_commit(&empty[s]);
    }
    tc_commit(done);
    if (!mbar_wait(done, 0u, limit)) ok = false;
  }
  if (!ok) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 4) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS));
  }
}

}  // namespace mdfnn

// Weight gradient of the 3x3 convolution on the 5th-generation tensor cores,
// fed by the Tensor Memory Accelerator.
//
// dW[o][t][ci] = sum_p dz[p][o] x[p + s_t][ci]: for every tap t a GEMM over
// pixel positions p (the K dimension) with M = output channels o and N =
// input channels ci.
//
// A chunk is a block of `rows` image rows x TW columns of one image
// (TW x rows = KC = 64 or 128 positions, TW the power of two in {16, 32,
// 64} that covers the width, or 64 with column strips).  The taps are split over
// CTAs by kernel row kh: per chunk the CTA of row kh loads, with one TMA box
// per 8-channel column,
//   * dz at the chunk's positions (A, M = output channels), and
//   * for kw = 0, 1, 2, x at the same positions shifted by (kh - 1, kw - 1)
//     (B, N = input channels),
// so tap (kh, kw) is a plain GEMM of the chunk: no pad columns and no start
// offsets.  Layers with fewer output than input channels (where fewer of
// the 128 M rows would be padding the other way round) swap the roles: A =
// the three shifted x blocks (M = input channels), B = dz (N = output
// channels), and the epilogue stores the accumulators transposed.  Boxes that reach past the image edges (the -1 and +1 shifts,
// ragged strips and rows) are filled with zeros by the TMA unit, which is
// the convolution's zero padding; dz positions past the image are zero, so
// nothing outside it contributes.
//
// Both operands are MN-major with the 32-, 64- or 128-byte swizzle: a box
// of W channels (W = 16, 32 or 64) x TW x rows lands in shared memory as KC
// rows (positions) of 2W bytes, in groups of 8 rows that the TMA unit and
// the tensor cores swizzle alike, so a K step of 16 positions is an advance
// of two groups.  A (M = 128 output channels) is 128 / W such boxes side by
// side; the ones past Cout are never loaded: the MMA reads whatever lies
// there, and the D rows they make are never stored (each D row depends only
// on its own A row).  The shared memory allocation covers the full 128-row
// read of every stage.
//
// Three FP32 accumulators of BN columns live in TMEM (64 to 256 columns), so
// several CTAs share an SM.  One thread issues the TMA boxes of a stage
// against its `full` mbarrier (expected bytes), one thread issues the
// 3 x KC / 16 MMAs of a chunk and commits them to the stage's `empty`
// mbarrier, and the four warps then read TMEM and store the partial sums
// part[split][Cout][9 Cin] of their split of the chunks.  Every wait is
// bounded; after a time-out the CTA raises the error flag, waits (bounded)
// for the boxes it issued and its MMAs, and frees TMEM.
#pragma once

#include <cuda.h>  // CUtensorMap (the tensor maps are encoded on the host)

#include "mdf_nn_halo.cuh"

namespace mdfnn {

constexpr int WG_THREADS = 128;  // producer lane, MMA lane, four epilogue warps

struct WgradTmaArgs {
  float *part;     // [splits][Cout][9 Cin]
  int B, H, W, Cin, Cout;
  int TW, rows;    // chunk: rows x TW positions (TW x rows = KC of the kernel)
  int strips, rblocks;
  int splits;      // pixel splits; the grid's z is 3 x splits (kernel rows)
  int wa, na;      // A box width in channels, A boxes per copy in the first M tile (layout)
};

// Chunk width of an image of width W: the power of two in {16, 32, 64}
// covering W, or 64 (column strips).
__host__ __device__ inline int wgrad_tw(int W) { return W <= 16 ? 16 : W <= 32 ? 32 : 64; }

// A box width for an M extent of C channels (Cout, or Cin when the roles
// are swapped), and the boxes of the first M tile.
__host__ __device__ inline int wgrad_wa(int C) { return C >= 64 ? 64 : C >= 32 ? 32 : 16; }
__host__ __device__ inline int wgrad_na(int C) {
  const int m = C < 128 ? C : 128, w = wgrad_wa(C);
  return (m + w - 1) / w;
}

// Shared memory of S stages of KC positions: the A boxes of all stages
// first (na boxes of 2 KC wa bytes per copy; one copy, or three shifted
// copies when SWAP), then the B boxes (three shifted copies of 2 KC BN
// bytes, or one when SWAP), then the mbarriers, from a 1024-byte aligned
// base (1 KB of slack).  The MMA reads 128 A rows, 256 KC bytes, from every
// A copy's start, so the data area reaches that far past the last one,
// plus 4 KB (every address an A descriptor can form, with the two byte
// offsets taken either way round).
__host__ __device__ inline size_t wgrad_tma_data_bytes(bool swap, int KC, int BN, int S, int wa, int na) {
  const size_t ac = (size_t)na * 2 * KC * wa, as = (swap ? 3 : 1) * ac;
  const size_t a = S * as, b = (size_t)S * (swap ? 1 : 3) * 2 * KC * BN;
  const size_t reach = (size_t)S * as - ac + 256 * (size_t)KC + 4096;
  return a + b > reach ? a + b : reach;
}
__host__ __device__ inline size_t wgrad_tma_smem_bytes(bool swap, int KC, int BN, int S, int wa, int na) {
  return 1024 + wgrad_tma_data_bytes(swap, KC, BN, S, wa, na) + (2 * S + 1) * 8 + 16;
}

// Swizzle field of a tcgen05 shared-memory descriptor for rows of `bytes`
// (32, 64 or 128) bytes.
__host__ __device__ constexpr uint32_t umma_swizzle(int bytes) { return bytes == 128 ? 2u : bytes == 64 ? 4u : 6u; }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// One box of a 4D tensor map (c0 innermost) into shared memory, completing
// on `bar` with its byte count.  c0 is a channel offset, a multiple of 8
// (16 bytes); the other coordinates may lie outside the tensor (zero fill).
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            int c3, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// SWAP = false: A = dz (M = output channels), B = x (N = input channels),
// three shifted B copies.  SWAP = true, for layers with more input than
// output channels: A = x (M = input channels), three shifted A copies, B =
// dz (N = output channels); the accumulators hold dW transposed.
template <bool SWAP, int KC, int BN, int S>
__global__ void __launch_bounds__(WG_THREADS)
    k_conv_wgrad_tma(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dzmap,
                     WgradTmaArgs a, int *err) {
  static_assert(BN == 16 || BN == 32 || BN == 64, "N tile");
  static_assert(S >= 2 && S <= 8, "stages");
  static_assert(KC == 64 || KC == 128, "positions per chunk");
  constexpr int NA = SWAP ? 3 : 1, NB = SWAP ? 1 : 3;  // copies of A and of B per stage
  constexpr uint32_t BBOX = 2 * KC * BN;                // bytes of one B box (KC positions x BN channels)
  constexpr uint32_t TCOLS = 3 * BN <= 64 ? 64 : 3 * BN <= 128 ? 128 : 256;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // the swizzle pattern repeats every 1024 bytes of the shared address
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t abox = 2u * KC * (uint32_t)a.wa, acopy = abox * (uint32_t)a.na, astage = NA * acopy;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + wgrad_tma_data_bytes(SWAP, KC, BN, S, a.wa, a.na));
  uint64_t *empty = full + S;
  uint64_t *done = empty + S;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  const uint32_t a0 = smem_u32(smem), b0 = a0 + (uint32_t)S * astage;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.z / 3, kh = blockIdx.z - 3 * (blockIdx.z / 3);
  const long long NQ = (long long)a.B * a.strips * a.rblocks;
  const long long q0 = NQ * split / a.splits, q1 = NQ * (split + 1) / a.splits;
  const int NL = (int)(q1 - q0);  // chunks of this CTA (>= 1)
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * 128;
  const int mrem = min(128, (SWAP ? a.Cin : a.Cout) - m0);
  const int na = (mrem + a.wa - 1) / a.wa;  // A boxes per copy this CTA loads (<= a.na)
  const uint32_t stage_bytes = (uint32_t)(NA * na) * abox + NB * BBOX;
  const long long limit = 2000000000LL;

  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int k = 0; k < S; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  if (tid == 0) {
    // ---------------- producer: the boxes of chunk i into stage i % S; the
    // x boxes are shifted by (kh - 1, kw - 1)
    int issued = 0;
    for (int i = 0; i < NL; ++i) {
      const int s = i % S;
      if (i >= S && !mbar_wait(&empty[s], (uint32_t)((i / S - 1) & 1), limit)) {
        ok = false;
        break;
      }
      const long long q = q0 + i;
      const int rb = (int)(q % a.rblocks);
      const long long bs = q / a.rblocks;
      const int strip = (int)(bs % a.strips), b = (int)(bs / a.strips);
      const int r0 = rb * a.rows, c0 = strip * a.TW;
      mbar_expect_tx(&full[s], stage_bytes);
      const uint32_t sa = a0 + (uint32_t)s * astage, sb = b0 + (uint32_t)s * NB * BBOX;
      if constexpr (SWAP) {
#pragma unroll
        for (int kw = 0; kw < 3; ++kw)
          for (int j = 0; j < na; ++j)
            tma_load_4d(sa + kw * acopy + j * abox, &xmap, m0 + a.wa * j, c0 + kw - 1, r0 + kh - 1, b, &full[s]);
        tma_load_4d(sb, &dzmap, n0, c0, r0, b, &full[s]);
      } else {
        for (int j = 0; j < na; ++j) tma_load_4d(sa + j * abox, &dzmap, m0 + a.wa * j, c0, r0, b, &full[s]);
#pragma unroll
        for (int kw = 0; kw < 3; ++kw)
          tma_load_4d(sb + kw * BBOX, &xmap, n0, c0 + kw - 1, r0 + kh - 1, b, &full[s]);
      }
      issued = i + 1;
    }
    // every box issued has landed before the CTA can leave (on the normal
    // path the MMA lane already consumed them all and these return at once)
    for (int i = issued > S ? issued - S : 0; i < issued; ++i)
      if (!mbar_wait(&full[i % S], (uint32_t)((i / S) & 1), limit)) ok = false;
  } else if (tid == 32) {
    // ---------------- MMA issuer, K = the chunk's KC positions.  Swizzled
    // MN-major descriptors: stride byte offset = the next group of 8
    // positions (8 rows of the box), leading byte offset = the next box
    // along M (B is one box wide; its leading offset is set to the group
    // stride so that every address the descriptor can form stays inside
    // the box).  A K step of 16 positions advances two groups.
    const uint32_t idesc = umma_idesc_bf16(128, BN) | (1u << 15) | (1u << 16);
    const uint32_t ag = 16u * (uint32_t)a.wa, bg = 16u * BN;  // bytes of 8 rows
    const uint64_t aswz = (uint64_t)umma_swizzle(2 * a.wa) << 61, bswz = (uint64_t)umma_swizzle(2 * BN) << 61;
    for (int i = 0; i < NL; ++i) {
      const int s = i % S;
      if (!mbar_wait(&full[s], (uint32_t)((i / S) & 1), limit)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t sa = a0 + (uint32_t)s * astage, sb = b0 + (uint32_t)s * NB * BBOX;
#pragma unroll
      for (int kw = 0; kw < 3; ++kw) {
        const uint64_t da = umma_smem_desc(sa + (SWAP ? kw * acopy : 0u), abox, ag) | aswz;
        const uint64_t db = umma_smem_desc(sb + (SWAP ? 0u : kw * BBOX), bg, bg) | bswz;
#pragma unroll
        for (int ks = 0; ks < KC / 16; ++ks)
          tc_mma(tmem + (uint32_t)(kw * BN), da + (uint64_t)(ks * (2 * ag >> 4)), db + (uint64_t)(ks * (2 * bg >> 4)),
                 idesc, (i > 0 || ks > 0) ? 1u : 0u);
      }
      tc_commit(&empty[s]);
    }
    tc_commit(done);  // arrives once every MMA issued above has completed
  }
  __syncwarp();
  // ---------------- epilogue: lane = M row, three taps of BN columns
  if (!mbar_wait(done, 0u, limit)) ok = false;
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if (__all_sync(0xffffffffu, ok)) {
    const int r = m0 + warp * 32 + lane;  // output channel, or input channel when SWAP
#pragma unroll 1
    for (int kw = 0; kw < 3; ++kw) {
      const int t = 3 * kh + kw;
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        tc_ld<16>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kw * BN + c), v);
        if constexpr (SWAP) {  // dW[n0 + c + k][t][r]: consecutive lanes, consecutive addresses
          if (r < a.Cin) {
            float *dst = a.part + (((size_t)split * a.Cout + n0 + c) * 9 + t) * a.Cin + r;
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (n0 + c + k < a.Cout) dst[(size_t)k * 9 * a.Cin] = v[k];
          }
        } else {  // dW[r][t][n0 + c .. + 15]
          if (r < a.Cout && n0 + c < a.Cin) {
            float4 *d = reinterpret_cast<float4 *>(a.part + (((size_t)split * a.Cout + r) * 9 + t) * a.Cin + n0 + c);
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
          }
        }
      }
    }
  }
  if (!ok) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS));
  }
}

}  // namespace mdfnn

// Forward 3x3 convolution on the 5th-generation tensor cores with one staged
// input halo per channel chunk, reused by all nine taps.
//
// Geometry.  The image is cut into column strips of TW <= 64 columns; a
// strip with a one-pixel zero border, row pitch P = TW + 2, is a 1D array of
// "padded positions".  Output (r, c) of a strip is position o = r P + c
// (columns c >= TW are discarded), and tap (kh, kw) of it reads padded
// position o + kh P + kw.  A CTA computes M = 128 MT consecutive outputs
// o0 .. o0 + M - 1 for BN output channels; its halo is the R = M + 2 P + 2
// padded positions from o0 on, so every tap of every output is the halo
// shifted by kh P + kw rows.
//
// Operands.  The halo of a KC-channel chunk sits in shared memory K-major
// with rows 16 bytes apart inside each 8-channel core column (8-row groups
// 128 B apart, core columns RMAX 16 B apart), so the A operand of a tap is a
// plain descriptor at a 16-byte-aligned start: no re-gather per tap.  The
// weights of one (chunk, tap) pair, BN x KC, sit in the canonical K-major
// core-matrix layout.  One thread issues tcgen05.mma (kind::f16, BF16 in,
// FP32 accumulator in TMEM, one 128 x BN accumulator per M tile).
//
// Pipeline.  Warps 0-3 load with cp.async (halo chunk c into one of two
// halo slots with the weights of unit (c, tap 0), the weights of the other
// taps alone) and signal `hfull` / `wfull` once their copies of a unit have
// landed; warp 4 allocates TMEM and one lane issues the MMAs, committing
// each unit to `wempty` and the last tap of a chunk to `hempty`.  The
// epilogue (warps 0-3) reads TMEM with tcgen05.ld, applies bias / ReLU and
// stores through a shared-memory stage as 16-byte channel vectors.  Every
// wait is bounded; a time-out raises the error flag and the CTA still
// drains its copies and MMAs before freeing TMEM.
#pragma once

#include "mdf_nn_tc.cuh"

namespace mdfnn {

constexpr int HX_THREADS = 160;

// Halo rows reserved per core column for MT M tiles: 128 MT + 2 P + 2 with
// P <= 66, rounded up to whole 8-row groups.
template <int MT>
__host__ __device__ constexpr int halo_rmax() {
  return ((128 * MT + 2 * 66 + 2) + 7) & ~7;
}

struct HaloGeom {
  int TW, P, strips, tiles, R;
};

__host__ __device__ inline HaloGeom halo_geom(int H, int W, int MT) {
  HaloGeom g;
  g.TW = W + 2 <= 66 ? W : 64;
  g.P = g.TW + 2;
  g.strips = (W + g.TW - 1) / g.TW;
  g.tiles = (H * g.P + 128 * MT - 1) / (128 * MT);
  g.R = 128 * MT + 2 * g.P + 2;
  return g;
}

template <int BN, int KC, int MT, int S>
constexpr size_t halo_smem_bytes() {
  return (size_t)2 * halo_rmax<MT>() * KC * 2 + (size_t)S * BN * KC * 2 + (4 + 2 * S + 1) * 8 + 16;
}

template <int BN, int KC, int MT, int S>
__global__ void __launch_bounds__(HX_THREADS) k_conv_fwd_halo(ConvArgs a, int *err) {
  static_assert(BN == 16 || BN == 32 || BN == 64 || BN == 128 || BN == 256, "N tile");
  static_assert(KC == 16 || KC == 32, "channel chunk");
  static_assert(MT == 1 || MT == 2, "M tiles");
  constexpr int LAG = S >= 4 ? S - 2 : 1;  // copy groups in flight; < S and <= 9
  static_assert(LAG >= 1 && LAG < S, "look-ahead");
  constexpr int NCORE = KC / 8;
  constexpr int RMAX = halo_rmax<MT>();
  constexpr int HALO_BYTES = RMAX * KC * 2;  // one halo slot
  constexpr int W_BYTES = BN * KC * 2;       // one weight slot
  constexpr uint32_t TCOLS = MT * BN < 32 ? 32 : MT * BN;
  constexpr int CW = BN < 32 ? BN : 32;      // epilogue slice width
  constexpr int ROWS_PER_PASS = 8 * (16 / NCORE);  // 128 threads = 8 rows x NCORE cores x groups
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sH = smem;
  uint8_t *sW = smem + 2 * HALO_BYTES;
  uint64_t *hfull = reinterpret_cast<uint64_t *>(sW + S * W_BYTES);
  uint64_t *hempty = hfull + 2;
  uint64_t *wfull = hempty + 2;
  uint64_t *wempty = wfull + S;
  uint64_t *done = wempty + S;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const HaloGeom g = halo_geom(a.H, a.W, MT);
  const int tile = blockIdx.x % g.tiles, bs = blockIdx.x / g.tiles;
  const int strip = bs % g.strips, b = bs / g.strips;
  const int o0 = tile * 128 * MT;
  const int col0 = strip * g.TW;
  const int TWs = min(g.TW, a.W - col0);
  const int n0 = blockIdx.y * BN;
  const int NU = (a.Cin / KC) * 9;  // (chunk, tap) units
  const long long limit = 2000000000LL;

  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(&hfull[k], 128);
      mbar_init(&hempty[k], 1);
    }
    for (int k = 0; k < S; ++k) {
      mbar_init(&wfull[k], 128);
      mbar_init(&wempty[k], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  if (warp < 4) {
    // ---------------- producers: lane owns rows r0 + k ROWS_PER_PASS of core `core`
    const int rr = tid & 7, core = (tid >> 3) % NCORE, rg = (tid >> 3) / NCORE;
    const int r0 = rg * 8 + rr;
    auto arrive_unit = [&](int u) {
      mbar_arrive(&wfull[u % S]);
      if (u % 9 == 0) mbar_arrive(&hfull[(u / 9) & 1]);
    };
    for (int j = 0; j < NU; ++j) {
      const int c = j / 9, t = j - 9 * (j / 9);
      if (t == 0) {
        const int hs = c & 1;
        if (c >= 2 && !mbar_wait(&hempty[hs], (uint32_t)((c / 2 - 1) & 1), limit)) {
          ok = false;
          break;
        }
        uint8_t *dst0 = sH + hs * HALO_BYTES + core * (RMAX * 16);
        // padded position of this lane's first row, advanced ROWS_PER_PASS at a time
        int q = o0 + r0;
        int pr = q / g.P, pc = q - pr * g.P;
        for (int row = r0; row < g.R; row += ROWS_PER_PASS) {
          const int h = pr - 1, w = col0 + pc - 1;
          const bool v = (unsigned)h < (unsigned)a.H && (unsigned)w < (unsigned)a.W;
          const bf16 *src = v ? a.x + (((size_t)b * a.H + h) * a.W + w) * a.Cin + c * KC + core * 8 : a.x;
          cp_async16(dst0 + row * 16, src, v);
          pc += ROWS_PER_PASS;
          while (pc >= g.P) {
            pc -= g.P;
            ++pr;
          }
        }
      }
      const int ws = j % S;
      if (j >= S && !mbar_wait(&wempty[ws], (uint32_t)((j / S - 1) & 1), limit)) {
        ok = false;
        break;
      }
      uint8_t *wdst = sW + ws * W_BYTES;
      for (int r = r0; r < BN; r += ROWS_PER_PASS) {
        const int o = n0 + r;
        const bool v = o < a.Cout;
        const bf16 *src = v ? a.w + ((size_t)o * 9 + t) * a.Cin + c * KC + core * 8 : a.w;
        cp_async16(wdst + (r >> 3) * (NCORE * 128) + core * 128 + (r & 7) * 16, src, v);
      }
      cp_async_commit();
      if (j >= LAG) {
        cp_async_wait<LAG>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        arrive_unit(j - LAG);
      }
    }
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (ok)
      for (int u = NU > LAG ? NU - LAG : 0; u < NU; ++u) arrive_unit(u);
    // ---------------- epilogue
    if (!mbar_wait(done, 0u, limit)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (__all_sync(0xffffffffu, ok)) {
      float *stg = reinterpret_cast<float *>(smem) + warp * 32 * 33;  // the halo slots are free now
      const bool vb = a.y && (((a.ldy | a.yoff) & 7) == 0) && (((uintptr_t)a.y & 15) == 0);
      const bool vf = a.yf && (((a.ldy | a.yoff) & 3) == 0) && (((uintptr_t)a.yf & 15) == 0);
#pragma unroll 1
      for (int mt = 0; mt < MT; ++mt) {
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += CW) {
          float v[CW];
          tc_ld<CW>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * BN + c0), v);
#pragma unroll
          for (int e = 0; e < CW; ++e) {
            const int o = n0 + c0 + e;
            float x = v[e];
            if (a.bias && o < a.Cout) x += a.bias[o];
            if (a.relu) x = fmaxf(x, 0.f);
            stg[lane * 33 + e] = x;
          }
          __syncwarp();
          // output pixel of staged row lr (position o0 + mt 128 + 32 warp + lr)
          auto pixel = [&](int lr, size_t &m) {
            const int o = o0 + mt * 128 + warp * 32 + lr;
            const int r = o / g.P, cc = o - r * g.P;
            m = ((size_t)b * a.H + r) * a.W + col0 + cc;
            return r < a.H && cc < TWs;
          };
          if (a.y) {
            constexpr int LPR = CW / 8, RPP = 32 / LPR;
#pragma unroll
            for (int p = 0; p < 32; p += RPP) {
              const int lr = p + lane / LPR, ch = lane % LPR;
              const int oc = n0 + c0 + ch * 8;
              size_t m;
              if (pixel(lr, m) && oc < a.Cout) {
                const float *q = stg + lr * 33 + ch * 8;
                bf16 *dst = a.y + m * a.ldy + a.yoff + oc;
                if (vb) {
                  uint4 pk;
                  pk.x = pack_bf16(q[0], q[1]);
                  pk.y = pack_bf16(q[2], q[3]);
                  pk.z = pack_bf16(q[4], q[5]);
                  pk.w = pack_bf16(q[6], q[7]);
                  *reinterpret_cast<uint4 *>(dst) = pk;
                } else {
#pragma unroll
                  for (int e = 0; e < 8; ++e) dst[e] = __float2bfloat16_rn(q[e]);
                }
              }
            }
          }
          if (a.yf) {
            constexpr int LPR = CW / 4, RPP = 32 / LPR;
#pragma unroll
            for (int p = 0; p < 32; p += RPP) {
              const int lr = p + lane / LPR, ch = lane % LPR;
              const int oc = n0 + c0 + ch * 4;
              size_t m;
              if (pixel(lr, m) && oc < a.Cout) {
                const float *q = stg + lr * 33 + ch * 4;
                float *dst = a.yf + m * a.ldy + a.yoff + oc;
                if (vf) {
                  *reinterpret_cast<float4 *>(dst) = make_float4(q[0], q[1], q[2], q[3]);
                } else {
#pragma unroll
                  for (int e = 0; e < 4; ++e) dst[e] = q[e];
                }
              }
            }
          }
          __syncwarp();
        }
      }
    }
  } else if (lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = umma_idesc_bf16(128, BN);
    // halo: K-adjacent core columns RMAX x 16 B apart, 8-row groups 128 B apart;
    // weights: K-adjacent cores 128 B apart, 8-row groups NCORE x 128 B apart
    const uint32_t hlbo = RMAX * 16, hsbo = 128, wlbo = 128, wsbo = NCORE * 128;
    for (int j = 0; j < NU; ++j) {
      const int c = j / 9, t = j - 9 * (j / 9);
      const int kh = t / 3, kw = t - 3 * (t / 3);
      if (t == 0 && !mbar_wait(&hfull[c & 1], (uint32_t)((c >> 1) & 1), limit)) {
        ok = false;
        break;
      }
      if (!mbar_wait(&wfull[j % S], (uint32_t)((j / S) & 1), limit)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      // descriptors of the slots, advanced through their start-address field
      // (address / 16; shared memory stays below 256 KB, so no carry)
      const uint64_t hd = umma_smem_desc(smem_u32(sH + (c & 1) * HALO_BYTES), hlbo, hsbo);
      const uint64_t wd = umma_smem_desc(smem_u32(sW + (j % S) * W_BYTES), wlbo, wsbo);
      const uint64_t tap = (uint64_t)(kh * g.P + kw);  // rows of 16 B
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
          tc_mma(tmem + (uint32_t)(mt * BN), hd + (uint64_t)(2 * ks * RMAX + mt * 128) + tap,
                 wd + (uint64_t)(ks * 16), idesc, (j > 0 || ks > 0) ? 1u : 0u);
      }
      tc_commit(&wempty[j % S]);
      if (t == 8) tc_commit(&hempty[c & 1]);
    }
    tc_commit(done);  // arrives once every MMA issued above has completed
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

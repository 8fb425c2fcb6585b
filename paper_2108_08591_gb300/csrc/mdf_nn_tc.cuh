// Forward 3x3 convolution as an implicit GEMM on the 5th-generation tensor
// cores (tcgen05.mma, kind::f16, BF16 operands, FP32 accumulator in TMEM).
//
// Tile: 128 pixels (M, one TMEM lane each) x BN output channels (N) per CTA,
// K = 9 Cin swept 64 at a time through a ring of S shared-memory stages.
// All 128 threads gather the im2col rows of A and the weight rows of B with
// cp.async into the canonical K-major, non-swizzled layout (8-row x 16-byte
// core matrices: K-adjacent cores 128 B apart, 8-row groups 1024 B apart);
// one thread issues four K=16 MMAs per stage and commits them to the stage's
// mbarrier, which releases the stage for the next gather.  The epilogue reads
// the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31) and
// applies bias / ReLU.  Every mbarrier wait is bounded: on time-out the CTA
// records an error flag, waits (bounded) for its MMAs, frees its TMEM and
// returns.
#pragma once

#include "mdf_nn.cuh"

namespace mdfnn {

constexpr int TC_BM = 128, TC_BK = 64, TC_STAGES = 3;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;  // 16 KB per stage

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  // base offset 0, absolute LBO mode 0, layout type 0 (no swizzle)
  return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4)                      // D format: F32
         | (1u << 7)                    // A format: BF16
         | (1u << 10)                   // B format: BF16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait for the phase with the given parity; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity));
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
      smem_u32(bar)));
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of row r, K-core kc in a stage of the canonical layout.
__device__ __forceinline__ uint32_t core_off(int r, int kc) {
  return (uint32_t)((r >> 3) * 1024 + kc * 128 + (r & 7) * 16);
}

template <int BN>
__global__ void __launch_bounds__(128) k_conv_fwd_tc(ConvArgs a, int *err) {
  static_assert(BN == 16 || BN == 32 || BN == 64 || BN == 128, "N tile");
  constexpr int B_BYTES = BN * TC_BK * 2;
  constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sA = smem;                                   // S x 16 KB
  uint8_t *sB = smem + TC_STAGES * TC_A_BYTES;          // S x B_BYTES
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + TC_STAGES * B_BYTES);  // S barriers
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + TC_STAGES);
  int *sflag = reinterpret_cast<int *>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
  const int HW = a.H * a.W, M = a.B * HW, K = 9 * a.Cin;
  const int KT = (K + TC_BK - 1) / TC_BK;
  const long long limit = 2000000000LL;  // ~1 s

  if (warp == 0) {  // TMEM for the accumulator (a power of two >= 32 columns)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) mbar_init(&bars[s], 1);
    *sflag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  // this thread's 8 A rows (pixels) and 8 B rows: row = tid / 8 + 16 j, core = tid % 8
  const int kc = tid & 7, rbase = tid >> 3;
  auto load = [&](int kt, int s) {
    const int k = kt * TC_BK + kc * 8;
    const bool kv = k < K;
    const int tap = kv ? k / a.Cin : 0, ci = kv ? k - tap * a.Cin : 0;
    const int kh = tap / 3, kw = tap - kh * 3;
    uint8_t *stA = sA + s * TC_A_BYTES;
#pragma unroll
    for (int j = 0; j < TC_BM / 16; ++j) {
      const int r = rbase + 16 * j;
      const int m = m0 + r;
      bool v = kv && m < M;
      const int mm = v ? m : 0;
      const int b = mm / HW, rem = mm - b * HW, h = rem / a.W, w = rem - h * a.W;
      const int hh = h + kh - 1, ww = w + kw - 1;
      v = v && hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      const bf16 *src = v ? a.x + ((size_t)(b * a.H + hh) * a.W + ww) * a.Cin + ci : a.x;
      cp_async16(stA + core_off(r, kc), src, v);
    }
    uint8_t *stB = sB + s * B_BYTES;
#pragma unroll
    for (int j = 0; j < (BN + 15) / 16; ++j) {
      const int r = rbase + 16 * j;
      if (r < BN) {
        const int co = n0 + r;
        const bool v = kv && co < a.Cout;
        cp_async16(stB + core_off(r, kc), v ? a.w + (size_t)co * K + k : a.w, v);
      }
    }
  };

#pragma unroll
  for (int s = 0; s < TC_STAGES; ++s) {
    if (s < KT) load(s, s);
    cp_async_commit();
  }
  const uint32_t idesc = umma_idesc_bf16(TC_BM, BN);
  bool ok = true;
  int lastc = -1;  // last tile whose MMAs were committed
  for (int kt = 0; kt < KT; ++kt) {
    const int s = kt % TC_STAGES;
    cp_async_wait<TC_STAGES - 1>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t a0 = smem_u32(sA + s * TC_A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
      // K-adjacent core matrices 128 B apart (leading byte offset), 8-row
      // groups 1024 B apart (stride byte offset)
      const uint32_t lbo = 128u, sbo = 1024u;
#pragma unroll
      for (int j = 0; j < TC_BK / 16; ++j)
        tc_mma(tmem, umma_smem_desc(a0 + j * 256, lbo, sbo), umma_smem_desc(b0 + j * 256, lbo, sbo),
               idesc, (kt > 0 || j > 0) ? 1u : 0u);
      tc_commit(&bars[s]);
    }
    lastc = kt;
    // refill the stage of tile kt - 1 with tile kt - 1 + S once its MMAs are done
    const int kp = kt - 1;
    if (kp >= 0 && kp + TC_STAGES < KT) {
      const int sp = kp % TC_STAGES;
      if (!mbar_wait(&bars[sp], (uint32_t)((kp / TC_STAGES) & 1), limit)) {
        ok = false;
        *sflag = 1;
      }
      if (ok) load(kp + TC_STAGES, sp);
    }
    cp_async_commit();
    __syncthreads();
    if (*sflag) { ok = false; break; }
  }
  // MMAs complete in order: the last committed tile's barrier covers them
  // all (also on the error path, so TMEM is freed only when they are done)
  const int last = ok ? KT - 1 : lastc;
  if (last >= 0 && !mbar_wait(&bars[last % TC_STAGES], (uint32_t)((last / TC_STAGES) & 1), limit))
    ok = false;
  cp_async_wait<0>();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if (ok) {
    const int r = warp * 32 + lane;  // TMEM lane = tile row = pixel
    const int m = m0 + r;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 8) {
      float v[8];
      tc_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (m < M) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int o = n0 + c0 + e;
          if (o >= a.Cout) continue;
          float x = v[e];
          if (a.bias) x += a.bias[o];
          if (a.relu) x = fmaxf(x, 0.f);
          const size_t at = (size_t)m * a.ldy + a.yoff + o;
          if (a.y) a.y[at] = __float2bfloat16_rn(x);
          if (a.yf) a.yf[at] = x;
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS));
}

template <int BN>
constexpr size_t tc_smem_bytes() {
  return (size_t)TC_STAGES * (TC_A_BYTES + BN * TC_BK * 2) + TC_STAGES * 8 + 16;
}

}  // namespace mdfnn

// Forward 3x3 convolution as an implicit GEMM on the 5th-generation tensor
// cores (tcgen05.mma, kind::f16, BF16 operands, FP32 accumulator in TMEM).
//
// Tile: 128 pixels (M, one TMEM lane each) x BN output channels (N) per CTA,
// K = 9 Cin swept 64 at a time through a ring of S shared-memory stages.
// Warp-specialised: warps 0-3 gather the im2col rows of A and the weight
// rows of B with cp.async into the canonical K-major, non-swizzled layout
// (8-row x 16-byte core matrices: K-adjacent cores 128 B apart, 8-row groups
// 1024 B apart) and signal a stage's `full` mbarrier once their copies of it
// have landed; warp 4 allocates TMEM and one of its lanes issues four K=16
// MMAs per stage, committing them to the stage's `empty` mbarrier (and, at
// the end, to `done`).  Each producer lane owns eight fixed pixels, so the
// pixel -> (b, h, w) division happens once; the eight lanes of a shared-
// memory phase write the eight rows of one core matrix (conflict-free).  The
// epilogue (warps 0-3; warp w owns TMEM lanes 32w..32w+31) reads the
// accumulator with tcgen05.ld, applies bias / ReLU and stages 32-column
// slices through shared memory so that global stores are 16-byte vectors
// along the channel rows.  Every mbarrier wait is bounded: on time-out the
// thread raises the error flag and the CTA still waits (bounded) for its
// MMAs and copies before freeing TMEM.
#pragma once

#include "mdf_nn.cuh"

namespace mdfnn {

constexpr int TC_BM = 128, TC_BK = 64;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;  // 16 KB per stage
constexpr int TC_THREADS = 160;                // 4 producer / epilogue warps + 1 MMA warp

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

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
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
        : "r"(a), "r"(parity)
        : "memory");
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

// 32 lanes x N consecutive 32-bit TMEM columns (N = 16 or 32) into registers.
template <int N>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&v)[N]) {
  uint32_t r[N];
  if constexpr (N == 32) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
  } else {
    static_assert(N == 16, "tcgen05.ld width");
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = __uint_as_float(r[i]);
}

// Two floats as a BF16 pair (lo at the lower address), round to nearest even.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 t = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&t);
}

// Byte offset of row r, K-core kc in a stage of the canonical layout.
__device__ __forceinline__ uint32_t core_off(int r, int kc) {
  return (uint32_t)((r >> 3) * 1024 + kc * 128 + (r & 7) * 16);
}

// Producer look-ahead: a producer lane signals tile kt - LAG after issuing
// tile kt, so LAG tiles of copies are in flight and the MMA has S - LAG
// tiles of slack before a producer waits on a stage it wants to refill.
template <int S>
constexpr int tc_lag() { return S >= 4 ? S - 2 : 1; }

template <int BN, int S>
constexpr size_t tc_smem_bytes() {
  return (size_t)S * (TC_A_BYTES + BN * TC_BK * 2) + (2 * S + 1) * 8 + 16;
}

template <int BN, int S>
__global__ void __launch_bounds__(TC_THREADS) k_conv_fwd_tc(ConvArgs a, int *err) {
  static_assert(BN == 16 || BN == 32 || BN == 64 || BN == 128 || BN == 256, "N tile");
  constexpr int LAG = tc_lag<S>();
  static_assert(LAG >= 1 && LAG < S, "look-ahead");
  constexpr int B_BYTES = BN * TC_BK * 2;
  constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
  constexpr int CW = BN < 32 ? BN : 32;  // epilogue slice width (columns)
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t *sA = smem;                                   // S x 16 KB
  uint8_t *sB = smem + S * TC_A_BYTES;                  // S x B_BYTES
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + S * B_BYTES);
  uint64_t *empty = full + S;
  uint64_t *done = empty + S;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
  const int HW = a.H * a.W, M = a.B * HW, K = 9 * a.Cin;
  const int KT = (K + TC_BK - 1) / TC_BK;
  const long long limit = 2000000000LL;  // ~1 s

  if (warp == 4) {  // TMEM for the accumulator (a power of two >= 32 columns)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 128);
      mbar_init(&empty[s], 1);
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
    // ---------------- producers: lane owns rows (g0 + 2j) * 8 + rr, K core kc
    const int rr = tid & 7, kc = (tid >> 3) & 7, g0 = tid >> 6;
    int ph[8], pw[8];
    const bf16 *pp[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int m = m0 + (g0 + 2 * j) * 8 + rr;
      if (m < M) {
        const int b = m / HW, rem = m - b * HW, h = rem / a.W;
        ph[j] = h;
        pw[j] = rem - h * a.W;
        pp[j] = a.x + (size_t)m * a.Cin;
      } else {  // out of range: no tap is ever inside the image
        ph[j] = -4;
        pw[j] = -4;
        pp[j] = a.x;
      }
    }
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % S;
      if (kt >= S && !mbar_wait(&empty[s], (uint32_t)((kt / S - 1) & 1), limit)) {
        ok = false;
        break;
      }
      const int k = kt * TC_BK + kc * 8;
      const bool kv = k < K;
      const int tap = kv ? k / a.Cin : 0, ci = k - tap * a.Cin;
      const int kh = tap / 3, kw = tap - kh * 3;
      const int off = ((kh - 1) * a.W + (kw - 1)) * a.Cin + ci;
      uint8_t *stA = sA + s * TC_A_BYTES;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int hh = ph[j] + kh - 1, ww = pw[j] + kw - 1;
        const bool v = kv && (unsigned)hh < (unsigned)a.H && (unsigned)ww < (unsigned)a.W;
        cp_async16(stA + core_off((g0 + 2 * j) * 8 + rr, kc), v ? pp[j] + off : a.x, v);
      }
      uint8_t *stB = sB + s * B_BYTES;
#pragma unroll
      for (int j = 0; j < BN / 16; ++j) {
        const int r = (g0 + 2 * j) * 8 + rr, co = n0 + r;
        const bool v = kv && co < a.Cout;
        cp_async16(stB + core_off(r, kc), v ? a.w + (size_t)co * K + k : a.w, v);
      }
      cp_async_commit();
      if (kt >= LAG) {
        cp_async_wait<LAG>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive(&full[(kt - LAG) % S]);
      }
    }
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (ok)
      for (int t = KT > LAG ? KT - LAG : 0; t < KT; ++t) mbar_arrive(&full[t % S]);
    // ---------------- epilogue
    if (!mbar_wait(done, 0u, limit)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (__all_sync(0xffffffffu, ok)) {
      float *stg = reinterpret_cast<float *>(smem) + warp * 32 * 33;  // stages are free now
      const int rbase = m0 + warp * 32;
      const bool vb = a.y && (((a.ldy | a.yoff) & 7) == 0) && (((uintptr_t)a.y & 15) == 0);
      const bool vf = a.yf && (((a.ldy | a.yoff) & 3) == 0) && (((uintptr_t)a.yf & 15) == 0);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += CW) {
        float v[CW];
        tc_ld<CW>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
        for (int e = 0; e < CW; ++e) {
          const int o = n0 + c0 + e;
          float x = v[e];
          if (a.bias && o < a.Cout) x += a.bias[o];
          if (a.relu) x = fmaxf(x, 0.f);
          stg[lane * 33 + e] = x;
        }
        __syncwarp();
        if (a.y) {  // 8 channels (16 B) per lane, CW / 8 lanes per row
          constexpr int LPR = CW / 8, RPP = 32 / LPR;
#pragma unroll
          for (int p = 0; p < 32; p += RPP) {
            const int lr = p + lane / LPR, ch = lane % LPR;
            const int m = rbase + lr, o = n0 + c0 + ch * 8;
            if (m < M && o < a.Cout) {
              const float *q = stg + lr * 33 + ch * 8;
              bf16 *dst = a.y + (size_t)m * a.ldy + a.yoff + o;
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
        if (a.yf) {  // 4 channels (16 B) per lane, CW / 4 lanes per row
          constexpr int LPR = CW / 4, RPP = 32 / LPR;
#pragma unroll
          for (int p = 0; p < 32; p += RPP) {
            const int lr = p + lane / LPR, ch = lane % LPR;
            const int m = rbase + lr, o = n0 + c0 + ch * 4;
            if (m < M && o < a.Cout) {
              const float *q = stg + lr * 33 + ch * 4;
              float *dst = a.yf + (size_t)m * a.ldy + a.yoff + o;
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
  } else if (lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = umma_idesc_bf16(TC_BM, BN);
    // K-adjacent core matrices 128 B apart (leading byte offset), 8-row
    // groups 1024 B apart (stride byte offset); one K=16 step = 256 B
    const uint32_t lbo = 128u, sbo = 1024u;
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % S;
      if (!mbar_wait(&full[s], (uint32_t)((kt / S) & 1), limit)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t a0 = smem_u32(sA + s * TC_A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
      for (int j = 0; j < TC_BK / 16; ++j)
        tc_mma(tmem, umma_smem_desc(a0 + j * 256, lbo, sbo), umma_smem_desc(b0 + j * 256, lbo, sbo),
               idesc, (kt > 0 || j > 0) ? 1u : 0u);
      tc_commit(&empty[s]);
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

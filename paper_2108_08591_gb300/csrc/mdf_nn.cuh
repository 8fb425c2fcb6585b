// Kernels of the warm-start network: 3x3 convolutions as implicit GEMMs on
// the BF16 tensor cores (mma.sync m16n8k16, FP32 accumulation; operands
// staged in shared memory by cp.async and fed by ldmatrix), and the
// element-wise pieces (ReLU gradient, 2x2 average pooling, nearest 2x
// upsampling, MSE, Adam).  Activations are NHWC BF16; convolution weights
// are [Cout][3][3][Cin] BF16 with FP32 master copies.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mdfnn {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// 16-byte global -> shared copy; valid = false writes 16 zero bytes.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem),
               "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
// D += A (16x16, row-major) * B (16x8, column-major), BF16 in, FP32 out.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------------------
// Forward convolution: y[m][o] = sum_k A[m][k] W[o][k] (+ bias, ReLU), with
// m = (b, h, w) a pixel, k = (kh, kw, i) and A the zero-padded 3x3 window
// (im2col, formed on the fly).  Tile 64 pixels x 64 outputs x 32 of K per
// step, 4 warps of 32 x 32, double-buffered.  Needs Cin % 8 == 0.
// ---------------------------------------------------------------------------
struct ConvArgs {
  const bf16 *x;      // [B][H][W][Cin]
  const bf16 *w;      // [Cout][9 * Cin]
  const float *bias;  // [Cout] or null
  bf16 *y;            // output (BF16), element [m][yoff + o] with row stride ldy; nullable
  float *yf;          // output (FP32), same indexing; nullable
  int B, H, W, Cin, Cout;
  int ldy, yoff;
  int relu;
};

constexpr int CBM = 64, CBN = 64, CBK = 32, CSK = CBK + 8;  // padded smem rows (80 B)

__global__ void __launch_bounds__(128) k_conv_fwd(ConvArgs a) {
  __shared__ __align__(128) bf16 sA[2][CBM][CSK];
  __shared__ __align__(128) bf16 sB[2][CBN][CSK];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * CBM, n0 = blockIdx.y * CBN;
  const int HW = a.H * a.W, M = a.B * HW, K = 9 * a.Cin;
  const int KT = (K + CBK - 1) / CBK;
  const int q = tid & 3;  // 16-byte chunk within a 32-wide row
  int prow[2], pb[2], ph[2], pw[2];
  bool pv[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    prow[j] = (tid >> 2) + 32 * j;
    const int m = m0 + prow[j];
    pv[j] = m < M;
    const int mm = pv[j] ? m : 0;
    pb[j] = mm / HW;
    const int rem = mm - pb[j] * HW;
    ph[j] = rem / a.W;
    pw[j] = rem - ph[j] * a.W;
  }
  auto load = [&](int kt, int buf) {
    const int k = kt * CBK + q * 8;
    const bool kv = k < K;
    const int tap = kv ? k / a.Cin : 0, ci = kv ? k - tap * a.Cin : 0;
    const int kh = tap / 3, kw = tap - kh * 3;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int hh = ph[j] + kh - 1, ww = pw[j] + kw - 1;
      const bool v = pv[j] && kv && hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      const bf16 *src = v ? a.x + ((size_t)(pb[j] * a.H + hh) * a.W + ww) * a.Cin + ci : a.x;
      cp_async16(&sA[buf][prow[j]][q * 8], src, v);
      const int co = n0 + prow[j];
      const bool wv = kv && co < a.Cout;
      cp_async16(&sB[buf][prow[j]][q * 8], wv ? a.w + (size_t)co * K + k : a.w, wv);
    }
    cp_async_commit();
  };
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  load(0, 0);
  for (int kt = 0; kt < KT; ++kt) {
    if (kt + 1 < KT) {
      load(kt + 1, (kt + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int buf = kt & 1;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t af[2][4], bfr[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        ldsm_x4(af[mt], &sA[buf][wm + mt * 16 + (lane & 15)][ks * 16 + (lane >> 4) * 8]);
#pragma unroll
      for (int np = 0; np < 2; ++np)
        ldsm_x4(bfr[np], &sB[buf][wn + np * 16 + (lane & 7) + (lane >> 4) * 8][ks * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          mma16816(acc[mt][nt], af[mt], bfr[nt >> 1][(nt & 1) * 2], bfr[nt >> 1][(nt & 1) * 2 + 1]);
    }
    __syncthreads();
  }
  // epilogue: rows lane/4 (+8), column pairs (lane%4)*2
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int m = m0 + wm + mt * 16 + (lane >> 2) + half * 8;
      if (m >= M) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int o = n0 + wn + nt * 8 + (lane & 3) * 2;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (o + e >= a.Cout) continue;
          float v = acc[mt][nt][half * 2 + e];
          if (a.bias) v += a.bias[o + e];
          if (a.relu) v = fmaxf(v, 0.f);
          const size_t at = (size_t)m * a.ldy + a.yoff + o + e;
          if (a.y) a.y[at] = __float2bfloat16_rn(v);
          if (a.yf) a.yf[at] = v;
        }
      }
    }
}

// ---------------------------------------------------------------------------
// Weight gradient: dW[o][k] = sum_m dZ[m][o] A[m][k], the sum over pixels
// split into `splits` slices whose partials are reduced in a fixed order.
// Tile 64 outputs x 64 of K, 32 pixels per step; both operands go through
// ldmatrix.trans (pixels are the reduction index).  Needs Cin, Cout % 8 == 0.
// ---------------------------------------------------------------------------
struct WgradArgs {
  const bf16 *x;   // [B][H][W][Cin] layer input
  const bf16 *dz;  // [B][H][W][Cout] gradient of the pre-activation
  float *part;     // [splits][Cout][9 * Cin]
  int B, H, W, Cin, Cout;
  int pix_per_split;
};

constexpr int WBP = 32, WSK = 64 + 8;  // pixels per step; padded smem rows (144 B)

__global__ void __launch_bounds__(128) k_conv_wgrad(WgradArgs a) {
  __shared__ __align__(128) bf16 sD[2][WBP][WSK];
  __shared__ __align__(128) bf16 sX[2][WBP][WSK];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k0 = blockIdx.x * 64, o0 = blockIdx.y * 64, split = blockIdx.z;
  const int HW = a.H * a.W, M = a.B * HW, K = 9 * a.Cin;
  const int pbeg = split * a.pix_per_split;
  const int pend = min(M, pbeg + a.pix_per_split);
  const int steps = (pend - pbeg + WBP - 1) / WBP;
  const int q = tid & 7, r0 = tid >> 3;  // chunk q of rows r0, r0 + 16
  // the im2col column of this thread's chunk
  const int kc = k0 + q * 8;
  const bool kv = kc < K;
  const int tap = kv ? kc / a.Cin : 0, ci = kv ? kc - tap * a.Cin : 0;
  const int kh = tap / 3, kw = tap - kh * 3;
  const int oc = o0 + q * 8;
  const bool ov = oc < a.Cout;
  auto load = [&](int s, int buf) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = r0 + 16 * j;
      const int m = pbeg + s * WBP + r;
      const bool mv = m < pend;
      const int mm = mv ? m : 0;
      const int b = mm / HW, rem = mm - b * HW, h = rem / a.W, w = rem - h * a.W;
      cp_async16(&sD[buf][r][q * 8], mv && ov ? a.dz + (size_t)mm * a.Cout + oc : a.dz, mv && ov);
      const int hh = h + kh - 1, ww = w + kw - 1;
      const bool xv = mv && kv && hh >= 0 && hh < a.H && ww >= 0 && ww < a.W;
      cp_async16(&sX[buf][r][q * 8], xv ? a.x + ((size_t)(b * a.H + hh) * a.W + ww) * a.Cin + ci : a.x, xv);
    }
    cp_async_commit();
  };
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const int wo = (warp >> 1) * 32, wk = (warp & 1) * 32;
  if (steps > 0) load(0, 0);
  for (int s = 0; s < steps; ++s) {
    if (s + 1 < steps) {
      load(s + 1, (s + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int buf = s & 1;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t af[2][4], bfr[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)  // A' = dZ^T: rows outputs, columns pixels
        ldsm_x4_t(af[mt], &sD[buf][ks * 16 + (lane & 7) + (lane >> 4) * 8][wo + mt * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
      for (int np = 0; np < 2; ++np)  // B' = im2col: reduction over pixels, columns K
        ldsm_x4_t(bfr[np], &sX[buf][ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8][wk + np * 16 + (lane >> 4) * 8]);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          mma16816(acc[mt][nt], af[mt], bfr[nt >> 1][(nt & 1) * 2], bfr[nt >> 1][(nt & 1) * 2 + 1]);
    }
    __syncthreads();
  }
  float *out = a.part + (size_t)split * a.Cout * K;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int o = o0 + wo + mt * 16 + (lane >> 2) + half * 8;
      if (o >= a.Cout) continue;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int k = k0 + wk + nt * 8 + (lane & 3) * 2;
#pragma unroll
        for (int e = 0; e < 2; ++e)
          if (k + e < K) out[(size_t)o * K + k + e] = acc[mt][nt][half * 2 + e];
      }
    }
}

// dst[i] = sum_s part[s][i], fixed order.
__global__ void k_sum_splits(const float *__restrict__ part, int splits, long long n,
                             float *__restrict__ dst, int accumulate) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.f;
  for (int k = 0; k < splits; ++k) s += part[(long long)k * n + i];
  dst[i] = accumulate ? dst[i] + s : s;
}

// db[o] = sum_m dz[m][o]: one block per output channel, fixed tree order.
__global__ void k_bias_grad(const bf16 *__restrict__ dz, int M, int C, float *__restrict__ db) {
  __shared__ float sh[256];
  const int o = blockIdx.x;
  float s = 0.f;
  for (int m = threadIdx.x; m < M; m += blockDim.x) s += __bfloat162float(dz[(size_t)m * C + o]);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[o] = sh[0];
}

// Wt[i][t'][o] = W[o][t][i] with t' = 8 - t (spatial flip): the data gradient
// of a convolution is the forward convolution of dZ with Wt.
__global__ void k_flip_weights(const bf16 *__restrict__ w, int Cout, int Cin, bf16 *__restrict__ wt) {
  const long long n = (long long)Cout * 9 * Cin;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int o = (int)(e / (9 * Cin));
  const int rem = (int)(e - (long long)o * 9 * Cin);
  const int t = rem / Cin, i = rem - t * Cin;
  wt[((long long)i * 9 + (8 - t)) * Cout + o] = w[e];
}

// ---------------------------------------------------------------------------
// Element-wise pieces (strided channel slices: element [m][off + c])
// ---------------------------------------------------------------------------
// dz[m][c] = dy[m][dyoff + c] * (y[m][yoff + c] > 0)
__global__ void k_relu_bwd(const bf16 *dy, int lddy, int dyoff, const bf16 *y, int ldy, int yoff,
                           bf16 *dz, long long M, int C) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * C) return;
  const long long m = e / C;
  const int c = (int)(e - m * C);
  const float g = __bfloat162float(dy[m * lddy + dyoff + c]);
  dz[e] = __float2bfloat16_rn(__bfloat162float(y[m * ldy + yoff + c]) > 0.f ? g : 0.f);
}

// out[b][h][w][c] = mean of the 2x2 block of in (in: H x W, slice [off, off+C))
__global__ void k_avgpool2(const bf16 *in, int ldi, int ioff, int B, int H, int W, int C, bf16 *out) {
  const int Ho = H / 2, Wo = W / 2;
  const long long n = (long long)B * Ho * Wo * C;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int c = (int)(e % C);
  long long p = e / C;
  const int wo = (int)(p % Wo);
  p /= Wo;
  const int ho = (int)(p % Ho);
  const int b = (int)(p / Ho);
  float s = 0.f;
#pragma unroll
  for (int dh = 0; dh < 2; ++dh)
#pragma unroll
    for (int dw = 0; dw < 2; ++dw)
      s += __bfloat162float(in[((long long)(b * H + 2 * ho + dh) * W + 2 * wo + dw) * ldi + ioff + c]);
  out[e] = __float2bfloat16_rn(0.25f * s);
}

// dx[m][c] = dpool[parent(m)][c] / 4 + dskip[m][soff + c]   (dx: H x W, contiguous C)
__global__ void k_avgpool2_bwd_add(const bf16 *dpool, const bf16 *dskip, int lds, int soff, int B,
                                   int H, int W, int C, bf16 *dx) {
  const long long n = (long long)B * H * W * C;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int c = (int)(e % C);
  long long p = e / C;
  const int w = (int)(p % W);
  p /= W;
  const int h = (int)(p % H);
  const int b = (int)(p / H);
  const long long parent = ((long long)(b * (H / 2) + h / 2) * (W / 2) + w / 2) * C + c;
  float v = 0.25f * __bfloat162float(dpool[parent]);
  if (dskip) v += __bfloat162float(dskip[(e / C) * lds + soff + c]);
  dx[e] = __float2bfloat16_rn(v);
}

// out[b][2h+i][2w+j][c] = in[b][h][w][c], into a slice of width C at column 0
// of rows of stride ldo.
__global__ void k_upsample2(const bf16 *in, int B, int H, int W, int C, bf16 *out, int ldo) {
  const long long n = (long long)B * 4 * H * W * C;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int c = (int)(e % C);
  long long p = e / C;
  const int w2 = (int)(p % (2 * W));
  p /= 2 * W;
  const int h2 = (int)(p % (2 * H));
  const int b = (int)(p / (2 * H));
  out[((long long)(b * 2 * H + h2) * 2 * W + w2) * ldo + c] =
      in[((long long)(b * H + h2 / 2) * W + w2 / 2) * C + c];
}

// d[b][h][w][c] = sum of the 2x2 children of dup (slice [0, C) of stride ldu)
__global__ void k_upsample2_bwd(const bf16 *dup, int ldu, int B, int H, int W, int C, bf16 *d) {
  const long long n = (long long)B * H * W * C;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int c = (int)(e % C);
  long long p = e / C;
  const int w = (int)(p % W);
  p /= W;
  const int h = (int)(p % H);
  const int b = (int)(p / H);
  float s = 0.f;
#pragma unroll
  for (int dh = 0; dh < 2; ++dh)
#pragma unroll
    for (int dw = 0; dw < 2; ++dw)
      s += __bfloat162float(dup[((long long)(b * 2 * H + 2 * h + dh) * 2 * W + 2 * w + dw) * ldu + c]);
  d[e] = __float2bfloat16_rn(s);
}

// MSE over the first `cv` of `cp` channels: per-block partial loss (FP64)
// and dy = 2 (y - t) / (M cv) for those channels, 0 for the padding.
__global__ void k_mse(const float *y, int cp, const float *t, int cv, long long M, bf16 *dy,
                      double *part) {
  __shared__ double sh[256];
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (e < M * cp) {
    const long long m = e / cp;
    const int c = (int)(e - m * cp);
    float g = 0.f;
    if (c < cv) {
      const float d = y[e] - t[m * cv + c];
      l = (double)d * d;
      g = 2.f * d / (float)(M * cv);
    }
    dy[e] = __float2bfloat16_rn(g);
  }
  sh[threadIdx.x] = l;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Adam (Kingma & Ba 2015) on FP32 master parameters, with the BF16 copy.
__global__ void k_adam(float *p, const float *g, float *m, float *v, bf16 *pb, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (pb) pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_f32_to_bf16(const float *x, bf16 *y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

}  // namespace mdfnn

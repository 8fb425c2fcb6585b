// Warm-start network runtime: a U-Net that maps cavity parameters to an
// approximate steady (P - P0, u, v), trained on the GPU with the tensor-core
// convolution kernels of mdf_nn.cuh.  Host code here only sequences kernels
// and owns buffers.
//
// Architecture (L levels, channels C_0 .. C_{L-1}, 3x3 convolutions):
//   encoder l:  in -> conv(C_l)+ReLU -> conv(C_l)+ReLU = s_l -> (l < L-1) 2x2 avg pool
//   decoder l = L-2 .. 0:  [upsample2(level l+1 output), s_l] -> conv(C_l)+ReLU
//                          -> conv(C_l)+ReLU
//   head: conv(Cout) on the level-0 decoder output; loss = MSE over the
//   first `cout_used` output channels.
// The encoder's second convolution of level l < L-1 writes s_l straight into
// the channel slice [C_{l+1}, C_{l+1} + C_l) of the decoder's concatenation
// buffer, so no copy is made.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <map>
#include <mutex>

#include "mdf.h"
#include "mdf_nn.cuh"
#include "mdf_nn_wgrad_tc.cuh"

using namespace mdfnn;

namespace {

thread_local std::string g_ws_error = "no error";

struct Layer {
  int cin, cout, relu, level;
  long long woff, boff;  // offsets of weights / bias in the parameter vector
};

inline unsigned grid1(long long n, int b = 256) { return (unsigned)((n + b - 1) / b); }

// SplitMix64 (Steele, Lea & Flood 2014) for the weight initialisation.
inline uint64_t splitmix(uint64_t &s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct mdf_ws_s {
  int H = 0, W = 0, L = 0, cin = 0, cout = 0, cout_used = 0, maxb = 0;
  std::vector<int> C;
  std::vector<Layer> layers;  // e0a e0b e1a e1b ... d{L-2}a d{L-2}b ... d0a d0b head
  long long nparam = 0;
  cudaStream_t stream = nullptr;
  float *p32 = nullptr, *g32 = nullptr, *m = nullptr, *v = nullptr;
  bf16 *pbf = nullptr;  // BF16 copy (biases unused)
  long long adam_step = 0;
  // activations
  bf16 *xin = nullptr;
  std::vector<bf16 *> a, pool, cat, sdeep, da, db;  // per level
  float *yf = nullptr;
  // gradients / scratch
  bf16 *dyh = nullptr, *wt = nullptr, *gA = nullptr, *gB = nullptr, *gC = nullptr;
  std::vector<bf16 *> dcat;
  float *part = nullptr;
  double *lpart = nullptr;
  long long part_n = 0, wt_n = 0, gbuf_n = 0;
  std::string err = "no error";

  int Hl(int l) const { return H >> l; }
  int Wl(int l) const { return W >> l; }
  long long Ml(int l, int B) const { return (long long)B * Hl(l) * Wl(l); }
  const Layer &enc(int l, int k) const { return layers[2 * l + k]; }
  const Layer &dec(int l, int k) const { return layers[2 * L + 2 * (L - 2 - l) + k]; }
  const Layer &head() const { return layers.back(); }
};

namespace {

mdf_status wfail(mdf_ws_t w, mdf_status st, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (w) w->err = msg;
  else g_ws_error = msg;
  return st;
}

#define WCU(w, call)                                                                    \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return wfail((w), MDF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

// Forward-convolution kernel in use: 2 = tcgen05 with a staged input halo
// (default; needs Cin % 16 == 0, else kernel 1), 1 = tcgen05 with im2col
// gathers, 0 = mma.sync.
int g_conv_kernel = 2;
int g_halo_mt = 0, g_halo_kc = 0;  // halo kernel tile override (0 = automatic)
// Weight-gradient kernel: 1 = tcgen05 fed by TMA, one kernel row of taps per
// CTA (default; needs Cin % 16 == 0 and Cout % 8 == 0, else 0), 0 = mma.sync
// split-K.  On the network's layers the tcgen05 one measured 1.8-3.9x
// faster.
int g_wgrad_kernel = 1;
int g_wgrad_bn = 0;  // tcgen05 weight-gradient channel tile override (0 = automatic)
int g_wgrad_ctas = 3;  // tcgen05 weight-gradient CTAs per SM its stage count leaves room for
int g_wgrad_kc = 0;    // tcgen05 weight-gradient positions per chunk (0 = automatic)
constexpr int kMaxSmemOptin = 227 * 1024;  // dynamic shared memory a CTA may opt in to
constexpr int kSmemPerSm = 228 * 1024;     // shared memory of an SM (1 KB of it reserved per CTA)
std::mutex g_tc_mu;
std::map<int, int *> g_tc_err;  // per-device error flag of the tcgen05 kernel

int *tc_error_flag() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_tc_mu);
  int *&p = g_tc_err[dev];
  if (!p) {
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) { p = nullptr; return nullptr; }
    cudaMemset(p, 0, sizeof(int));
  }
  return p;
}

int g_tc_bn = 0, g_tc_stages = 0;  // tile override of the tcgen05 kernel (0 = automatic)

template <int BN, int S>
cudaError_t launch_tc(cudaStream_t s, const ConvArgs &a, long long M, int *err) {
  static bool configured = false;
  const size_t smem = tc_smem_bytes<BN, S>();
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_fwd_tc<BN, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid((unsigned)((M + TC_BM - 1) / TC_BM), (unsigned)((a.Cout + BN - 1) / BN));
  k_conv_fwd_tc<BN, S><<<grid, TC_THREADS, smem, s>>>(a, err);
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_tc_s(cudaStream_t s, const ConvArgs &a, long long M, int *err, int stages) {
  if (stages == 3) return launch_tc<BN, 3>(s, a, M, err);
  if (stages == 4) return launch_tc<BN, 4>(s, a, M, err);
  if (stages == 6) return launch_tc<BN, 6>(s, a, M, err);
  return cudaErrorInvalidValue;
}

// Tile of the tcgen05 kernel: N tile = the output channels rounded up to a
// power of two (16..256), halved from 256 when the pixel tiles alone do not
// fill the SMs once; ring depth 3 for N <= 32 and N = 128 (two CTAs per SM),
// 4 for N = 64 and N = 256 (measured over the network's layer shapes).
void tc_tile(long long M, int Cout, int &bn, int &stages) {
  bn = Cout <= 16 ? 16 : Cout <= 32 ? 32 : Cout <= 64 ? 64 : Cout <= 128 ? 128 : 256;
  if (bn == 256 && (M + TC_BM - 1) / TC_BM < 152) bn = 128;
  stages = (bn == 64 || bn == 256) ? 4 : 3;
  if (g_tc_bn) bn = g_tc_bn;
  if (g_tc_stages) stages = g_tc_stages;
}

template <int BN, int KC, int MT>
cudaError_t launch_halo(cudaStream_t s, const ConvArgs &a, int *err) {
  constexpr int S = 4;
  static bool configured = false;
  const size_t smem = halo_smem_bytes<BN, KC, MT, S>();
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_fwd_halo<BN, KC, MT, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const HaloGeom g = halo_geom(a.H, a.W, MT);
  const long long nx = (long long)a.B * g.strips * g.tiles;
  if (nx > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)nx, (unsigned)((a.Cout + BN - 1) / BN));
  k_conv_fwd_halo<BN, KC, MT, S><<<grid, HX_THREADS, smem, s>>>(a, err);
  return cudaGetLastError();
}

template <int BN>
cudaError_t launch_halo_bn(cudaStream_t s, const ConvArgs &a, int *err, int kc, int mt) {
  if (kc == 32) return mt == 2 ? launch_halo<BN, 32, 2>(s, a, err) : launch_halo<BN, 32, 1>(s, a, err);
  return mt == 2 ? launch_halo<BN, 16, 2>(s, a, err) : launch_halo<BN, 16, 1>(s, a, err);
}

// Tile of the halo kernel, from a sweep over the network's layer shapes
// (B = 8, 32^2 .. 256^2, Cin 16 .. 384, Cout 16 .. 256; every shape then runs
// its fastest measured tile): N tile = Cout rounded up to a power of two, at
// most 64 (more CTAs resident beat wider tiles); 16-channel chunks, 32 for
// deep layers (Cin >= 128) on images at most 64 wide; two M tiles per CTA
// when that still gives at least 1.5 CTAs per SM.
void halo_tile(const ConvArgs &a, int &bn, int &kc, int &mt) {
  bn = a.Cout <= 16 ? 16 : a.Cout <= 32 ? 32 : 64;
  kc = (a.Cin % 32 == 0 && a.Cin >= 128 && a.W <= 64) ? 32 : 16;
  const HaloGeom g2 = halo_geom(a.H, a.W, 2);
  const long long ctas = (long long)a.B * g2.strips * g2.tiles * ((a.Cout + bn - 1) / bn);
  mt = 2 * ctas >= 3 * 152 ? 2 : 1;
  if (g_tc_bn) bn = g_tc_bn;
  if (g_halo_kc && a.Cin % g_halo_kc == 0) kc = g_halo_kc;
  if (g_halo_mt) mt = g_halo_mt;
}

cudaError_t conv_fwd(cudaStream_t s, const bf16 *x, const bf16 *w, const float *bias, bf16 *y,
                     float *yf, int B, int H, int W, int Cin, int Cout, int ldy, int yoff,
                     int relu) {
  ConvArgs a{x, w, bias, y, yf, B, H, W, Cin, Cout, ldy, yoff, relu};
  const long long M = (long long)B * H * W;
  if (g_conv_kernel == 2 && Cin % 16 == 0) {
    int *err = tc_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    int bn, kc, mt;
    halo_tile(a, bn, kc, mt);
    switch (bn) {
      case 16: return launch_halo_bn<16>(s, a, err, kc, mt);
      case 32: return launch_halo_bn<32>(s, a, err, kc, mt);
      case 64: return launch_halo_bn<64>(s, a, err, kc, mt);
      case 128: return launch_halo_bn<128>(s, a, err, kc, mt);
      case 256: return launch_halo_bn<256>(s, a, err, kc, mt);
      default: return cudaErrorInvalidValue;
    }
  }
  if (g_conv_kernel >= 1) {
    int *err = tc_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    int bn, st;
    tc_tile(M, Cout, bn, st);
    switch (bn) {
      case 16: return launch_tc_s<16>(s, a, M, err, st);
      case 32: return launch_tc_s<32>(s, a, M, err, st);
      case 64: return launch_tc_s<64>(s, a, M, err, st);
      case 128: return launch_tc_s<128>(s, a, M, err, st);
      case 256: return launch_tc_s<256>(s, a, M, err, st);
      default: return cudaErrorInvalidValue;
    }
  }
  dim3 grid((unsigned)((M + CBM - 1) / CBM), (unsigned)((Cout + CBN - 1) / CBN));
  k_conv_fwd<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

int pix_per_split(long long M) { return M >= 8192 ? 2048 : 256; }

// Streaming multiprocessors of the current device (152 when the query fails).
int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      n < 1)
    return 152;
  return n;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link against the driver library); null when unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor map of an NHWC BF16 tensor [B][H][W][C] (C % 8 == 0, 16-byte
// aligned base) with boxes of bc channels (16, 32 or 64: rows of 32, 64 or
// 128 bytes, swizzled at that width) x TW columns x `rows` rows x one
// image; coordinates outside the tensor read as zero.
bool nhwc_map(CUtensorMap *m, const bf16 *p, int B, int H, int W, int C, int bc, int TW, int rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || C % 8 != 0 || (reinterpret_cast<uintptr_t>(p) & 15u) != 0) return false;
  const CUtensorMapSwizzle swz = bc == 64   ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : bc == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                            : CU_TENSOR_MAP_SWIZZLE_32B;
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  const cuuint32_t box[4] = {(cuuint32_t)bc, (cuuint32_t)TW, (cuuint32_t)rows, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(p), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool SWAP, int KC, int BN, int S>
cudaError_t launch_wgrad_tma(cudaStream_t s, const CUtensorMap &xm, const CUtensorMap &dm, const WgradTmaArgs &a,
                             int *err) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad_tma<SWAP, KC, BN, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemOptin);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int nn = SWAP ? a.Cout : a.Cin, mm = SWAP ? a.Cin : a.Cout;
  dim3 grid((unsigned)((nn + BN - 1) / BN), (unsigned)((mm + 127) / 128), (unsigned)(3 * a.splits));
  k_conv_wgrad_tma<SWAP, KC, BN, S>
      <<<grid, WG_THREADS, wgrad_tma_smem_bytes(SWAP, KC, BN, S, a.wa, a.na), s>>>(xm, dm, a, err);
  return cudaGetLastError();
}

// Pipeline of the TMA weight gradient: chunks of g_wgrad_kc positions (128
// when automatic: on every layer of the network it measured fastest or
// within 2 % of 64) and the most stages, up to 4, whose shared memory still
// lets g_wgrad_ctas CTAs share an SM, at least 2.
void wgrad_pipeline(bool swap, int bn, int wa, int na, int *kc, int *stages) {
  const size_t budget = (size_t)kSmemPerSm / (size_t)std::max(1, g_wgrad_ctas);
  *kc = g_wgrad_kc ? g_wgrad_kc : 128;
  *stages = 2;
  for (int S = 4; S > 2; --S) {
    const size_t b = wgrad_tma_smem_bytes(swap, *kc, bn, S, wa, na);
    if (b + 1024 <= budget && b <= (size_t)kMaxSmemOptin) {
      *stages = S;
      break;
    }
  }
}

// CTAs of the TMA weight gradient that fit on one SM: shared memory (1 KB
// reserved per CTA), TMEM columns (512 per SM) and threads.
int wgrad_fit(bool swap, int kc, int bn, int S, int wa, int na) {
  const int by_smem = (int)((size_t)kSmemPerSm / (wgrad_tma_smem_bytes(swap, kc, bn, S, wa, na) + 1024));
  const int tcols = 3 * bn <= 64 ? 64 : 3 * bn <= 128 ? 128 : 256;
  return std::max(1, std::min(std::min(by_smem, 512 / tcols), 2048 / WG_THREADS));
}

template <bool SWAP, int KC, int BN>
cudaError_t launch_wgrad_tma_s(cudaStream_t s, int S, const CUtensorMap &xm, const CUtensorMap &dm,
                               const WgradTmaArgs &a, int *err) {
  switch (S) {
    case 4: return launch_wgrad_tma<SWAP, KC, BN, 4>(s, xm, dm, a, err);
    case 3: return launch_wgrad_tma<SWAP, KC, BN, 3>(s, xm, dm, a, err);
    default: return launch_wgrad_tma<SWAP, KC, BN, 2>(s, xm, dm, a, err);
  }
}

template <bool SWAP, int KC>
cudaError_t launch_wgrad_tma_b(cudaStream_t s, int bn, int S, const CUtensorMap &xm, const CUtensorMap &dm,
                               const WgradTmaArgs &a, int *err) {
  return bn == 64   ? launch_wgrad_tma_s<SWAP, KC, 64>(s, S, xm, dm, a, err)
         : bn == 32 ? launch_wgrad_tma_s<SWAP, KC, 32>(s, S, xm, dm, a, err)
                    : launch_wgrad_tma_s<SWAP, KC, 16>(s, S, xm, dm, a, err);
}

template <bool SWAP>
cudaError_t launch_wgrad_tma_k(cudaStream_t s, int kc, int bn, int S, const CUtensorMap &xm, const CUtensorMap &dm,
                               const WgradTmaArgs &a, int *err) {
  return kc == 128 ? launch_wgrad_tma_b<SWAP, 128>(s, bn, S, xm, dm, a, err)
                   : launch_wgrad_tma_b<SWAP, 64>(s, bn, S, xm, dm, a, err);
}

// Largest of 64, 32, 16 channels that divides C (C % 16 == 0), or the
// override when it divides.
int wgrad_tile(int C) {
  if (g_wgrad_bn && C % g_wgrad_bn == 0) return g_wgrad_bn;
  return C % 64 == 0 ? 64 : C % 32 == 0 ? 32 : 16;
}

cudaError_t conv_wgrad(cudaStream_t s, const bf16 *x, const bf16 *dz, float *part, float *dw,
                       int B, int H, int W, int Cin, int Cout) {
  const long long M = (long long)B * H * W;
  const int pps = pix_per_split(M);
  const int splits = (int)((M + pps - 1) / pps);
  // orientation: M (128-row MMA tiles) on the channel count that leaves
  // fewer of its rows as padding (output channels on a tie), unless that
  // leaves N tiles of 16 output channels, whose MMAs are too small (64 -> 16
  // measured 83 us swapped against 63 us); the N tile divides the other one
  const long long pad_out = ((Cout + 127) / 128) * 128LL * Cin, pad_in = ((Cin + 127) / 128) * 128LL * Cout;
  const bool swap = pad_in < pad_out && Cout % 32 == 0;
  const int mext = swap ? Cin : Cout, next = swap ? Cout : Cin;
  CUtensorMap xm, dm;
  const int bn = next % 16 == 0 ? wgrad_tile(next) : 16;
  const int wa = wgrad_wa(mext), na = wgrad_na(mext);
  int kc = 128, S = 2;
  wgrad_pipeline(swap, bn, wa, na, &kc, &S);
  const int TW = wgrad_tw(W), rows = kc / TW;
  if (g_wgrad_kernel == 1 && Cin % 16 == 0 && Cout % 8 == 0 &&
      nhwc_map(&xm, x, B, H, W, Cin, swap ? wa : bn, TW, rows) &&
      nhwc_map(&dm, dz, B, H, W, Cout, swap ? bn : wa, TW, rows)) {
    int *err = tc_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    // split the chunks so that one wave fills every SM with the CTAs that
    // fit there (each tile has three kernel-row CTAs per split), within the
    // partial buffer sized for the mma.sync kernel's splits
    const int strips = (W + TW - 1) / TW, rblocks = (H + rows - 1) / rows;
    const long long nq = (long long)B * strips * rblocks;
    const long long tiles = 3LL * ((next + bn - 1) / bn) * ((mext + 127) / 128);
    long long sp = (long long)wgrad_fit(swap, kc, bn, S, wa, na) * sm_count() / tiles;  // no second wave
    sp = std::min<long long>(std::min<long long>(sp, splits), nq);
    WgradTmaArgs a{part, B, H, W, Cin, Cout, TW, rows, strips, rblocks, (int)std::max<long long>(1, sp), wa, na};
    cudaError_t e = swap ? launch_wgrad_tma_k<true>(s, kc, bn, S, xm, dm, a, err)
                         : launch_wgrad_tma_k<false>(s, kc, bn, S, xm, dm, a, err);
    if (e != cudaSuccess) return e;
    const long long n = (long long)Cout * 9 * Cin;
    k_sum_splits<<<grid1(n), 256, 0, s>>>(part, a.splits, n, dw, 0);
    return cudaGetLastError();
  }
  const int K = 9 * Cin;
  WgradArgs a{x, dz, part, B, H, W, Cin, Cout, pps};
  dim3 grid((unsigned)((K + 63) / 64), (unsigned)((Cout + 63) / 64), (unsigned)splits);
  k_conv_wgrad<<<grid, 128, 0, s>>>(a);
  const long long n = (long long)Cout * K;
  k_sum_splits<<<grid1(n), 256, 0, s>>>(part, splits, n, dw, 0);
  return cudaGetLastError();
}

long long wgrad_part_size(long long M, int Cin, int Cout) {
  const int pps = pix_per_split(M);
  return ((M + pps - 1) / pps) * (long long)Cout * 9 * Cin;
}

cudaError_t conv_dgrad(cudaStream_t s, const bf16 *dz, const bf16 *w, bf16 *wt, bf16 *dx, int B,
                       int H, int W, int Cin, int Cout) {
  const long long n = (long long)Cout * 9 * Cin;
  k_flip_weights<<<grid1(n), 256, 0, s>>>(w, Cout, Cin, wt);
  return conv_fwd(s, dz, wt, nullptr, dx, nullptr, B, H, W, Cout, Cin, Cin, 0, 0);
}

}  // namespace

extern "C" {

mdf_status mdf_ws_create(mdf_ws_t *out, int H, int W, int levels, const int *channels, int cin,
                         int cout, int cout_used, int max_batch, unsigned long long seed,
                         void *stream) {
  if (!out) return wfail(nullptr, MDF_EINVAL, "null handle pointer");
  *out = nullptr;
  if (levels < 2 || levels > 8 || !channels) return wfail(nullptr, MDF_EINVAL, "need 2..8 levels");
  if (H % (1 << (levels - 1)) || W % (1 << (levels - 1)) || H < 8 || W < 8)
    return wfail(nullptr, MDF_EINVAL, "H and W must be divisible by 2^(levels-1)");
  if (cin % 16 || cout % 16 || cout_used < 1 || cout_used > cout)
    return wfail(nullptr, MDF_EINVAL, "cin, cout must be multiples of 16, 1 <= cout_used <= cout");
  for (int l = 0; l < levels; ++l)
    if (channels[l] % 16 || channels[l] <= 0) return wfail(nullptr, MDF_EINVAL, "channels must be multiples of 16");
  if (max_batch < 1) return wfail(nullptr, MDF_EINVAL, "max_batch >= 1");
  mdf_ws_t w = new (std::nothrow) mdf_ws_s;
  if (!w) return wfail(nullptr, MDF_ENOMEM, "host allocation");
  w->H = H; w->W = W; w->L = levels; w->cin = cin; w->cout = cout; w->cout_used = cout_used;
  w->maxb = max_batch;
  w->C.assign(channels, channels + levels);
  w->stream = static_cast<cudaStream_t>(stream);
  const int L = levels;
  long long off = 0;
  auto add = [&](int ci, int co, int relu, int level) {
    Layer ly{ci, co, relu, level, off, off + (long long)co * 9 * ci};
    off = ly.boff + co;
    w->layers.push_back(ly);
  };
  int c = cin;
  for (int l = 0; l < L; ++l) {
    add(c, w->C[l], 1, l);
    add(w->C[l], w->C[l], 1, l);
    c = w->C[l];
  }
  for (int l = L - 2; l >= 0; --l) {
    add(w->C[l + 1] + w->C[l], w->C[l], 1, l);
    add(w->C[l], w->C[l], 1, l);
  }
  add(w->C[0], cout, 0, 0);
  w->nparam = off;

  // He-uniform weights (bound sqrt(6 / fan_in)), zero biases
  std::vector<float> p(w->nparam, 0.f);
  uint64_t st = seed;
  for (const Layer &ly : w->layers) {
    const double bound = std::sqrt(6.0 / (9.0 * ly.cin));
    for (long long i = 0; i < (long long)ly.cout * 9 * ly.cin; ++i) {
      const double u = (splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      p[ly.woff + i] = (float)((2.0 * u - 1.0) * bound);
    }
  }
  const int B = max_batch;
  long long part_n = 0, wt_n = 0, gbuf = 0;
  for (const Layer &ly : w->layers) {
    part_n = std::max(part_n, wgrad_part_size(w->Ml(ly.level, B), ly.cin, ly.cout));
    wt_n = std::max(wt_n, (long long)ly.cout * 9 * ly.cin);
    gbuf = std::max(gbuf, w->Ml(ly.level, B) * std::max(ly.cin, ly.cout));
  }
  w->part_n = part_n;
  w->wt_n = wt_n;
  w->gbuf_n = gbuf;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(*ptr, 0, bytes, w->stream);
  };
  const size_t np = (size_t)w->nparam;
  alloc((void **)&w->p32, np * 4);
  alloc((void **)&w->g32, np * 4);
  alloc((void **)&w->m, np * 4);
  alloc((void **)&w->v, np * 4);
  alloc((void **)&w->pbf, np * 2);
  alloc((void **)&w->xin, (size_t)w->Ml(0, B) * cin * 2);
  w->a.assign(L, nullptr); w->pool.assign(L, nullptr); w->cat.assign(L, nullptr);
  w->sdeep.assign(L, nullptr); w->da.assign(L, nullptr); w->db.assign(L, nullptr);
  w->dcat.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    const size_t Mp = (size_t)w->Ml(l, B);
    alloc((void **)&w->a[l], Mp * w->C[l] * 2);
    if (l > 0) alloc((void **)&w->pool[l], Mp * w->C[l - 1] * 2);
    if (l < L - 1) {
      alloc((void **)&w->cat[l], Mp * (w->C[l + 1] + w->C[l]) * 2);
      alloc((void **)&w->dcat[l], Mp * (w->C[l + 1] + w->C[l]) * 2);
      alloc((void **)&w->da[l], Mp * w->C[l] * 2);
      alloc((void **)&w->db[l], Mp * w->C[l] * 2);
    } else {
      alloc((void **)&w->sdeep[l], Mp * w->C[l] * 2);
    }
  }
  alloc((void **)&w->yf, (size_t)w->Ml(0, B) * cout * 4);
  alloc((void **)&w->dyh, (size_t)w->Ml(0, B) * cout * 2);
  alloc((void **)&w->wt, (size_t)wt_n * 2);
  alloc((void **)&w->gA, (size_t)gbuf * 2);
  alloc((void **)&w->gB, (size_t)gbuf * 2);
  alloc((void **)&w->gC, (size_t)gbuf * 2);
  alloc((void **)&w->part, (size_t)part_n * 4);
  alloc((void **)&w->lpart, (size_t)grid1(w->Ml(0, B) * cout) * 8);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w->p32, p.data(), np * 4, cudaMemcpyHostToDevice, w->stream);
  if (e == cudaSuccess) {
    k_f32_to_bf16<<<grid1(w->nparam), 256, 0, w->stream>>>(w->p32, w->pbf, w->nparam);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    const mdf_status s = e == cudaErrorMemoryAllocation ? MDF_ENOMEM : MDF_ECUDA;
    wfail(nullptr, s, "ws create: %s", cudaGetErrorString(e));
    mdf_ws_destroy(w);
    return s;
  }
  *out = w;
  return MDF_OK;
}

void mdf_ws_destroy(mdf_ws_t w) {
  if (!w) return;
  cudaStreamSynchronize(w->stream);
  for (void *p : {(void *)w->p32, (void *)w->g32, (void *)w->m, (void *)w->v, (void *)w->pbf,
                  (void *)w->xin, (void *)w->yf, (void *)w->dyh, (void *)w->wt, (void *)w->gA,
                  (void *)w->gB, (void *)w->gC, (void *)w->part, (void *)w->lpart})
    cudaFree(p);
  for (auto *vec : {&w->a, &w->pool, &w->cat, &w->sdeep, &w->da, &w->db, &w->dcat})
    for (bf16 *p : *vec) cudaFree(p);
  delete w;
}

long long mdf_ws_param_count(mdf_ws_t w) { return w ? w->nparam : 0; }

// Parameter vector layout: per layer in forward order (e0a, e0b, ..., e{L-1}b,
// d{L-2}a, d{L-2}b, ..., d0a, d0b, head), weights [Cout][3][3][Cin] then bias.
mdf_status mdf_ws_get_params(mdf_ws_t w, float *host, float *grad_host) {
  if (!w) return MDF_EINVAL;
  if (host) WCU(w, cudaMemcpyAsync(host, w->p32, w->nparam * 4, cudaMemcpyDeviceToHost, w->stream));
  if (grad_host) WCU(w, cudaMemcpyAsync(grad_host, w->g32, w->nparam * 4, cudaMemcpyDeviceToHost, w->stream));
  WCU(w, cudaStreamSynchronize(w->stream));
  return MDF_OK;
}

mdf_status mdf_ws_set_params(mdf_ws_t w, const float *host) {
  if (!w || !host) return MDF_EINVAL;
  WCU(w, cudaMemcpyAsync(w->p32, host, w->nparam * 4, cudaMemcpyHostToDevice, w->stream));
  k_f32_to_bf16<<<grid1(w->nparam), 256, 0, w->stream>>>(w->p32, w->pbf, w->nparam);
  WCU(w, cudaGetLastError());
  WCU(w, cudaMemsetAsync(w->m, 0, w->nparam * 4, w->stream));
  WCU(w, cudaMemsetAsync(w->v, 0, w->nparam * 4, w->stream));
  w->adam_step = 0;
  WCU(w, cudaStreamSynchronize(w->stream));
  return MDF_OK;
}

}  // extern "C"

namespace {

// Forward pass of B samples already in w->xin; output in w->yf (FP32).
mdf_status forward(mdf_ws_t w, int B) {
  const int L = w->L;
  cudaStream_t s = w->stream;
  const bf16 *in = w->xin;
  int cin = w->cin;
  for (int l = 0; l < L; ++l) {
    const Layer &la = w->enc(l, 0), &lb = w->enc(l, 1);
    const int H = w->Hl(l), W = w->Wl(l);
    if (l > 0) {  // pool s_{l-1} (a slice of cat_{l-1})
      const int ld = w->C[l] + w->C[l - 1];
      k_avgpool2<<<grid1(w->Ml(l, B) * w->C[l - 1]), 256, 0, s>>>(w->cat[l - 1], ld, w->C[l], B,
                                                                   2 * H, 2 * W, w->C[l - 1], w->pool[l]);
      in = w->pool[l];
      cin = w->C[l - 1];
    }
    WCU(w, conv_fwd(s, in, w->pbf + la.woff, w->p32 + la.boff, w->a[l], nullptr, B, H, W, cin,
                    la.cout, la.cout, 0, 1));
    if (l < L - 1)
      WCU(w, conv_fwd(s, w->a[l], w->pbf + lb.woff, w->p32 + lb.boff, w->cat[l], nullptr, B, H, W,
                      lb.cin, lb.cout, w->C[l + 1] + w->C[l], w->C[l + 1], 1));
    else
      WCU(w, conv_fwd(s, w->a[l], w->pbf + lb.woff, w->p32 + lb.boff, w->sdeep[l], nullptr, B, H, W,
                      lb.cin, lb.cout, lb.cout, 0, 1));
  }
  for (int l = L - 2; l >= 0; --l) {
    const Layer &la = w->dec(l, 0), &lb = w->dec(l, 1);
    const int H = w->Hl(l), W = w->Wl(l);
    const int ld = w->C[l + 1] + w->C[l];
    const bf16 *below = (l + 1 == L - 1) ? w->sdeep[l + 1] : w->db[l + 1];
    k_upsample2<<<grid1(w->Ml(l, B) * w->C[l + 1]), 256, 0, s>>>(below, B, H / 2, W / 2, w->C[l + 1],
                                                                  w->cat[l], ld);
    WCU(w, conv_fwd(s, w->cat[l], w->pbf + la.woff, w->p32 + la.boff, w->da[l], nullptr, B, H, W, ld,
                    la.cout, la.cout, 0, 1));
    WCU(w, conv_fwd(s, w->da[l], w->pbf + lb.woff, w->p32 + lb.boff, w->db[l], nullptr, B, H, W,
                    lb.cin, lb.cout, lb.cout, 0, 1));
  }
  const Layer &hd = w->head();
  WCU(w, conv_fwd(s, w->db[0], w->pbf + hd.woff, w->p32 + hd.boff, nullptr, w->yf, B, w->H, w->W,
                  hd.cin, hd.cout, hd.cout, 0, 0));
  return MDF_OK;
}

// Backward of one convolution: dz = dout (x) relu'(out) (or dout when linear),
// weight and bias gradients, and (when dx) the input gradient.
mdf_status conv_back(mdf_ws_t w, const Layer &ly, int B, const bf16 *x, const bf16 *out, int ldo,
                     int ooff, const bf16 *dout, int lddo, int dooff, bf16 *dz, bf16 *dx) {
  cudaStream_t s = w->stream;
  const int H = w->Hl(ly.level), W = w->Wl(ly.level);
  const long long M = w->Ml(ly.level, B);
  const bf16 *dzp = dout;
  if (ly.relu) {
    k_relu_bwd<<<grid1(M * ly.cout), 256, 0, s>>>(dout, lddo, dooff, out, ldo, ooff, dz, M, ly.cout);
    dzp = dz;
  }
  WCU(w, conv_wgrad(s, x, dzp, w->part, w->g32 + ly.woff, B, H, W, ly.cin, ly.cout));
  k_bias_grad<<<ly.cout, 256, 0, s>>>(dzp, (int)M, ly.cout, w->g32 + ly.boff);
  if (dx) WCU(w, conv_dgrad(s, dzp, w->pbf + ly.woff, w->wt, dx, B, H, W, ly.cin, ly.cout));
  return MDF_OK;
}

mdf_status backward(mdf_ws_t w, int B) {
  const int L = w->L;
  cudaStream_t s = w->stream;
  mdf_status st;
  // head (linear): dz = dyh; d(db_0) -> gA
  const Layer &hd = w->head();
  if ((st = conv_back(w, hd, B, w->db[0], nullptr, 0, 0, w->dyh, hd.cout, 0, nullptr, w->gA))) return st;
  bf16 *dout = w->gA;  // gradient of the level-l decoder output
  for (int l = 0; l <= L - 2; ++l) {
    const Layer &la = w->dec(l, 0), &lb = w->dec(l, 1);
    const int ld = w->C[l + 1] + w->C[l];
    if ((st = conv_back(w, lb, B, w->da[l], w->db[l], lb.cout, 0, dout, lb.cout, 0, w->gB, w->gC))) return st;
    if ((st = conv_back(w, la, B, w->cat[l], w->da[l], la.cout, 0, w->gC, la.cout, 0, w->gB, w->dcat[l]))) return st;
    // gradient of the tensor upsampled into cat_l: level l+1's output
    const int Hn = w->Hl(l + 1), Wn = w->Wl(l + 1);
    k_upsample2_bwd<<<grid1(w->Ml(l + 1, B) * w->C[l + 1]), 256, 0, s>>>(w->dcat[l], ld, B, Hn, Wn,
                                                                       w->C[l + 1], w->gA);
    dout = w->gA;
  }
  // encoder, deepest first; `dout` holds the gradient of s_{L-1}
  for (int l = L - 1; l >= 0; --l) {
    const Layer &la = w->enc(l, 0), &lb = w->enc(l, 1);
    const int H = w->Hl(l), W = w->Wl(l);
    const bf16 *sl;
    int lds, soff;
    if (l < L - 1) {
      // gradient of s_l = pooled path (in gA, level l+1 sized) + skip slice of dcat_l
      k_avgpool2_bwd_add<<<grid1(w->Ml(l, B) * w->C[l]), 256, 0, s>>>(
          w->gA, w->dcat[l], w->C[l + 1] + w->C[l], w->C[l + 1], B, H, W, w->C[l], w->gB);
      WCU(w, cudaMemcpyAsync(w->gA, w->gB, w->Ml(l, B) * w->C[l] * 2, cudaMemcpyDeviceToDevice, s));
      sl = w->cat[l];
      lds = w->C[l + 1] + w->C[l];
      soff = w->C[l + 1];
    } else {
      sl = w->sdeep[l];
      lds = w->C[l];
      soff = 0;
    }
    if ((st = conv_back(w, lb, B, w->a[l], sl, lds, soff, w->gA, w->C[l], 0, w->gB, w->gC))) return st;
    const bf16 *xin = l == 0 ? w->xin : w->pool[l];
    if ((st = conv_back(w, la, B, xin, w->a[l], la.cout, 0, w->gC, la.cout, 0, w->gB,
                        l == 0 ? nullptr : w->gA)))
      return st;
  }
  return MDF_OK;
}

mdf_status load_input(mdf_ws_t w, const float *x, int B) {
  const long long n = w->Ml(0, B) * w->cin;
  k_f32_to_bf16<<<grid1(n), 256, 0, w->stream>>>(x, w->xin, n);
  WCU(w, cudaGetLastError());
  return MDF_OK;
}

}  // namespace

extern "C" {

mdf_status mdf_ws_forward(mdf_ws_t w, const float *x, int B, float *y) {
  if (!w || !x || !y) return MDF_EINVAL;
  if (B < 1 || B > w->maxb) return wfail(w, MDF_EINVAL, "batch %d outside [1, %d]", B, w->maxb);
  mdf_status st = load_input(w, x, B);
  if (st == MDF_OK) st = forward(w, B);
  if (st != MDF_OK) return st;
  WCU(w, cudaMemcpyAsync(y, w->yf, w->Ml(0, B) * w->cout * 4, cudaMemcpyDeviceToDevice, w->stream));
  return MDF_OK;
}

mdf_status mdf_ws_train_step(mdf_ws_t w, const float *x, const float *t, int B, float lr,
                             double *loss) {
  if (!w || !x || !t) return MDF_EINVAL;
  if (B < 1 || B > w->maxb) return wfail(w, MDF_EINVAL, "batch %d outside [1, %d]", B, w->maxb);
  mdf_status st = load_input(w, x, B);
  if (st == MDF_OK) st = forward(w, B);
  if (st != MDF_OK) return st;
  const long long n = w->Ml(0, B) * w->cout;
  const unsigned nb = grid1(n);
  k_mse<<<nb, 256, 0, w->stream>>>(w->yf, w->cout, t, w->cout_used, w->Ml(0, B), w->dyh, w->lpart);
  WCU(w, cudaGetLastError());
  if ((st = backward(w, B))) return st;
  if (lr > 0.f) {
    ++w->adam_step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)w->adam_step), c2 = 1.f - std::pow(b2, (float)w->adam_step);
    k_adam<<<grid1(w->nparam), 256, 0, w->stream>>>(w->p32, w->g32, w->m, w->v, w->pbf, w->nparam, lr,
                                                     b1, b2, 1e-8f, c1, c2);
    WCU(w, cudaGetLastError());
  }
  if (loss) {
    std::vector<double> parts(nb);
    WCU(w, cudaMemcpyAsync(parts.data(), w->lpart, nb * 8, cudaMemcpyDeviceToHost, w->stream));
    WCU(w, cudaStreamSynchronize(w->stream));
    double sum = 0.0;
    for (double p : parts) sum += p;
    *loss = sum / (double)(w->Ml(0, B) * w->cout_used);
  }
  return MDF_OK;
}

// Raw kernels on caller-owned device buffers (for tests and benchmarks).
// x, dz, w, y, dx: BF16 arrays; yf, dw: FP32; part: FP32 scratch of
// mdf_nn_wgrad_scratch(...) floats; wt: BF16 scratch of Cout * 9 * Cin.
mdf_status mdf_nn_conv_fwd(const void *x, const void *w, const float *bias, void *y, float *yf,
                           int B, int H, int W, int Cin, int Cout, int relu, void *stream) {
  if (!x || !w || (!y && !yf) || Cin % 8 || Cout % 8 || B < 1 || H < 1 || W < 1) return MDF_EINVAL;
  return conv_fwd((cudaStream_t)stream, (const bf16 *)x, (const bf16 *)w, bias, (bf16 *)y, yf, B, H,
                  W, Cin, Cout, Cout, 0, relu) == cudaSuccess ? MDF_OK : MDF_ECUDA;
}

long long mdf_nn_wgrad_scratch(int B, int H, int W, int Cin, int Cout) {
  return wgrad_part_size((long long)B * H * W, Cin, Cout);
}

mdf_status mdf_nn_conv_wgrad(const void *x, const void *dz, float *dw, float *part, int B, int H,
                             int W, int Cin, int Cout, void *stream) {
  if (!x || !dz || !dw || !part || Cin % 8 || Cout % 8) return MDF_EINVAL;
  return conv_wgrad((cudaStream_t)stream, (const bf16 *)x, (const bf16 *)dz, part, dw, B, H, W, Cin,
                    Cout) == cudaSuccess ? MDF_OK : MDF_ECUDA;
}

mdf_status mdf_nn_conv_dgrad(const void *dz, const void *w, void *wt, void *dx, int B, int H, int W,
                             int Cin, int Cout, void *stream) {
  if (!dz || !w || !wt || !dx || Cin % 8 || Cout % 8) return MDF_EINVAL;
  return conv_dgrad((cudaStream_t)stream, (const bf16 *)dz, (const bf16 *)w, (bf16 *)wt, (bf16 *)dx, B,
                    H, W, Cin, Cout) == cudaSuccess ? MDF_OK : MDF_ECUDA;
}

// Select the forward-convolution kernel (2 tcgen05 + halo, 1 tcgen05 +
// im2col, 0 mma.sync), process-wide.
mdf_status mdf_nn_set_conv_kernel(int which) {
  if (which < 0 || which > 2) return MDF_EINVAL;
  g_conv_kernel = which;
  return MDF_OK;
}

// Weight-gradient kernel (1 tcgen05, 0 mma.sync), process-wide.
mdf_status mdf_nn_set_wgrad_kernel(int which) {
  if (which != 0 && which != 1) return MDF_EINVAL;
  g_wgrad_kernel = which;
  return MDF_OK;
}

// tcgen05 weight-gradient channel tile override (0 = automatic), process-wide.
mdf_status mdf_nn_set_wgrad_tile(int bn, int ctas_per_sm, int kc) {
  if (bn != 0 && bn != 16 && bn != 32 && bn != 64) return MDF_EINVAL;
  if (ctas_per_sm < 0 || ctas_per_sm > 16) return MDF_EINVAL;
  if (kc != 0 && kc != 64 && kc != 128) return MDF_EINVAL;
  g_wgrad_bn = bn;
  g_wgrad_ctas = ctas_per_sm ? ctas_per_sm : 3;
  g_wgrad_kc = kc;
  return MDF_OK;
}

// Halo kernel tile override (0, 0 = automatic), process-wide.
mdf_status mdf_nn_set_halo_tile(int mt, int kc) {
  if (mt != 0 && mt != 1 && mt != 2) return MDF_EINVAL;
  if (kc != 0 && kc != 16 && kc != 32) return MDF_EINVAL;
  g_halo_mt = mt;
  g_halo_kc = kc;
  return MDF_OK;
}

// Tile override of the tcgen05 kernel (0, 0 = automatic), process-wide.
mdf_status mdf_nn_set_tc_tile(int bn, int stages) {
  if (bn && bn != 16 && bn != 32 && bn != 64 && bn != 128 && bn != 256) return MDF_EINVAL;
  if (stages && stages != 3 && stages != 4 && stages != 6) return MDF_EINVAL;
  if (bn == 256 && stages == 6) return MDF_EINVAL;  // 288 KB of shared memory
  g_tc_bn = bn;
  g_tc_stages = stages;
  return MDF_OK;
}

// Read and clear the tcgen05 kernel's time-out flag of the current device
// (synchronises the device).  *flag = 1 when a bounded wait gave up.
mdf_status mdf_nn_conv_error(int *flag) {
  if (!flag) return MDF_EINVAL;
  int *p = tc_error_flag();
  if (!p) return MDF_ENOMEM;
  if (cudaDeviceSynchronize() != cudaSuccess) return MDF_ECUDA;
  if (cudaMemcpy(flag, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return MDF_ECUDA;
  if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return MDF_ECUDA;
  return MDF_OK;
}

const char *mdf_ws_last_error(mdf_ws_t w) { return w ? w->err.c_str() : g_ws_error.c_str(); }

}  // extern "C"

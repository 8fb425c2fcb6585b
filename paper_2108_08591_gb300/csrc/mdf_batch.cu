// Batched lid-driven cavities advanced to steady state by one persistent
// kernel per convergence period, captured in a CUDA graph.
//
// Every cavity is a closed box (anti-halfway bounce-back walls on all faces,
// the + face of the last axis moving with the lid velocity, Sec. 4) with its
// own side N and relaxation rates.  Nodes of all cavities live in one pool,
// cavity after cavity, each cavity padded to whole tiles of kTile nodes, so a
// tile belongs to exactly one cavity; populations are structure of arrays
// f[set][i][pool node], rest-shifted FP32.  Per step the persistent kernel
// walks the list of tiles of the cavities still running, with a bounded grid
// barrier between steps.  Every R = `check` steps a residual pass (FP64:
// r = |u^n - u^{n-R}|_2 / (R |u^n|_2) per cavity, the mean per-step relative
// change over the period, which FP32 rounding noise does not floor near
// 1e-7 as the single-step difference does), a status pass and a compaction
// pass retire converged or diverged cavities; the four kernels form one
// captured graph replayed until no cavity runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mdf.h"
#include "mdf_kernels.cuh"

namespace mdf {

constexpr int kTile = 128;  // nodes per tile = threads per block

struct CavParam {
  int N;                   // nodes per side
  int tile0;               // first tile of this cavity
  int ntiles;              // tiles of this cavity
  int pad;
  long long base;          // first pool node of this cavity
  float s1, s2;
  double s1d;
  unsigned long long mN;   // ceil(2^64 / N): floor(k / N) = mulhi(k, mN) for k < 2^32
};

// Word offsets in the barrier buffer, each counter on its own 128-byte line
// so that the arrivals, the polled generation and the tickets of even and
// odd steps do not share a line.
constexpr int kBarGen = 0, kBarArrive = 32, kBarTicket = 64, kBarWords = 128;
// Schedule 3: rounds of tiles, at the end of every step, that blocks claim
// from a ticket counter instead of taking them round-robin (8 measured
// fastest on 64 cavities, against 1 .. 24 and all tiles claimed).
#ifndef MDF_BATCH_TAIL_ROUNDS
#define MDF_BATCH_TAIL_ROUNDS 8
#endif
constexpr int kDynRounds = MDF_BATCH_TAIL_ROUNDS;
// Sleep between polls of the barrier's generation, in nanoseconds.
#ifndef MDF_BATCH_BAR_SLEEP
#define MDF_BATCH_BAR_SLEEP 256
#endif

enum CavStatus { CAV_RUNNING = 0, CAV_CONVERGED = 1, CAV_DIVERGED = 2, CAV_MAXSTEPS = 3 };

struct BatchArgs {
  float *f[2];              // population pools [nsets][Q][tot]
  long long tot;            // pool size in nodes (direction stride)
  const CavParam *cav;
  const int *tile_cav;      // cavity of every tile
  int *live;                // tile ids of running cavities
  int *n_live;
  int ncav, ntiles, with_rho;
  double lid_u[3];
  float *usave;             // [d][tot] velocity saved by the first update of a period
  double *part;             // [ntiles][2] residual partial sums
  int *badtile;             // [ntiles] non-finite flags
  int *status;              // [ncav]
  long long *steps;         // [ncav]
  double *res;              // [ncav]
  unsigned int *bar;        // [kBarArrive] arrivals, [kBarGen] generation, [kBarTicket + 32 (s & 1)]
                            // tile tickets of step s (schedule 3); one 128-byte line each
  int *err;                 // MDF_ETIMEOUT on a barrier or neighbour-wait time-out
  long long timeout;        // barrier spin limit in clock cycles
  int *prog;                // [ntiles] steps completed in the current launch (schedule 2)
  int *clock;               // steps since the batch was seeded (dither draws of FP32 rounding)
};

// Bounded grid-wide barrier for a cooperative launch after step s: the
// last block to arrive clears the ticket counter of step s + 1 and advances
// the generation; the others poll it, give up after `timeout` cycles (or
// when another block already gave up), and report.
__device__ __forceinline__ bool grid_barrier(const BatchArgs &B, int s) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = B.bar + kBarGen;
    volatile int *err = B.err;
    const unsigned int g = *gen;
    __threadfence();
    const bool last = atomicAdd(B.bar + kBarArrive, 1u) + 1u == gridDim.x;
    if (last) {
      atomicExch(B.bar + kBarArrive, 0u);
      atomicExch(B.bar + kBarTicket + 32 * ((s + 1) & 1), 0u);
      __threadfence();
      atomicAdd(B.bar + kBarGen, 1u);
    } else {
      const long long t0 = clock64();
      for (unsigned int k = 0; *gen == g; ++k) {
        if ((k & 15) == 0) {  // from the first poll on, every 16th
          if (*err) break;
          if (clock64() - t0 > B.timeout) {
            atomicCAS(B.err, 0, (int)MDF_ETIMEOUT);
            break;
          }
        }
        __nanosleep(MDF_BATCH_BAR_SLEEP);
      }
    }
    __threadfence();
    ok = *err == 0;
  }
  __syncthreads();
  return ok != 0;
}

// Wall bits of node (x, y[, z]) of a closed box of side N: bit i when the
// link along c_i leaves the box, bit 7 when it crosses the lid.
template <class L>
__device__ __forceinline__ uint8_t box_mask(const int (&p)[3], int N) {
  uint8_t m = 0;
#pragma unroll
  for (int i = 1; i < L::Q; ++i)
#pragma unroll
    for (int b = 0; b < L::D; ++b) {
      const int t = p[b] + L::c(i, b);
      if (t < 0 || t >= N) {
        m |= uint8_t(1u << i);
        if (b == L::D - 1 && t >= N) m |= 0x80u;
      }
    }
  return m;
}

// (x, y[, z]) of local node k = x + N (y + N z).  Division by N is a
// 64-bit multiply-high by mN = ceil(2^64 / N): with mN N = 2^64 + r, 0 <= r
// < N, the product k mN / 2^64 exceeds k / N by k r / (N 2^64) < 1 / N for
// every k < 2^32, so its floor is floor(k / N) exactly.
template <class L>
__device__ __forceinline__ void node_pos(int k, const CavParam &C, int (&p)[3]) {
  const unsigned q1 = (unsigned)__umul64hi((unsigned long long)(unsigned)k, C.mN);
  p[0] = k - (int)q1 * C.N;
  if (L::D == 3) {
    const unsigned q2 = (unsigned)__umul64hi((unsigned long long)q1, C.mN);
    p[1] = (int)q1 - (int)q2 * C.N;
    p[2] = (int)q2;
  } else {
    p[1] = (int)q1;
    p[2] = 0;
  }
}

template <class L>
__device__ __forceinline__ long long node_count(int N) {
  return L::D == 3 ? (long long)N * N * N : (long long)N * N;
}

// Pull every carried set at pool node idx (local node k of cavity C).
template <class L>
__device__ __forceinline__ void batch_pull(const BatchArgs &B, const float *fin, const CavParam &C,
                                           int k, float (&g)[L::D][L::Q], float (&h)[L::Q],
                                           long long &idx) {
  constexpr int D = L::D, Q = L::Q;
  int p[3];
  node_pos<L>(k, C, p);
  idx = C.base + k;
  const uint8_t m = box_mask<L>(p, C.N);
  long long src[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i)
    src[i] = idx - (L::c(i, 0) + (long long)L::c(i, 1) * C.N +
                    (D == 3 ? (long long)L::c(i, 2) * C.N * C.N : 0));
  const long long setstride = (long long)Q * B.tot;
#pragma unroll
  for (int al = 1; al <= D; ++al)
    pull_set_p<L, float, true>(fin + (long long)(B.with_rho + al - 1) * setstride, B.tot, al, idx,
                               src, m, B.lid_u, g[al - 1]);
  if (B.with_rho) pull_set_p<L, float, true>(fin, B.tot, 0, idx, src, m, B.lid_u, h);
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Schedule 2 (no grid barrier): before step s of tile `tile`, wait until
// every tile of the same cavity within one neighbour stride (N nodes in 2D,
// N^2 in 3D) has completed s steps.  Those are the tiles the pulls read, and
// the same tiles read this tile's step s - 1 values, which step s
// overwrites.  The block's threads watch the tile counters in parallel;
// each wait is bounded and a time-out raises MDF_ETIMEOUT.  The least
// advanced block waits only on tiles of lower steps, which are complete,
// so some block always progresses.
template <class L>
__device__ bool wait_neighbours(const BatchArgs &B, const CavParam &C, int tile, int s,
                                long long count) {
  const long long S = L::D == 3 ? (long long)C.N * C.N : (long long)C.N;
  const long long k0 = (long long)(tile - C.tile0) * kTile;
  const long long lo = k0 - S > 0 ? k0 - S : 0;
  const long long hi = k0 + kTile - 1 + S < count - 1 ? k0 + kTile - 1 + S : count - 1;
  const int tlo = C.tile0 + (int)(lo / kTile), thi = C.tile0 + (int)(hi / kTile);
  bool ok = true;
  volatile int *err = B.err;
  for (int j = tlo + (int)threadIdx.x; j <= thi && ok; j += blockDim.x) {
    const long long t0 = clock64();
    while (ld_acquire(B.prog + j) < s) {
      if (*err) { ok = false; break; }
      if (clock64() - t0 > B.timeout) {
        atomicCAS(B.err, 0, (int)MDF_ETIMEOUT);
        ok = false;
        break;
      }
      __nanosleep(32);
    }
  }
  __threadfence();
  return __syncthreads_and(ok) != 0;
}

// Schedule 2: publish that tile `tile` has completed `done` steps, after
// every thread's stores of it.
__device__ __forceinline__ void publish_tile(const BatchArgs &B, int tile, int done) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(B.prog + tile), "r"(done) : "memory");
  }
}

// One update of local node k of cavity C at time step t: pull from fin,
// collide (dithered FP32 rounding, drawn from the node's index in its own
// cavity and t, as a single lattice of that cavity draws), store to fout;
// with save, also store the velocity it pulled (for the residual).
template <class L>
__device__ __forceinline__ void batch_update_node(const BatchArgs &B, const float *fin, float *fout,
                                                  const CavParam &C, int k, bool save, int t) {
  constexpr int D = L::D, Q = L::Q;
  float g[D][Q], h[Q], F[D] = {}, M[D + 2];
  long long idx;
  batch_pull<L>(B, fin, C, k, g, h, idx);
  collide_node<L, float, false, true>(g, h, B.with_rho != 0, F, C.s1, C.s2, M, node_key(k, t));
  if (save)
#pragma unroll
    for (int a = 0; a < D; ++a) B.usave[a * B.tot + idx] = M[a];
  const long long setstride = (long long)Q * B.tot;
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int i = 0; i < Q; ++i)
      __stcs(fout + (long long)(B.with_rho + a) * setstride + (long long)i * B.tot + idx, g[a][i]);
  if (B.with_rho)
#pragma unroll
    for (int i = 0; i < Q; ++i) __stcs(fout + (long long)i * B.tot + idx, h[i]);
}

// `steps` updates of every running cavity; buffer `cur` holds the current
// state.  With save_first, the first update stores the velocity it pulled
// (u at the start of the period) for the residual pass.
//
// Schedule (chosen by mdf_batch_autotune): T threads per block, each thread
// updating kTile / T nodes of a tile, T apart (so every access of a warp
// stays on consecutive nodes); blocks take live tiles round-robin (SCHED 0)
// or one contiguous run of the live list each (SCHED 1), with a grid
// barrier between steps, or round-robin with per-tile step counters and
// neighbour waits instead of the barrier (SCHED 2).  SCHED 3 deals all but
// the last kDynRounds rounds of tiles round-robin and lets the blocks claim
// the rest one tile at a time from the step's ticket counter, so that a
// block that ran slow takes fewer of the tiles before the barrier.  Every
// schedule does the same arithmetic per node, so all give the same bits.
// Schedule 3 of D2Q5 at 128 threads is held to the 12 co-resident blocks
// per SM (40 registers) that schedules 0 .. 2 reach unconstrained, so its
// ticket logic costs no occupancy; 0 leaves the register count free.
template <class L, int T>
constexpr int batch_min_blocks() {
  return L::D == 2 && T == 128 ? 12 : 0;
}

template <class L, int T, int SCHED>
__global__ void __launch_bounds__(T, SCHED == 3 ? batch_min_blocks<L, T>() : 0)
    k_batch_chunk(BatchArgs B, int cur, int steps, int save_first) {
  constexpr int PER = kTile / T;
  const int nl = *B.n_live;
  const int G = (int)gridDim.x;
  const int nstat = SCHED == 3 ? max(0, nl / G - kDynRounds) * G : nl;  // tiles dealt round-robin
  const int t0 = SCHED != 1 ? (int)blockIdx.x : (int)((long long)nl * blockIdx.x / G);
  const int t1 = SCHED != 1 ? nl : (int)((long long)nl * (blockIdx.x + 1) / G);
  const int dt = SCHED != 1 ? G : 1;
  const int tclock = __ldg(B.clock);
  __shared__ int next_ticket;
  for (int s = 0; s < steps; ++s) {
    const float *fin = B.f[(cur + s) & 1];
    float *fout = B.f[(cur + s + 1) & 1];
    const bool save = save_first && s == 0;
    auto update_tile = [&](int tile) {
      const CavParam C = B.cav[B.tile_cav[tile]];
      const long long count = node_count<L>(C.N);
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        const int k = (tile - C.tile0) * kTile + r * T + (int)threadIdx.x;
        if (k < count) batch_update_node<L>(B, fin, fout, C, k, save, tclock + s);
      }
    };
    if (SCHED != 3) {
      for (int t = t0; t < t1; t += dt) {
        const int tile = B.live[t];
        if (SCHED == 2) {
          const CavParam &C = B.cav[B.tile_cav[tile]];
          if (!wait_neighbours<L>(B, C, tile, s, node_count<L>(C.N))) return;
        }
        update_tile(tile);
        if (SCHED == 2) publish_tile(B, tile, s + 1);
      }
    } else {
      // live-list positions blockIdx.x, + G, ... below nstat, then claimed
      // tickets; thread 0 claims the following ticket while the block
      // updates the current tile and publishes it afterwards
      unsigned int *ticket = B.bar + kBarTicket + 32 * (s & 1);
      int pos = (int)blockIdx.x;
      if (pos >= nstat) {
        if (threadIdx.x == 0) next_ticket = (int)atomicAdd(ticket, 1u);
        __syncthreads();
        pos = nstat + next_ticket;
      }
      while (pos < nl) {
        int npos = pos + G;
        const bool claim = npos >= nstat;  // the same in every thread
        int claimed = 0;
        if (claim) {
          __syncthreads();  // every thread has read next_ticket
          if (threadIdx.x == 0) claimed = (int)atomicAdd(ticket, 1u);
        }
        update_tile(B.live[pos]);
        if (claim) {
          if (threadIdx.x == 0) next_ticket = claimed;
          __syncthreads();
          npos = nstat + next_ticket;
        }
        pos = npos;
      }
    }
    if (SCHED != 2 && s + 1 < steps && !grid_barrier(B, s)) return;
  }
}

// Residual partial sums of every live tile against the saved velocity.
template <class L>
__global__ void __launch_bounds__(kTile) k_batch_residual(BatchArgs B, int cur) {
  constexpr int D = L::D, Q = L::Q;
  const int t = blockIdx.x;
  if (t >= *B.n_live) return;
  const int tile = B.live[t];
  const CavParam C = B.cav[B.tile_cav[tile]];
  const int k = (tile - C.tile0) * kTile + threadIdx.x;
  double v[2] = {0.0, 0.0};
  bool bad = false;
  if (k < node_count<L>(C.N)) {
    float g[D][Q], h[Q];
    long long idx;
    batch_pull<L>(B, B.f[cur], C, k, g, h, idx);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < Q; ++i) s += g[a][i];
      const double u = s, dlt = u - (double)B.usave[a * B.tot + idx];
      v[0] += dlt * dlt;
      v[1] += u * u;
      bad |= !isfinite(u);
    }
  }
  __shared__ double sh[2][kTile / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    double x = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[c][warp] = x;
  }
  const int anybad = __syncthreads_or(bad);
  if (threadIdx.x < 2) {
    double x = 0.0;
    for (int w = 0; w < kTile / 32; ++w) x += sh[threadIdx.x][w];
    B.part[(long long)tile * 2 + threadIdx.x] = x;
  }
  if (threadIdx.x == 0) B.badtile[tile] = anybad;
}

// Advances the batch's step counter by the steps of the chunk just run.
__global__ void k_batch_tick(int *clock, int steps) { *clock += steps; }

// Per cavity: residual from its tiles' partials (fixed order), step count,
// status.  One block per cavity.
__global__ void k_batch_status(BatchArgs B, int period, double tol, long long max_steps) {
  const int c = blockIdx.x;
  if (threadIdx.x != 0 || B.status[c] != CAV_RUNNING) return;
  const CavParam C = B.cav[c];
  double num = 0.0, den = 0.0;
  int bad = 0;
  for (int t = 0; t < C.ntiles; ++t) {
    num += B.part[(long long)(C.tile0 + t) * 2];
    den += B.part[(long long)(C.tile0 + t) * 2 + 1];
    bad |= B.badtile[C.tile0 + t];
  }
  const double r = den > 0.0 ? sqrt(num / den) / period : (num > 0.0 ? INFINITY : 0.0);
  B.res[c] = r;
  B.steps[c] += period;
  if (bad || !isfinite(r)) B.status[c] = CAV_DIVERGED;
  else if (r < tol) B.status[c] = CAV_CONVERGED;
  else if (B.steps[c] >= max_steps) B.status[c] = CAV_MAXSTEPS;
}

// Rebuild the live tile list from the cavity status (one block).
__global__ void k_batch_compact(BatchArgs B) {
  extern __shared__ int off[];  // [ncav + 1]
  if (threadIdx.x == 0) {
    int o = 0;
    for (int c = 0; c < B.ncav; ++c) {
      off[c] = o;
      if (B.status[c] == CAV_RUNNING) o += B.cav[c].ntiles;
    }
    off[B.ncav] = o;
    *B.n_live = o;
  }
  __syncthreads();
  for (int c = 0; c < B.ncav; ++c) {
    if (B.status[c] != CAV_RUNNING) continue;
    const CavParam C = B.cav[c];
    for (int t = threadIdx.x; t < C.ntiles; t += blockDim.x) B.live[off[c] + t] = C.tile0 + t;
  }
}

// Central difference of the seed velocity u_alpha along axis b at node p of
// a closed box of side N; beyond a wall the velocity is mirrored about the
// wall value (ghost = 2 u_wall - u), the wall lying half a cell outside the
// boundary node.  The lid moves the + face of the last axis.
template <class L>
__device__ double seed_grad(const double *u, long long NN, int N, const int (&p)[3], int alpha, int b,
                            const double (&lid)[3]) {
  const double *ua = u + (long long)(alpha - 1) * NN;
  auto at = [&](const int (&q)[3]) {
    return ua[((long long)q[2] * N + q[1]) * N + q[0]];
  };
  const double u0 = at(p);
  int q[3] = {p[0], p[1], p[2]};
  q[b] = p[b] + 1;
  const double wall_hi = b == L::D - 1 ? lid[alpha - 1] : 0.0;
  const double up = q[b] < N ? at(q) : 2.0 * wall_hi - u0;
  q[b] = p[b] - 1;
  const double dn = q[b] >= 0 ? at(q) : -u0;
  return 0.5 * (up - dn);
}

// First-order non-equilibrium part of the velocity set alpha along c_i at
// node p: the Chapman-Enskog term f^ne_i = -(w_i / s1) (c_i . grad) u_alpha,
// whose first moment -(c_s^2 / s1) grad u_alpha Eq. 3-16 inverts, with the
// trace removed, f^ne_i += (w_i / s1) c_{i,alpha} div u / d: Eq. 3-15 reads
// the trace of the first moments as pressure, so the traceless part keeps
// the seeded P, and the gradient differs only where the seed is not
// solenoidal.
template <class L>
__device__ double seed_fne(const double *u, long long NN, int N, const int (&p)[3], int alpha, int i,
                           double s1, const double (&lid)[3]) {
  if (alpha == 0 || i == 0) return 0.0;
  const int b = L::c(i, 0) != 0 ? 0 : L::c(i, 1) != 0 ? 1 : 2;
  const int sg = L::c(i, b);
  double g = seed_grad<L>(u, NN, N, p, alpha, b, lid);
  if (alpha - 1 == b) {
    double div = 0.0;
    for (int a = 0; a < L::D; ++a) div += seed_grad<L>(u, NN, N, p, a + 1, a, lid);
    g -= div / L::D;
  }
  return -(L::w(i) / s1) * sg * g;
}

// Initial state of one cavity in pull form (see k_init): f = f^eq(P, u),
// plus, with neq, the non-equilibrium part of the seed's velocity gradient.
template <class L>
__global__ void __launch_bounds__(kTile) k_batch_init(BatchArgs B, int cur, int c, const double *P,
                                                     const double *u, int neq) {
  constexpr int D = L::D, Q = L::Q;
  const CavParam C = B.cav[c];
  const long long n = (long long)blockIdx.x * kTile + threadIdx.x;
  const long long NN = node_count<L>(C.N);
  if (n >= NN) return;
  int p[3];
  node_pos<L>((int)n, C, p);
  const uint8_t m = box_mask<L>(p, C.N);
  DevArgs A;  // only the fields geq() reads
  A.Pin = P;
  A.uin = u;
  float *f = B.f[cur];
  const int nsets = D + B.with_rho;
  for (int a = 0; a < nsets; ++a) {
    const int alpha = a + 1 - B.with_rho;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float v;
      if (i != 0 && ((m >> i) & 1)) {
        v = -geq<L, float>(A, NN, n, alpha, L::opp(i));
        if (neq) v -= (float)seed_fne<L>(u, NN, C.N, p, alpha, L::opp(i), C.s1d, B.lid_u);
        if (alpha >= 1 && i == L::UP && (m & 0x80u)) v += float(2.0 * L::w(i) * B.lid_u[alpha - 1]);
      } else {
        const long long t = n + L::c(i, 0) + (long long)L::c(i, 1) * C.N +
                            (D == 3 ? (long long)L::c(i, 2) * C.N * C.N : 0);
        v = geq<L, float>(A, NN, t, alpha, i);
        if (neq) {
          const int pt[3] = {p[0] + L::c(i, 0), p[1] + L::c(i, 1), p[2] + (D == 3 ? L::c(i, 2) : 0)};
          v += (float)seed_fne<L>(u, NN, C.N, pt, alpha, i, C.s1d, B.lid_u);
        }
      }
      f[((long long)a * Q + i) * B.tot + C.base + n] = v;
    }
  }
}

// Derived fields of one cavity (dense [N^d] outputs, see write_fields).
template <class L>
__global__ void __launch_bounds__(kTile) k_batch_fields(BatchArgs B, int cur, int c, DevArgs A) {
  constexpr int D = L::D, Q = L::Q;
  const CavParam C = B.cav[c];
  const long long n = (long long)blockIdx.x * kTile + threadIdx.x;
  const long long NN = node_count<L>(C.N);
  if (n >= NN) return;
  float g[D][Q], h[Q];
  long long idx;
  batch_pull<L>(B, B.f[cur], C, (int)n, g, h, idx);
  const float F0[D] = {};  // cavities carry no body force
  write_fields<L, float>(A, n, NN, g, h, F0);
}

}  // namespace mdf

using namespace mdf;

struct mdf_batch_s {
  int d = 2, ncav = 0, ntiles = 0, with_rho = 1;
  long long tot = 0;
  double lid_u[3] = {0, 0, 0};
  cudaStream_t stream = nullptr;
  std::vector<CavParam> cav;
  BatchArgs B{};
  int cur = 0;
  int grid = 0;      // blocks of the persistent kernel
  int threads = 64;  // threads per block (kTile / threads nodes per thread)
  int sched = 3;     // 0: round-robin, 1: contiguous runs, 2: neighbour waits, 3: claimed tail
  int *host_live = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_period = 0, graph_cur = 0;
  double graph_tol = 0;
  long long graph_max = 0;
  std::string err = "no error";
};

namespace {

thread_local std::string g_batch_error = "no error";

mdf_status bfail(mdf_batch_t b, mdf_status st, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (b) b->err = msg;
  else g_batch_error = msg;
  return st;
}

#define BCU(b, call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return bfail((b), MDF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

template <class L, int T, int S>
cudaError_t launch_chunk_t(mdf_batch_t b, int steps, int save_first) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(T);
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_chunk<L, T, S>, b->B, b->cur, steps, save_first);
}

template <class L, int T>
cudaError_t launch_chunk_s(mdf_batch_t b, int steps, int save_first) {
  switch (b->sched) {
    case 0: return launch_chunk_t<L, T, 0>(b, steps, save_first);
    case 1: return launch_chunk_t<L, T, 1>(b, steps, save_first);
    case 2: {  // step counters start at zero for every launch
      cudaError_t e = cudaMemsetAsync(b->B.prog, 0, sizeof(int) * (size_t)b->ntiles, b->stream);
      return e != cudaSuccess ? e : launch_chunk_t<L, T, 2>(b, steps, save_first);
    }
    case 3: {  // so do the tickets of the first two steps
      cudaError_t e = cudaMemsetAsync(b->B.bar + kBarTicket, 0, sizeof(unsigned int) * (kBarWords - kBarTicket),
                                      b->stream);
      return e != cudaSuccess ? e : launch_chunk_t<L, T, 3>(b, steps, save_first);
    }
  }
  return cudaErrorInvalidValue;
}

template <class L>
cudaError_t launch_chunk(mdf_batch_t b, int steps, int save_first) {
  switch (b->threads) {
    case 128: return launch_chunk_s<L, 128>(b, steps, save_first);
    case 64: return launch_chunk_s<L, 64>(b, steps, save_first);
    case 32: return launch_chunk_s<L, 32>(b, steps, save_first);
  }
  return cudaErrorInvalidValue;
}

// Co-resident blocks per SM of the step kernel with this schedule.
template <class L, int T>
cudaError_t occupancy_t(int sched, int *per) {
  switch (sched) {
    case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_batch_chunk<L, T, 0>, T, 0);
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_batch_chunk<L, T, 1>, T, 0);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_batch_chunk<L, T, 2>, T, 0);
    case 3: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_batch_chunk<L, T, 3>, T, 0);
  }
  return cudaErrorInvalidValue;
}
template <class L>
cudaError_t occupancy_l(int threads, int sched, int *per) {
  switch (threads) {
    case 128: return occupancy_t<L, 128>(sched, per);
    case 64: return occupancy_t<L, 64>(sched, per);
    case 32: return occupancy_t<L, 32>(sched, per);
  }
  return cudaErrorInvalidValue;
}
cudaError_t occupancy(int d, int threads, int sched, int *per) {
  return d == 2 ? occupancy_l<D2Q5>(threads, sched, per) : occupancy_l<D3Q7>(threads, sched, per);
}

// Largest persistent grid for a schedule: co-resident blocks on every SM,
// at most one block per work unit (tile).
cudaError_t max_grid(mdf_batch_t b, int threads, int sched, int *grid) {
  int dev = 0, sms = 0, per = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = occupancy(b->d, threads, sched, &per);
  if (e == cudaSuccess) *grid = std::max(1, std::min(sms * per, b->ntiles));
  return e;
}

void drop_graph(mdf_batch_t b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

// All tiles live (plain stepping and tuning) and a cleared barrier.
mdf_status all_live(mdf_batch_t b) {
  std::vector<int> live(b->ntiles);
  for (int t = 0; t < b->ntiles; ++t) live[t] = t;
  BCU(b, cudaMemcpyAsync(b->B.live, live.data(), sizeof(int) * b->ntiles, cudaMemcpyHostToDevice, b->stream));
  BCU(b, cudaMemcpyAsync(b->B.n_live, &b->ntiles, sizeof(int), cudaMemcpyHostToDevice, b->stream));
  BCU(b, cudaMemsetAsync(b->B.err, 0, sizeof(int), b->stream));
  BCU(b, cudaMemsetAsync(b->B.bar, 0, sizeof(unsigned int) * kBarWords, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));  // `live` leaves scope
  return MDF_OK;
}

template <class L>
cudaError_t enqueue_period(mdf_batch_t b, int period, double tol, long long max_steps) {
  cudaError_t e = launch_chunk<L>(b, period, 1);
  if (e != cudaSuccess) return e;
  k_batch_tick<<<1, 1, 0, b->stream>>>(b->B.clock, period);
  const int cur_after = (b->cur + period) & 1;
  k_batch_residual<L><<<b->ntiles, kTile, 0, b->stream>>>(b->B, cur_after);
  k_batch_status<<<b->ncav, 32, 0, b->stream>>>(b->B, period, tol, max_steps);
  k_batch_compact<<<1, 256, sizeof(int) * (b->ncav + 1), b->stream>>>(b->B);
  return cudaGetLastError();
}

cudaError_t enqueue(mdf_batch_t b, int period, double tol, long long max_steps) {
  return b->d == 2 ? enqueue_period<D2Q5>(b, period, tol, max_steps)
                   : enqueue_period<D3Q7>(b, period, tol, max_steps);
}

}  // namespace

extern "C" {

mdf_status mdf_batch_create(mdf_batch_t *out, int d, int n, const int *side, const double *Re,
                            double lid_speed, const mdf_opts *o) {
  if (!out) return bfail(nullptr, MDF_EINVAL, "null handle pointer");
  *out = nullptr;
  if (d != 2 && d != 3) return bfail(nullptr, MDF_EINVAL, "d must be 2 or 3");
  if (n < 1 || n > 8192 || !side || !Re)
    return bfail(nullptr, MDF_EINVAL, "need 1 .. 8192 cavities with sides and Re");
  if (!(lid_speed > 0.0) || lid_speed > 0.5) return bfail(nullptr, MDF_EINVAL, "lid speed must lie in (0, 0.5]");
  mdf_opts opts{};
  opts.storage = MDF_F32;
  opts.with_rho = 1;
  if (o) opts = *o;
  if (opts.storage != MDF_F32) return bfail(nullptr, MDF_EUNSUPPORTED, "batched cavities use FP32 storage");
  if (opts.q != 0 && opts.q != (d == 2 ? 5 : 7))
    return bfail(nullptr, MDF_EUNSUPPORTED, "batched cavities use D2Q5 / D3Q7");
  if (opts.inplace) return bfail(nullptr, MDF_EUNSUPPORTED, "batched cavities use two population pools");
  mdf_batch_t b = new (std::nothrow) mdf_batch_s;
  if (!b) return bfail(nullptr, MDF_ENOMEM, "host allocation");
  b->d = d;
  b->ncav = n;
  b->with_rho = opts.with_rho ? 1 : 0;
  b->stream = static_cast<cudaStream_t>(opts.stream);
  b->lid_u[0] = lid_speed;
  const double cs2 = d == 2 ? 1.0 / 3.0 : 0.25;
  long long base = 0;
  int tile0 = 0;
  for (int c = 0; c < n; ++c) {
    if (side[c] < 2 || side[c] > (d == 2 ? 16384 : 1024) || !(Re[c] > 0)) {
      delete b;
      return bfail(nullptr, MDF_EINVAL, "cavity %d: bad side %d or Re %g", c, side[c], Re[c]);
    }
    const double nu = lid_speed * side[c] / Re[c];   // Re = U N / nu
    const double s1 = 1.0 / (nu / cs2 + 0.5);          // Eq. 3-13a with dt = 1
    const double s2 = 8.0 * (2.0 - s1) / (8.0 - s1);   // the rule of Sec. 4.1
    CavParam C{};
    C.N = side[c];
    const long long nn = d == 2 ? (long long)side[c] * side[c] : (long long)side[c] * side[c] * side[c];
    C.ntiles = (int)((nn + kTile - 1) / kTile);
    C.tile0 = tile0;
    C.base = base;
    C.s1 = (float)s1;
    C.s2 = (float)s2;
    C.s1d = s1;
    C.mN = ~0ull / (unsigned long long)side[c] + 1ull;  // ceil(2^64 / N)
    b->cav.push_back(C);
    tile0 += C.ntiles;
    base += (long long)C.ntiles * kTile;
  }
  b->ntiles = tile0;
  b->tot = base;
  const int nsets = d + b->with_rho, Q = d == 2 ? 5 : 7;
  BatchArgs &B = b->B;
  B.tot = b->tot;
  B.ncav = n;
  B.ntiles = b->ntiles;
  B.with_rho = b->with_rho;
  for (int k = 0; k < 3; ++k) B.lid_u[k] = b->lid_u[k];
  B.timeout = 4000000000LL;  // ~2 s at the GB300 clock
  const size_t popb = sizeof(float) * (size_t)nsets * Q * (size_t)b->tot;
  std::vector<int> tile_cav(b->ntiles);
  for (int c = 0; c < n; ++c)
    for (int t = 0; t < b->cav[c].ntiles; ++t) tile_cav[b->cav[c].tile0 + t] = c;
  cudaError_t e = cudaMalloc(&B.f[0], popb);
  if (e == cudaSuccess) e = cudaMalloc(&B.f[1], popb);
  if (e == cudaSuccess) e = cudaMalloc((void **)&B.cav, sizeof(CavParam) * n);
  if (e == cudaSuccess) e = cudaMalloc((void **)&B.tile_cav, sizeof(int) * b->ntiles);
  if (e == cudaSuccess) e = cudaMalloc(&B.live, sizeof(int) * b->ntiles);
  if (e == cudaSuccess) e = cudaMalloc(&B.n_live, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B.usave, sizeof(float) * d * (size_t)b->tot);
  if (e == cudaSuccess) e = cudaMalloc(&B.part, sizeof(double) * 2 * b->ntiles);
  if (e == cudaSuccess) e = cudaMalloc(&B.badtile, sizeof(int) * b->ntiles);
  if (e == cudaSuccess) e = cudaMalloc(&B.prog, sizeof(int) * b->ntiles);
  if (e == cudaSuccess) e = cudaMalloc(&B.status, sizeof(int) * n);
  if (e == cudaSuccess) e = cudaMalloc(&B.steps, sizeof(long long) * n);
  if (e == cudaSuccess) e = cudaMalloc(&B.res, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&B.bar, sizeof(unsigned int) * kBarWords);
  if (e == cudaSuccess) e = cudaMalloc(&B.err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B.clock, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(B.clock, 0, sizeof(int), b->stream);
  if (e == cudaSuccess) e = cudaMallocHost(&b->host_live, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(B.f[0], 0, popb, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.f[1], 0, popb, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.usave, 0, sizeof(float) * d * (size_t)b->tot, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.bar, 0, sizeof(unsigned int) * kBarWords, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.err, 0, sizeof(int), b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)B.cav, b->cav.data(), sizeof(CavParam) * n, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((void *)B.tile_cav, tile_cav.data(), sizeof(int) * b->ntiles,
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = max_grid(b, b->threads, b->sched, &b->grid);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    bfail(nullptr, e == cudaErrorMemoryAllocation ? MDF_ENOMEM : MDF_ECUDA, "batch create: %s",
          cudaGetErrorString(e));
    mdf_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? MDF_ENOMEM : MDF_ECUDA;
  }
  *out = b;
  return MDF_OK;
}

void mdf_batch_destroy(mdf_batch_t b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  BatchArgs &B = b->B;
  cudaFree(B.f[0]); cudaFree(B.f[1]); cudaFree((void *)B.cav); cudaFree((void *)B.tile_cav);
  cudaFree(B.live); cudaFree(B.n_live); cudaFree(B.usave); cudaFree(B.part); cudaFree(B.badtile);
  cudaFree(B.status); cudaFree(B.steps); cudaFree(B.res); cudaFree(B.bar); cudaFree(B.err);
  cudaFree(B.prog); cudaFree(B.clock);
  cudaFreeHost(b->host_live);
  delete b;
}

mdf_status mdf_batch_init(mdf_batch_t b, int cavity, const double *P, const double *u, int where) {
  return mdf_batch_seed(b, cavity, P, u, where, 0);
}

mdf_status mdf_batch_seed(mdf_batch_t b, int cavity, const double *P, const double *u, int where, int neq) {
  if (!b) return MDF_EINVAL;
  if (neq && !(P && u)) return bfail(b, MDF_EINVAL, "the non-equilibrium seed needs P and u");
  if (cavity < -1 || cavity >= b->ncav) return bfail(b, MDF_EINVAL, "cavity %d out of range", cavity);
  const int lo = cavity < 0 ? 0 : cavity, hi = cavity < 0 ? b->ncav : cavity + 1;
  if ((P || u) && cavity < 0) return bfail(b, MDF_EINVAL, "fields need a single cavity");
  // seeding every cavity restarts the step count of the dither draws
  if (cavity < 0) BCU(b, cudaMemsetAsync(b->B.clock, 0, sizeof(int), b->stream));
  for (int c = lo; c < hi; ++c) {
    const CavParam &C = b->cav[c];
    const long long nn = b->d == 2 ? (long long)C.N * C.N : (long long)C.N * C.N * C.N;
    const size_t bytes = sizeof(double) * (size_t)nn;
    double *dP = nullptr, *du = nullptr;
    BCU(b, cudaMallocAsync(&dP, bytes, b->stream));
    BCU(b, cudaMallocAsync(&du, bytes * b->d, b->stream));
    if (P && u) {
      const cudaMemcpyKind kind = where == MDF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
      BCU(b, cudaMemcpyAsync(dP, P, bytes, kind, b->stream));
      BCU(b, cudaMemcpyAsync(du, u, bytes * b->d, kind, b->stream));
    } else {  // rest state P = P0 = 1, u = 0
      std::vector<double> ones((size_t)nn, 1.0);
      BCU(b, cudaMemcpyAsync(dP, ones.data(), bytes, cudaMemcpyHostToDevice, b->stream));
      BCU(b, cudaMemsetAsync(du, 0, bytes * b->d, b->stream));
      BCU(b, cudaStreamSynchronize(b->stream));
    }
    const unsigned blocks = (unsigned)((nn + kTile - 1) / kTile);
    const int ne = (neq && P && u) ? 1 : 0;
    if (b->d == 2) k_batch_init<D2Q5><<<blocks, kTile, 0, b->stream>>>(b->B, b->cur, c, dP, du, ne);
    else k_batch_init<D3Q7><<<blocks, kTile, 0, b->stream>>>(b->B, b->cur, c, dP, du, ne);
    BCU(b, cudaGetLastError());
    BCU(b, cudaFreeAsync(dP, b->stream));
    BCU(b, cudaFreeAsync(du, b->stream));
  }
  BCU(b, cudaStreamSynchronize(b->stream));
  return MDF_OK;
}

mdf_status mdf_batch_run(mdf_batch_t b, double tol, long long max_steps, int check_every,
                         long long *steps_out, int *status_out, double *res_out) {
  if (!b) return MDF_EINVAL;
  if (check_every < 2 || (check_every & 1))
    return bfail(b, MDF_EINVAL, "check_every must be even and >= 2 (got %d)", check_every);
  if (max_steps < check_every) return bfail(b, MDF_EINVAL, "max_steps must be >= check_every");
  BatchArgs &B = b->B;
  // every cavity starts running, with all tiles live
  std::vector<int> zero(b->ncav, 0), live(b->ntiles);
  for (int t = 0; t < b->ntiles; ++t) live[t] = t;
  std::vector<long long> zsteps(b->ncav, 0);
  BCU(b, cudaMemcpyAsync(B.status, zero.data(), sizeof(int) * b->ncav, cudaMemcpyHostToDevice, b->stream));
  BCU(b, cudaMemcpyAsync(B.steps, zsteps.data(), sizeof(long long) * b->ncav, cudaMemcpyHostToDevice, b->stream));
  BCU(b, cudaMemcpyAsync(B.live, live.data(), sizeof(int) * b->ntiles, cudaMemcpyHostToDevice, b->stream));
  BCU(b, cudaMemcpyAsync(B.n_live, &b->ntiles, sizeof(int), cudaMemcpyHostToDevice, b->stream));
  BCU(b, cudaMemsetAsync(B.err, 0, sizeof(int), b->stream));
  BCU(b, cudaMemsetAsync(B.bar, 0, sizeof(unsigned int) * kBarWords, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));
  // one convergence period as a graph (on a non-legacy stream), else direct launches
  if (b->graph && (b->graph_period != check_every || b->graph_tol != tol || b->graph_max != max_steps ||
                   b->graph_cur != b->cur)) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (!b->graph && b->stream) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = enqueue(b, check_every, tol, max_steps);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->graph = nullptr;  // fall back to direct launches
    } else {
      b->graph_period = check_every;
      b->graph_cur = b->cur;
      b->graph_tol = tol;
      b->graph_max = max_steps;
    }
  }
  for (long long done = 0; done < max_steps; done += check_every) {
    if (b->graph) BCU(b, cudaGraphLaunch(b->graph, b->stream));
    else BCU(b, enqueue(b, check_every, tol, max_steps));
    // the period's step count is even: the current buffer index is unchanged
    BCU(b, cudaMemcpyAsync(b->host_live, B.n_live, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    int err = 0;
    BCU(b, cudaMemcpyAsync(&err, B.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCU(b, cudaStreamSynchronize(b->stream));
    if (err) return bfail(b, MDF_ETIMEOUT, "grid barrier timed out; the batch state is undefined");
    if (*b->host_live == 0) break;
  }
  std::vector<int> st(b->ncav);
  std::vector<long long> steps(b->ncav);
  std::vector<double> res(b->ncav);
  BCU(b, cudaMemcpyAsync(st.data(), B.status, sizeof(int) * b->ncav, cudaMemcpyDeviceToHost, b->stream));
  BCU(b, cudaMemcpyAsync(steps.data(), B.steps, sizeof(long long) * b->ncav, cudaMemcpyDeviceToHost, b->stream));
  BCU(b, cudaMemcpyAsync(res.data(), B.res, sizeof(double) * b->ncav, cudaMemcpyDeviceToHost, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));
  mdf_status worst = MDF_OK;
  for (int c = 0; c < b->ncav; ++c) {
    int s;
    switch (st[c]) {
      case CAV_CONVERGED: s = MDF_OK; break;
      case CAV_DIVERGED: s = MDF_EDIVERGED; break;
      default: s = MDF_ENOTCONVERGED; break;
    }
    if (status_out) status_out[c] = s;
    if (steps_out) steps_out[c] = steps[c];
    if (res_out) res_out[c] = res[c];
    if (s != MDF_OK && worst == MDF_OK) worst = (mdf_status)s;
  }
  if (worst != MDF_OK) bfail(b, worst, "some cavities did not converge; see the status array");
  return worst;
}

mdf_status mdf_batch_step(mdf_batch_t b, long long n) {
  if (!b) return MDF_EINVAL;
  if (n < 0) return bfail(b, MDF_EINVAL, "n < 0");
  mdf_status st = all_live(b);
  if (st != MDF_OK) return st;
  const int chunk = 1 << 20;
  while (n > 0) {
    const int s = (int)std::min<long long>(n, chunk);
    BCU(b, b->d == 2 ? launch_chunk<D2Q5>(b, s, 0) : launch_chunk<D3Q7>(b, s, 0));
    k_batch_tick<<<1, 1, 0, b->stream>>>(b->B.clock, s);
    BCU(b, cudaGetLastError());
    b->cur = (b->cur + s) & 1;
    n -= s;
  }
  int err = 0;
  BCU(b, cudaMemcpyAsync(&err, b->B.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));
  if (err) return bfail(b, MDF_ETIMEOUT, "grid barrier timed out");
  return MDF_OK;
}

mdf_status mdf_batch_fields(mdf_batch_t b, int cavity, const mdf_fields_t *out) {
  if (!b || !out) return MDF_EINVAL;
  if (cavity < 0 || cavity >= b->ncav) return bfail(b, MDF_EINVAL, "cavity %d out of range", cavity);
  if (out->rho && !b->with_rho) return bfail(b, MDF_EINVAL, "rho needs the alpha = 0 set");
  const CavParam &C = b->cav[cavity];
  const int d = b->d;
  const long long nn = d == 2 ? (long long)C.N * C.N : (long long)C.N * C.N * C.N;
  const int nsym = d == 2 ? 3 : 6;
  double *const host[8] = {out->P, out->u, out->rho, out->G, out->div, out->S, out->sigma, out->omega};
  const size_t count[8] = {(size_t)nn, (size_t)(d * nn), (size_t)nn, (size_t)(d * d * nn), (size_t)nn,
                           (size_t)(nsym * nn), (size_t)(nsym * nn), (size_t)((d == 2 ? 1 : 3) * nn)};
  DevArgs A;
  std::memset(&A, 0, sizeof A);
  A.s1 = C.s1d;
  A.with_rho = b->with_rho;
  double **slot[8] = {&A.P, &A.u, &A.rho, &A.G, &A.div, &A.S, &A.sigma, &A.omega};
  double *stage = nullptr;
  size_t total = 0;
  for (int k = 0; k < 8; ++k)
    if (host[k]) total += count[k];
  if (out->where == MDF_HOST && total) BCU(b, cudaMallocAsync(&stage, total * sizeof(double), b->stream));
  double *p = stage;
  for (int k = 0; k < 8; ++k)
    if (host[k]) {
      *slot[k] = out->where == MDF_HOST ? p : host[k];
      p += count[k];
    }
  const unsigned blocks = (unsigned)((nn + kTile - 1) / kTile);
  if (d == 2) k_batch_fields<D2Q5><<<blocks, kTile, 0, b->stream>>>(b->B, b->cur, cavity, A);
  else k_batch_fields<D3Q7><<<blocks, kTile, 0, b->stream>>>(b->B, b->cur, cavity, A);
  BCU(b, cudaGetLastError());
  if (out->where == MDF_HOST) {
    for (int k = 0; k < 8; ++k)
      if (host[k])
        BCU(b, cudaMemcpyAsync(host[k], *slot[k], count[k] * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    if (stage) BCU(b, cudaFreeAsync(stage, b->stream));
    BCU(b, cudaStreamSynchronize(b->stream));
  }
  return MDF_OK;
}

mdf_status mdf_batch_info(mdf_batch_t b, long long *nodes, int *tiles, int *grid) {
  if (!b) return MDF_EINVAL;
  long long nn = 0;
  for (const CavParam &C : b->cav)
    nn += b->d == 2 ? (long long)C.N * C.N : (long long)C.N * C.N * C.N;
  if (nodes) *nodes = nn;
  if (tiles) *tiles = b->ntiles;
  if (grid) *grid = b->grid;
  return MDF_OK;
}

mdf_status mdf_batch_set_timeout(mdf_batch_t b, long long cycles) {
  if (!b) return MDF_EINVAL;
  if (cycles < 0) return bfail(b, MDF_EINVAL, "timeout must be >= 0 cycles");
  b->B.timeout = cycles;
  drop_graph(b);  // the captured kernels hold the old value
  return MDF_OK;
}

mdf_status mdf_batch_set_schedule(mdf_batch_t b, int threads, int grid, int sched) {
  if (!b) return MDF_EINVAL;
  if (threads != 32 && threads != 64 && threads != 128)
    return bfail(b, MDF_EINVAL, "threads per block must be 32, 64 or 128 (got %d)", threads);
  if (sched < 0 || sched > 3) return bfail(b, MDF_EINVAL, "schedule must be 0, 1, 2 or 3 (got %d)", sched);
  int gmax = 0;
  BCU(b, max_grid(b, threads, sched, &gmax));
  if (grid < 0 || grid > gmax)
    return bfail(b, MDF_EINVAL, "grid %d outside 0 .. %d (co-resident blocks)", grid, gmax);
  b->threads = threads;
  b->sched = sched;
  b->grid = grid ? grid : gmax;
  drop_graph(b);  // the captured launch holds the old shape
  return MDF_OK;
}

mdf_status mdf_batch_get_schedule(mdf_batch_t b, int *threads, int *grid, int *sched) {
  if (!b) return MDF_EINVAL;
  if (threads) *threads = b->threads;
  if (grid) *grid = b->grid;
  if (sched) *sched = b->sched;
  return MDF_OK;
}

mdf_status mdf_batch_autotune(mdf_batch_t b, int reps, int *threads_out, int *grid_out, int *sched_out) {
  if (!b) return MDF_EINVAL;
  if (reps < 2) reps = 20;
  reps += reps & 1;  // an even chunk ends in the current buffer
  const int nsets = b->d + b->with_rho, Q = b->d == 2 ? 5 : 7;
  const size_t popb = sizeof(float) * (size_t)nsets * Q * (size_t)b->tot;
  float *save = nullptr;
  BCU(b, cudaMallocAsync(&save, popb, b->stream));
  BCU(b, cudaMemcpyAsync(save, b->B.f[b->cur], popb, cudaMemcpyDeviceToDevice, b->stream));
  mdf_status st = all_live(b);
  int dev = 0, sms = 1;
  if (st == MDF_OK && (cudaGetDevice(&dev) != cudaSuccess ||
                       cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess))
    st = bfail(b, MDF_ECUDA, "autotune: device query failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == MDF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    st = bfail(b, MDF_ECUDA, "autotune: event creation failed");
  const int old_threads = b->threads, old_sched = b->sched, old_grid = b->grid;
  int best_threads = old_threads, best_sched = old_sched, best_grid = old_grid;
  float best = 1e30f;
  const int threads_c[3] = {128, 64, 32};
  const int mult_c[10] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
  bool warmed = false;
  for (int ti = 0; ti < 3 && st == MDF_OK; ++ti)
    for (int sc = 0; sc < 4 && st == MDF_OK; ++sc) {
      int gmax = 0;
      if (max_grid(b, threads_c[ti], sc, &gmax) != cudaSuccess) {
        st = bfail(b, MDF_ECUDA, "autotune: occupancy query failed");
        break;
      }
      int last = 0;
      for (int mi = 0; mi < 10 && st == MDF_OK; ++mi) {
        const int g = std::min(gmax, mult_c[mi] * sms);
        if (g == last) continue;
        last = g;
        b->threads = threads_c[ti];
        b->sched = sc;
        b->grid = g;
        cudaError_t e = cudaMemsetAsync(b->B.bar, 0, sizeof(unsigned int) * kBarWords, b->stream);
        if (e == cudaSuccess && !warmed) {
          e = b->d == 2 ? launch_chunk<D2Q5>(b, 2, 0) : launch_chunk<D3Q7>(b, 2, 0);
          warmed = true;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = b->d == 2 ? launch_chunk<D2Q5>(b, reps, 0) : launch_chunk<D3Q7>(b, reps, 0);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        int err = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&err, b->B.err, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
          st = bfail(b, MDF_ECUDA, "autotune: %s", cudaGetErrorString(e));
        } else if (err) {
          st = bfail(b, MDF_ETIMEOUT, "autotune: grid barrier timed out");
        } else if (ms < best) {
          best = ms;
          best_threads = b->threads;
          best_sched = b->sched;
          best_grid = b->grid;
        }
      }
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // the tuning steps advanced the state: put it back
  cudaError_t e = cudaMemcpyAsync(b->B.f[b->cur], save, popb, cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess) e = cudaFreeAsync(save, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess && st == MDF_OK) st = bfail(b, MDF_ECUDA, "autotune restore: %s", cudaGetErrorString(e));
  if (st == MDF_OK) {
    b->threads = best_threads;
    b->sched = best_sched;
    b->grid = best_grid;
  } else {
    b->threads = old_threads;
    b->sched = old_sched;
    b->grid = old_grid;
  }
  drop_graph(b);
  if (st != MDF_OK) return st;
  if (threads_out) *threads_out = best_threads;
  if (grid_out) *grid_out = best_grid;
  if (sched_out) *sched_out = best_sched;
  return MDF_OK;
}

const char *mdf_batch_last_error(mdf_batch_t b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"

// Host side of the C-ABI declared in include/mdf.h: handle lifetime, buffer
// management, launch sequencing (with CUDA-graph chunks for long runs),
// FP64 reductions, checkpoints.  Every GPU step of the method runs in the
// kernels of mdf_kernels.cuh; this file only marshals and sequences.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "mdf.h"
#include "mdf_internal.h"

using namespace mdf;

namespace {

thread_local std::string g_create_error = "no error";

constexpr int kGraphChunk = 64;  // steps per captured graph (even: buffers return)

size_t storage_bytes(int st) {
  switch (st) {
    case MDF_F32: return 4;
    case MDF_F16: return 2;
    case MDF_BF16: return 2;
    case MDF_F64: return 8;
    case MDF_F16EQ: return 2;
    case MDF_BF16EQ: return 2;
  }
  return 0;
}

bool eq_storage(int st) { return st == MDF_F16EQ || st == MDF_BF16EQ; }

// Launch shape defaults of the update kernel, per lattice and storage, from
// a sweep on GB300 (4096^2 D2Q5 x 3 and 512^3 D3Q7 x 4; CUDA-event timing):
//   2D: vector kernel, 4 nodes per thread, 128 threads (FP32 6.91 TB/s,
//       FP16 6.80 TB/s, BF16 6.64 TB/s); FP64 2 nodes per thread.
//   3D: FP32 one node per thread, 256 threads (6.94 TB/s): with 28
//       populations per node the vector kernel's register pressure costs
//       more than its saved instructions; rest-shifted 16-bit 4 nodes per
//       thread, 128 threads, populations kept packed in registers (FP16
//       5.82 TB/s; 4.35 with the FP32-copy kernel at 8 nodes and 64 threads).
//   Equilibrium-shifted 16-bit: 2 nodes per thread (one FP32 pair), 64
//       threads in 2D (5.43 TB/s) and 128 in 3D (5.39 TB/s).
// mdf_autotune() measures the candidates for a given handle instead.
// Widest vector kernel built for a lattice (wider requests are clamped to
// it): 8 for 2D 16-bit, 4 otherwise; in 3D, where the wider kernels spill
// registers (FP32 with 4 nodes per thread: 424-1012 B at the 96-register
// budget of the 2D kernel), 4 for rest-shifted 16-bit and FP64 and 2 for
// FP32 and the equilibrium-shifted codecs.
int max_vx(int d, int storage, bool inplace) {
  (void)inplace;
  const bool s16 = storage == MDF_F16 || storage == MDF_BF16;
  if (d == 2) return s16 ? 8 : 4;
  return (storage == MDF_F32 || eq_storage(storage)) ? 2 : 4;
}
int default_vx(int d, int storage) {
  if (eq_storage(storage)) return 2;
  if (d == 3) return (storage == MDF_F16 || storage == MDF_BF16) ? 4 : 1;
  return storage == MDF_F64 ? 2 : 4;
}
// Launch shape of the in-place AA kernels (measured at 4096^2 and 512^3 on
// GB300): 2D FP32 4 nodes per thread (56.8 GLUPS, 56.3 with 2); 2D 16-bit
// 4 (92.0, 76.3 with 8); 3D FP32 2 (30.1, 28.1 with 1); 3D 16-bit 4 with
// 128 threads (39.8, 37.9 with 8 nodes and 64 threads); FP64 2.
int default_vx_aa(int d, int storage) {
  if (storage == MDF_F64) return 2;
  if (d == 3) return (storage == MDF_F16 || storage == MDF_BF16) ? 4 : 2;
  return 4;
}
int default_block_aa(int d, int storage) {
  if (d == 3) return (storage == MDF_F16 || storage == MDF_BF16) ? 128 : 256;
  return 128;
}
int default_block(int d, int storage) {
  if (eq_storage(storage)) return d == 3 ? 128 : 64;
  if (d == 3 && (storage == MDF_F16 || storage == MDF_BF16)) return 128;
  return d == 3 ? 256 : 128;
}

}  // namespace

struct mdf_s {
  int d = 0, q = 0, nsets = 0, with_rho = 0, storage = 0;
  int vx = 1, block = 128;  // update-kernel launch shape
  int nx = 0, ny = 0, nz = 0, px = 0;
  long long plane = 0, N = 0;
  double s0 = 1, s1 = 1, s2 = 1;
  mdf_bc bc{};
  bool walls = false;
  cudaStream_t stream = nullptr;
  void *cur = nullptr, *nxt = nullptr;  // population buffers
  uint8_t *mask = nullptr;
  void *force = nullptr;  // FP32, or FP64 with FP64 storage
  int forcing = MDF_FORCING_EQ321;  // forcing scheme of the update
  double *stage = nullptr;  // staging for host inputs/outputs
  size_t stage_bytes = 0;
  double *uprev = nullptr;  // residual memory [d][N]
  bool have_prev = false;
  double *partials = nullptr, *result = nullptr;
  int *nonfinite = nullptr;
  long long step = 0;
  int *clock = nullptr;     // device copy of `step` for the dither draws of a launch group
  long long key_base = 0;   // global index of local node 0 (slabs of a larger lattice)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // chunk starting from buffer 0 / 1
  void *buf[2] = {nullptr, nullptr};
  bool inplace = false;  // one buffer, AA pattern (buf[1] unused)
  int parity = 0;        // AA layout of the current state: 0 even, 1 odd
  void *mac[2] = {nullptr, nullptr};  // node moments of equilibrium-shifted storage
  int kmom = 0;                       // moment slots per node (0 for other storage)
  std::string err = "no error";

  size_t pop_bytes() const { return (size_t)nsets * q * (size_t)plane * storage_bytes(storage); }
  size_t mom_bytes() const { return (size_t)kmom * (size_t)plane * sizeof(float); }
  int cur_index() const { return cur == buf[0] ? 0 : 1; }
};

namespace {

mdf_status fail(mdf_t h, mdf_status st, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (h) h->err = msg;
  else g_create_error = msg;
  return st;
}

#define CU(h, call)                                                                     \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail((h), MDF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

DevArgs base_args(const mdf_t h) {
  DevArgs a;
  std::memset(&a, 0, sizeof a);
  a.fin = h->cur;
  a.fout = h->nxt;  // == cur for the in-place AA pattern
  a.aa = h->inplace ? 1 + h->parity : 0;
  a.mask = h->walls ? h->mask : nullptr;
  a.force = h->force;
  a.scheme2 = (h->forcing == MDF_FORCING_SCHEME2 && h->force) ? 1 : 0;
  a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.px = h->px;
  a.plane = h->plane;
  a.with_rho = h->with_rho;
  a.vx = h->vx;
  a.block = h->block;
  a.s1 = h->s1; a.s2 = h->s2;
  a.s1f = (float)h->s1; a.s2f = (float)h->s2;
  for (int b = 0; b < 3; ++b) a.lid_u[b] = h->bc.lid ? h->bc.lid_u[b] : 0.0;
  a.min = h->mac[h->cur_index()];
  a.mout = h->mac[1 - h->cur_index()];
  a.partials = h->partials;
  a.result = h->result;
  a.nonfinite = h->nonfinite;
  a.uprev = h->uprev;
  a.clock = h->clock;
  a.tk = 0;
  a.key_base = h->key_base;
  return a;
}

cudaError_t launch_update(const mdf_t h, int mode, const DevArgs &a) {
  return lattice_launch(h->d, h->q)->update(h->storage, mode, h->walls, a, h->stream);
}

cudaError_t launch_reduce(const mdf_t h, int kind, const DevArgs &a) {
  return lattice_launch(h->d, h->q)->reduce(h->storage, h->walls, kind, a, h->stream);
}

void drop_graphs(mdf_t h) {
  for (auto &g : h->graph)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

mdf_status ensure_stage(mdf_t h, size_t bytes) {
  if (h->stage_bytes >= bytes) return MDF_OK;
  if (h->stage) { cudaStreamSynchronize(h->stream); cudaFree(h->stage); h->stage = nullptr; }
  h->stage_bytes = 0;
  cudaError_t e = cudaMalloc(&h->stage, bytes);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(h, MDF_ENOMEM, "staging %zu bytes: %s", bytes, cudaGetErrorString(e)); }
  h->stage_bytes = bytes;
  return MDF_OK;
}

// One plain update from cur to nxt, then swap.
mdf_status one_update(mdf_t h, int mode, const mdf_fields_t *out) {
  DevArgs a = base_args(h);
  if (out) {
    a.P = out->P; a.u = out->u; a.rho = out->rho; a.G = out->G; a.div = out->div;
    a.S = out->S; a.sigma = out->sigma; a.omega = out->omega;
  }
  if (mode != MODE_FIELDS) CU(h, launch_set_clock(h->clock, (int)h->step, h->stream));
  CU(h, launch_update(h, mode, a));
  if (mode != MODE_FIELDS) {
    if (h->inplace) h->parity ^= 1;
    else std::swap(h->cur, h->nxt);
    ++h->step;
  }
  return MDF_OK;
}

// Capture kGraphChunk updates starting from buffer `which` (the AA parity
// for the in-place pattern) into a graph.
mdf_status build_graph(mdf_t h, int which) {
  void *c0 = h->cur, *n0 = h->nxt;
  const int p0 = h->parity;
  if (h->inplace) {
    h->parity = which;
  } else {
    h->cur = h->buf[which];
    h->nxt = h->buf[1 - which];
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < kGraphChunk && e == cudaSuccess; ++k) {
      DevArgs a = base_args(h);
      a.tk = k;  // the step is *clock + k; the clock is set before each replay
      e = launch_update(h, MODE_STEP, a);
      if (h->inplace) h->parity ^= 1;
      else std::swap(h->cur, h->nxt);
    }
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e == cudaSuccess) e = e2;
  }
  h->cur = c0;
  h->nxt = n0;
  h->parity = p0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph[which], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->graph[which] = nullptr;
    return fail(h, MDF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  }
  return MDF_OK;
}

mdf_status run_steps(mdf_t h, long long n) {
  // Graph chunks only on a real (non-legacy) stream: capture is not allowed
  // on the legacy default stream.
  const bool use_graph = h->stream != nullptr && n >= kGraphChunk;
  while (use_graph && n >= kGraphChunk) {
    const int which = h->inplace ? h->parity : (h->cur == h->buf[0] ? 0 : 1);
    if (!h->graph[which]) {
      mdf_status st = build_graph(h, which);
      if (st != MDF_OK) return st;
    }
    CU(h, launch_set_clock(h->clock, (int)h->step, h->stream));
    CU(h, cudaGraphLaunch(h->graph[which], h->stream));
    n -= kGraphChunk;  // even chunk: cur/nxt end where they started
    h->step += kGraphChunk;
  }
  if (n > 0) CU(h, launch_set_clock(h->clock, (int)h->step, h->stream));
  for (int k = 0; k < n; ++k) {
    DevArgs a = base_args(h);
    a.tk = k;
    CU(h, launch_update(h, MODE_STEP, a));
    if (h->inplace) h->parity ^= 1;
    else std::swap(h->cur, h->nxt);
  }
  h->step += n;
  return MDF_OK;
}

bool fields_empty(const mdf_fields_t *o) {
  return !(o->P || o->u || o->rho || o->G || o->div || o->S || o->sigma || o->omega);
}

mdf_status check_handle(mdf_t h) {
  if (!h) return MDF_EINVAL;
  return MDF_OK;
}

int nsym(int d) { return d == 2 ? 3 : 6; }

uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t hsh = 1469598103934665603ull) {
  for (size_t i = 0; i < n; ++i) { hsh ^= p[i]; hsh *= 1099511628211ull; }
  return hsh;
}

struct CkptHeader {
  char magic[8];
  int32_t version, d, q, nsets, storage, nx, ny, nz, px, wall[3], lid;
  int32_t forcing;  // the state is fbar under Scheme II: part of its meaning
  int32_t layout;   // 0: two buffers (pull); in-place AA: 1 even, 2 odd layout
  double s0, s1, s2, lid_u[3];
  int64_t step, payload;
  uint64_t checksum;
};

}  // namespace

extern "C" {

mdf_status mdf_create(mdf_t *out, const mdf_grid *g, int d, const mdf_rates *r,
                      const mdf_bc *bc, const mdf_opts *o) {
  if (!out) return fail(nullptr, MDF_EINVAL, "null handle pointer");
  *out = nullptr;
  if (!g || !r) return fail(nullptr, MDF_EINVAL, "null grid or rates");
  if (d != 2 && d != 3) return fail(nullptr, MDF_EINVAL, "d must be 2 or 3 (got %d)", d);
  if (g->nx < 2 || g->ny < 2 || (d == 2 && g->nz != 1) || (d == 3 && g->nz < 2))
    return fail(nullptr, MDF_EINVAL, "bad grid %d x %d x %d for d = %d", g->nx, g->ny, g->nz, d);
  if ((long long)g->nx * g->ny * g->nz > (1LL << 40) || g->ny > 65535 || g->nz > 65535)
    return fail(nullptr, MDF_EINVAL, "grid too large (ny, nz <= 65535)");
  const double s1 = r->s1;
  const double s2 = r->s2 < 0 ? 8.0 * (2.0 - s1) / (8.0 - s1) : r->s2;
  if (!(s1 > 0 && s1 < 2) || !(s2 > 0 && s2 < 2) || !(r->s0 > 0 && r->s0 < 2))
    return fail(nullptr, MDF_EINVAL, "relaxation rates must lie in (0, 2): s0=%g s1=%g s2=%g",
                r->s0, s1, s2);
  mdf_opts opts{};
  opts.storage = MDF_F32;
  opts.with_rho = 1;
  if (o) opts = *o;
  if (storage_bytes(opts.storage) == 0)
    return fail(nullptr, MDF_EUNSUPPORTED, "unknown storage %d", opts.storage);
  const int q = opts.q ? opts.q : (d == 2 ? 5 : 7);
  if (!lattice_launch(d, q))
    return fail(nullptr, MDF_EUNSUPPORTED, "no D%dQ%d lattice (D2Q5, D2Q4, D3Q7, D3Q6)", d, q);
  if (q != 5 && q != 7 && eq_storage(opts.storage))
    return fail(nullptr, MDF_EUNSUPPORTED, "equilibrium-shifted storage needs D2Q5 or D3Q7");

  mdf_t h = new (std::nothrow) mdf_s;
  if (!h) return fail(nullptr, MDF_ENOMEM, "host allocation");
  h->d = d;
  h->q = q;
  h->with_rho = opts.with_rho ? 1 : 0;
  h->nsets = d + h->with_rho;
  h->storage = opts.storage;
  h->nx = g->nx; h->ny = g->ny; h->nz = g->nz;
  // x pitch: 128-byte rows; the equilibrium-shifted codecs store x in tiles
  // of 64 nodes (mdf_eq.cuh), so their pitch is a multiple of 64
  const int pitch = eq_storage(opts.storage) ? 64 : 32;
  h->px = (g->nx + pitch - 1) / pitch * pitch;
  h->plane = (long long)h->px * g->ny * g->nz;
  h->N = (long long)g->nx * g->ny * g->nz;
  h->s0 = r->s0; h->s1 = s1; h->s2 = s2;
  if (bc) h->bc = *bc;
  for (int b = 0; b < 3; ++b) h->bc.wall[b] = (b < d && h->bc.wall[b]) ? 1 : 0;
  h->walls = h->bc.wall[0] || h->bc.wall[1] || h->bc.wall[2];
  if (h->bc.lid && !h->bc.wall[d - 1]) {
    delete h;
    return fail(nullptr, MDF_EINVAL, "a lid needs walls on the last axis");
  }
  h->stream = static_cast<cudaStream_t>(opts.stream);
  if (opts.block != 0 && (opts.block < 32 || opts.block > kMaxBlock || opts.block % 32)) {
    delete h;
    return fail(nullptr, MDF_EINVAL, "block must be a multiple of 32 in [32, %d]", kMaxBlock);
  }
  if (opts.vx < 0 || opts.vx > 8) {
    delete h;
    return fail(nullptr, MDF_EINVAL, "vx must be 0 (default), 1, 2, 4 or 8");
  }
  h->inplace = opts.inplace != 0;
  if (h->inplace && eq_storage(h->storage)) {
    delete h;
    return fail(nullptr, MDF_EUNSUPPORTED, "the in-place AA pattern takes the rest-shifted storage types");
  }
  if (eq_storage(h->storage)) {
    h->kmom = d + 1 + h->with_rho;
    if (h->plane >= (1LL << 31) - 64) {
      delete h;
      return fail(nullptr, MDF_EUNSUPPORTED, "equilibrium-shifted storage needs < 2^31 padded nodes");
    }
  }
  h->block = opts.block ? opts.block : (h->inplace ? default_block_aa(d, h->storage) : default_block(d, h->storage));
  h->vx = opts.vx ? opts.vx : (h->inplace ? default_vx_aa(d, h->storage) : default_vx(d, h->storage));
  h->vx = std::min(h->vx, max_vx(d, h->storage, h->inplace));

  const size_t pb = h->pop_bytes();
  cudaError_t e = cudaMalloc(&h->buf[0], pb);
  if (e == cudaSuccess && !h->inplace) e = cudaMalloc(&h->buf[1], pb);
  if (e == cudaSuccess) e = cudaMalloc(&h->partials, sizeof(double) * kReduceBlocks * 4);
  if (e == cudaSuccess) e = cudaMalloc(&h->result, sizeof(double) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&h->nonfinite, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->clock, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->clock, 0, sizeof(int), h->stream);
  if (e == cudaSuccess && h->walls) e = cudaMalloc(&h->mask, (size_t)h->plane);
  if (e == cudaSuccess && h->kmom) e = cudaMalloc(&h->mac[0], h->mom_bytes());
  if (e == cudaSuccess && h->kmom) e = cudaMalloc(&h->mac[1], h->mom_bytes());
  if (e == cudaSuccess && h->kmom) e = cudaMemsetAsync(h->mac[0], 0, h->mom_bytes(), h->stream);
  if (e == cudaSuccess && h->kmom) e = cudaMemsetAsync(h->mac[1], 0, h->mom_bytes(), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[0], 0, pb, h->stream);
  if (e == cudaSuccess && !h->inplace) e = cudaMemsetAsync(h->buf[1], 0, pb, h->stream);
  if (e == cudaSuccess && h->walls) {
    e = cudaMemsetAsync(h->mask, 0, (size_t)h->plane, h->stream);
    if (e == cudaSuccess) {
      DevArgs a = base_args(h);
      e = lattice_launch(h->d, h->q)->mask(h->bc.wall, h->bc.lid, a, h->mask, h->stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mdf_status st = e == cudaErrorMemoryAllocation ? MDF_ENOMEM : MDF_ECUDA;
    fail(nullptr, st, "create: %s", cudaGetErrorString(e));
    mdf_destroy(h);
    return st;
  }
  h->cur = h->buf[0];
  h->nxt = h->inplace ? h->buf[0] : h->buf[1];
  *out = h;
  return MDF_OK;
}

void mdf_destroy(mdf_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  cudaFree(h->buf[0]); cudaFree(h->buf[1]); cudaFree(h->mask); cudaFree(h->force);
  cudaFree(h->mac[0]); cudaFree(h->mac[1]);
  cudaFree(h->stage); cudaFree(h->uprev); cudaFree(h->partials); cudaFree(h->result);
  cudaFree(h->nonfinite); cudaFree(h->clock);
  delete h;
}

static mdf_status init_state(mdf_t h, const double *P, const double *u, const double *G, int where) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!P || !u) return fail(h, MDF_EINVAL, "init: null P or u");
  const size_t nb = sizeof(double) * (size_t)h->N;
  const int dd = h->d * h->d;
  DevArgs a = base_args(h);
  if (where == MDF_HOST) {
    mdf_status st = ensure_stage(h, nb * (1 + h->d + (G ? dd : 0)));
    if (st != MDF_OK) return st;
    CU(h, cudaMemcpyAsync(h->stage, P, nb, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->stage + h->N, u, nb * h->d, cudaMemcpyHostToDevice, h->stream));
    a.Pin = h->stage;
    a.uin = h->stage + h->N;
    if (G) {
      CU(h, cudaMemcpyAsync(h->stage + (1 + h->d) * h->N, G, nb * dd, cudaMemcpyHostToDevice, h->stream));
      a.Gin = h->stage + (1 + h->d) * h->N;
    }
  } else if (where == MDF_DEVICE) {
    a.Pin = P;
    a.uin = u;
    a.Gin = G;
  } else {
    return fail(h, MDF_EINVAL, "init: bad `where` %d", where);
  }
  a.fout = h->cur;
  a.mout = h->mac[h->cur_index()];
  CU(h, lattice_launch(h->d, h->q)->init(h->storage, h->walls, a, h->stream));
  if (where == MDF_HOST) CU(h, cudaStreamSynchronize(h->stream));
  h->parity = 0;  // the in-place pattern starts in the even layout
  h->step = 0;
  h->have_prev = false;
  return MDF_OK;
}

mdf_status mdf_init(mdf_t h, const double *P, const double *u, int where) {
  return init_state(h, P, u, nullptr, where);
}

mdf_status mdf_init_neq(mdf_t h, const double *P, const double *u, const double *G, int where) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!G) return fail(h, MDF_EINVAL, "init_neq: null G");
  return init_state(h, P, u, G, where);
}

mdf_status mdf_set_force(mdf_t h, const double *F, int where) {
  if (check_handle(h)) return MDF_EINVAL;
  CU(h, cudaStreamSynchronize(h->stream));
  drop_graphs(h);  // captured launches hold the old force pointer
  if (!F) {
    cudaFree(h->force);
    h->force = nullptr;
    return MDF_OK;
  }
  const bool f64 = h->storage == MDF_F64;
  const size_t fbytes = (f64 ? sizeof(double) : sizeof(float)) * (size_t)h->plane * h->d;
  if (!h->force) {
    cudaError_t e = cudaMalloc(&h->force, fbytes);
    if (e != cudaSuccess) { cudaGetLastError(); h->force = nullptr; return fail(h, MDF_ENOMEM, "force: %s", cudaGetErrorString(e)); }
    CU(h, cudaMemsetAsync(h->force, 0, fbytes, h->stream));
  }
  const double *src = F;
  const size_t nb = sizeof(double) * (size_t)h->N * h->d;
  if (where == MDF_HOST) {
    mdf_status st = ensure_stage(h, nb);
    if (st != MDF_OK) return st;
    CU(h, cudaMemcpyAsync(h->stage, F, nb, cudaMemcpyHostToDevice, h->stream));
    src = h->stage;
  } else if (where != MDF_DEVICE) {
    return fail(h, MDF_EINVAL, "set_force: bad `where` %d", where);
  }
  CU(h, launch_pad_force(src, h->force, f64, h->d, h->nx, h->ny, h->nz, h->px, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return MDF_OK;
}

mdf_status mdf_set_forcing(mdf_t h, int scheme) {
  if (check_handle(h)) return MDF_EINVAL;
  if (scheme != MDF_FORCING_EQ321 && scheme != MDF_FORCING_SCHEME2)
    return fail(h, MDF_EINVAL, "set_forcing: unknown scheme %d", scheme);
  if (scheme == h->forcing) return MDF_OK;
  CU(h, cudaStreamSynchronize(h->stream));
  drop_graphs(h);  // captured launches hold the old scheme
  h->forcing = scheme;
  return MDF_OK;
}

mdf_status mdf_get_forcing(mdf_t h, int *scheme) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!scheme) return fail(h, MDF_EINVAL, "get_forcing: null output");
  *scheme = h->forcing;
  return MDF_OK;
}

mdf_status mdf_step(mdf_t h, long long n) {
  if (check_handle(h)) return MDF_EINVAL;
  if (n < 0) return fail(h, MDF_EINVAL, "step: n < 0");
  return run_steps(h, n);
}

mdf_status mdf_step_fields(mdf_t h, long long n, const mdf_fields_t *out) {
  if (check_handle(h)) return MDF_EINVAL;
  if (n < 1 || !out) return fail(h, MDF_EINVAL, "step_fields: need n >= 1 and outputs");
  if (out->where != MDF_DEVICE) return fail(h, MDF_EINVAL, "step_fields: outputs must be on the device");
  if (out->rho && !h->with_rho) return fail(h, MDF_EINVAL, "rho requested without the alpha = 0 set");
  mdf_status st = one_update(h, fields_empty(out) ? MODE_STEP : MODE_STEP_FIELDS, out);
  if (st != MDF_OK) return st;
  return run_steps(h, n - 1);
}

mdf_status mdf_fields(mdf_t h, const mdf_fields_t *out) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!out) return fail(h, MDF_EINVAL, "fields: null outputs");
  if (out->rho && !h->with_rho) return fail(h, MDF_EINVAL, "rho requested without the alpha = 0 set");
  if (fields_empty(out)) return MDF_OK;
  if (out->where == MDF_DEVICE) return one_update(h, MODE_FIELDS, out);
  if (out->where != MDF_HOST) return fail(h, MDF_EINVAL, "fields: bad `where`");
  // host outputs: compute into staging, then copy each requested field back
  const long long N = h->N;
  const int d = h->d;
  struct F { double *host; size_t count; } f[8] = {
      {out->P, (size_t)N}, {out->u, (size_t)(d * N)}, {out->rho, (size_t)N},
      {out->G, (size_t)(d * d * N)}, {out->div, (size_t)N}, {out->S, (size_t)(nsym(d) * N)},
      {out->sigma, (size_t)(nsym(d) * N)}, {out->omega, (size_t)((d == 2 ? 1 : 3) * N)}};
  size_t total = 0;
  for (auto &x : f)
    if (x.host) total += x.count;
  mdf_status st = ensure_stage(h, total * sizeof(double));
  if (st != MDF_OK) return st;
  mdf_fields_t dev{};
  dev.where = MDF_DEVICE;
  double *p = h->stage;
  double **slots[8] = {&dev.P, &dev.u, &dev.rho, &dev.G, &dev.div, &dev.S, &dev.sigma, &dev.omega};
  for (int k = 0; k < 8; ++k)
    if (f[k].host) { *slots[k] = p; p += f[k].count; }
  st = one_update(h, MODE_FIELDS, &dev);
  if (st != MDF_OK) return st;
  for (int k = 0; k < 8; ++k)
    if (f[k].host)
      CU(h, cudaMemcpyAsync(f[k].host, *slots[k], f[k].count * sizeof(double),
                            cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return MDF_OK;
}

mdf_status mdf_moments(mdf_t h, double *P, double *u, double *rho) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!P || !u) return fail(h, MDF_EINVAL, "moments: P and u are required");
  mdf_fields_t o{};
  o.P = P; o.u = u; o.rho = rho; o.where = MDF_DEVICE;
  return mdf_fields(h, &o);
}

mdf_status mdf_gradients(mdf_t h, double *G, double *div, double *S, double *sigma,
                         double *omega) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!G && !div && !S && !sigma && !omega)
    return fail(h, MDF_EINVAL, "gradients: no output requested");
  mdf_fields_t o{};
  o.G = G; o.div = div; o.S = S; o.sigma = sigma; o.omega = omega; o.where = MDF_DEVICE;
  return mdf_fields(h, &o);
}

static mdf_status reduce(mdf_t h, int kind, double out[4]) {
  DevArgs a = base_args(h);
  CU(h, cudaMemsetAsync(h->nonfinite, 0, sizeof(int), h->stream));
  CU(h, launch_reduce(h, kind, a));
  CU(h, launch_reduce_final(a, kReduceBlocks, 4, h->stream));
  int bad = 0;
  CU(h, cudaMemcpyAsync(out, h->result, sizeof(double) * 4, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaMemcpyAsync(&bad, h->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (bad) return fail(h, MDF_EDIVERGED, "non-finite populations");
  return MDF_OK;
}

mdf_status mdf_sums(mdf_t h, double *sums) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!sums) return fail(h, MDF_EINVAL, "sums: null output");
  double r[4];
  mdf_status st = reduce(h, RED_SUMS, r);
  if (st != MDF_OK) return st;
  for (int k = 0; k < h->nsets; ++k) sums[k] = r[k];
  return MDF_OK;
}

mdf_status mdf_residual(mdf_t h, double *res) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!res) return fail(h, MDF_EINVAL, "residual: null output");
  if (!h->uprev) {
    cudaError_t e = cudaMalloc(&h->uprev, sizeof(double) * (size_t)h->N * h->d);
    if (e != cudaSuccess) { cudaGetLastError(); h->uprev = nullptr; return fail(h, MDF_ENOMEM, "residual: %s", cudaGetErrorString(e)); }
    h->have_prev = false;
  }
  double r[4];
  mdf_status st = reduce(h, RED_RESIDUAL, r);
  if (st != MDF_OK) return st;
  if (!h->have_prev) {
    h->have_prev = true;
    *res = INFINITY;
    return MDF_OK;
  }
  *res = r[1] > 0 ? std::sqrt(r[0] / r[1]) : (r[0] > 0 ? INFINITY : 0.0);
  return MDF_OK;
}

mdf_status mdf_mask(mdf_t h, unsigned char *host_out) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!host_out) return fail(h, MDF_EINVAL, "mask: null output");
  if (!h->walls) {
    std::memset(host_out, 0, (size_t)h->N);
    return MDF_OK;
  }
  std::vector<unsigned char> tmp((size_t)h->plane);
  CU(h, cudaMemcpyAsync(tmp.data(), h->mask, (size_t)h->plane, cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  for (long long z = 0; z < h->nz; ++z)
    for (long long y = 0; y < h->ny; ++y)
      std::memcpy(host_out + (z * h->ny + y) * h->nx, tmp.data() + (z * h->ny + y) * h->px,
                  (size_t)h->nx);
  return MDF_OK;
}

static void fill_header(const mdf_t h, CkptHeader &hd) {
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, "MDFLBM1", 8);
  hd.version = 2;
  hd.d = h->d; hd.q = h->q; hd.nsets = h->nsets; hd.storage = h->storage;
  hd.nx = h->nx; hd.ny = h->ny; hd.nz = h->nz; hd.px = h->px;
  for (int b = 0; b < 3; ++b) { hd.wall[b] = h->bc.wall[b]; hd.lid_u[b] = h->bc.lid_u[b]; }
  hd.lid = h->bc.lid;
  hd.forcing = h->forcing;
  hd.layout = h->inplace ? 1 + h->parity : 0;
  hd.s0 = h->s0; hd.s1 = h->s1; hd.s2 = h->s2;
  hd.step = h->step;
  hd.payload = (int64_t)(h->pop_bytes() + h->mom_bytes());
}

mdf_status mdf_save(mdf_t h, const char *path) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!path) return fail(h, MDF_EINVAL, "save: null path");
  std::vector<unsigned char> buf(h->pop_bytes() + h->mom_bytes());
  CU(h, cudaMemcpyAsync(buf.data(), h->cur, h->pop_bytes(), cudaMemcpyDeviceToHost, h->stream));
  if (h->kmom)
    CU(h, cudaMemcpyAsync(buf.data() + h->pop_bytes(), h->mac[h->cur_index()], h->mom_bytes(),
                          cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  CkptHeader hd;
  fill_header(h, hd);
  hd.checksum = fnv1a(buf.data(), buf.size());
  FILE *fp = std::fopen(path, "wb");
  if (!fp) return fail(h, MDF_EIO, "save: cannot open %s", path);
  bool ok = std::fwrite(&hd, sizeof hd, 1, fp) == 1 &&
            std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? MDF_OK : fail(h, MDF_EIO, "save: write failed for %s", path);
}

mdf_status mdf_load(mdf_t h, const char *path) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!path) return fail(h, MDF_EINVAL, "load: null path");
  FILE *fp = std::fopen(path, "rb");
  if (!fp) return fail(h, MDF_EIO, "load: cannot open %s", path);
  CkptHeader hd, want;
  fill_header(h, want);
  bool ok = std::fread(&hd, sizeof hd, 1, fp) == 1;
  if (ok) {
    want.step = hd.step;
    want.checksum = hd.checksum;
    if (h->inplace && (hd.layout == 1 || hd.layout == 2)) want.layout = hd.layout;
    ok = std::memcmp(&hd, &want, sizeof hd) == 0;
  }
  if (!ok) { std::fclose(fp); return fail(h, MDF_EIO, "load: header of %s does not match this handle", path); }
  std::vector<unsigned char> buf(h->pop_bytes() + h->mom_bytes());
  ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
  std::fclose(fp);
  if (!ok) return fail(h, MDF_EIO, "load: short file %s", path);
  if (fnv1a(buf.data(), buf.size()) != hd.checksum) return fail(h, MDF_EIO, "load: checksum mismatch in %s", path);
  CU(h, cudaMemcpyAsync(h->cur, buf.data(), h->pop_bytes(), cudaMemcpyHostToDevice, h->stream));
  if (h->kmom)
    CU(h, cudaMemcpyAsync(h->mac[h->cur_index()], buf.data() + h->pop_bytes(), h->mom_bytes(),
                          cudaMemcpyHostToDevice, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  h->step = hd.step;
  if (h->inplace) h->parity = hd.layout - 1;
  h->have_prev = false;
  return MDF_OK;
}

mdf_status mdf_info(mdf_t h, mdf_info_t *out) {
  if (check_handle(h) || !out) return MDF_EINVAL;
  out->d = h->d; out->q = h->q; out->nsets = h->nsets; out->storage = h->storage;
  out->nx = h->nx; out->ny = h->ny; out->nz = h->nz; out->pitch = h->px;
  out->nodes = h->N;
  out->step = h->step;
  out->bytes_per_update = 2.0 * h->q * h->nsets * (double)storage_bytes(h->storage) +
                         2.0 * 4.0 * h->kmom;
  out->vx = h->vx;
  out->block = h->block;
  out->s0 = h->s0; out->s1 = h->s1; out->s2 = h->s2;
  return MDF_OK;
}

mdf_status mdf_autotune(mdf_t h, int reps, int *vx_out, int *block_out) {
  if (check_handle(h)) return MDF_EINVAL;
  if (h->inplace)  // its trial updates run out of place, and there is one buffer
    return fail(h, MDF_EUNSUPPORTED, "autotune needs the two-buffer layout");
  if (reps < 1) reps = 10;
  // Candidates: one node per thread, and every vector width built for the
  // storage type that divides nx; 64, 128 and 256 threads per block.
  int widths[4] = {1, 0, 0, 0}, nw = 1;
  // by MDF_F32, F16, BF16, F64, F16EQ, BF16EQ
  const int built[6][2] = {{2, 4}, {4, 8}, {4, 8}, {2, 2}, {2, 4}, {2, 4}};
  for (int k = 0; k < 2; ++k) {
    const int v = std::min(built[h->storage][k], max_vx(h->d, h->storage, false));
    bool dup = false;
    for (int j = 0; j < nw; ++j) dup |= widths[j] == v;
    if (!dup && h->nx % v == 0) widths[nw++] = v;
  }
  const int blocks[3] = {64, 128, 256};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(h, cudaEventCreate(&e0));
  CU(h, cudaEventCreate(&e1));
  float best = 1e30f;
  int best_vx = h->vx, best_block = h->block;
  mdf_status st = MDF_OK;
  for (int w = 0; w < nw && st == MDF_OK; ++w)
    for (int b = 0; b < 3 && st == MDF_OK; ++b) {
      h->vx = widths[w];
      h->block = blocks[b];
      // out-of-place updates cur -> nxt without swapping: the state is kept
      const DevArgs a = base_args(h);
      cudaError_t e = launch_update(h, MODE_STEP, a);
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_update(h, MODE_STEP, a);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        st = fail(h, MDF_ECUDA, "autotune: %s", cudaGetErrorString(e));
        break;
      }
      if (ms < best) { best = ms; best_vx = widths[w]; best_block = blocks[b]; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->vx = best_vx;
  h->block = best_block;
  drop_graphs(h);  // captured launches hold the old shape
  if (st != MDF_OK) return st;
  if (vx_out) *vx_out = best_vx;
  if (block_out) *block_out = best_block;
  return MDF_OK;
}

mdf_status mdf_sync(mdf_t h) {
  if (check_handle(h)) return MDF_EINVAL;
  CU(h, cudaStreamSynchronize(h->stream));
  return MDF_OK;
}

const char *mdf_last_error(mdf_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free readback of the derived fields to host memory.
//
// mdf_fields() with host outputs stages the fields in a device buffer that
// the handle grows with cudaMalloc on demand.  Some callers cannot let the
// library allocate at that point: a process whose GPU memory is fully
// reserved by another allocator (a framework's caching pool, an MPS memory
// quota), or code running while allocation is forbidden (for instance while
// another thread captures work in global capture mode, where a cudaMalloc
// would invalidate that capture).  mdf_fields_host_noalloc stages through
// the fixed buffer below instead and calls no allocating routine.
// ---------------------------------------------------------------------------
namespace {

// 2,097,152 doubles = 16 MiB, held on every GPU that loads this library
// until the process exits.  Shared by all calls on that GPU.
constexpr size_t kNoallocStageDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_noalloc_stage[kNoallocStageDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_addr[kMaxDevices] = {};  // device address of the buffer, per GPU

// Device address of g_noalloc_stage on the GPU that holds h's populations.
// Looked up once per GPU (with that GPU current) and cached: in host code the
// symbol name is only a host-side stand-in, never a device address.
mdf_status noalloc_stage_address(mdf_t h, double **out) {
  cudaPointerAttributes attr;
  CU(h, cudaPointerGetAttributes(&attr, h->buf[0]));
  const int dev = attr.device;
  if (dev < 0 || dev >= kMaxDevices)
    return fail(h, MDF_EUNSUPPORTED, "fields_host_noalloc: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    int cur = 0;
    CU(h, cudaGetDevice(&cur));
    if (cur != dev) CU(h, cudaSetDevice(dev));
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_stage);
    if (cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess || !p)
      return fail(h, MDF_ECUDA, "fields_host_noalloc: cudaGetSymbolAddress failed: %s",
                  cudaGetErrorString(e));
    g_noalloc_addr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_addr[dev];
  return MDF_OK;
}

}  // namespace

extern "C" mdf_status mdf_fields_host_noalloc(mdf_t h, const mdf_fields_t *out) {
  if (check_handle(h)) return MDF_EINVAL;
  if (!out) return fail(h, MDF_EINVAL, "fields_host_noalloc: null outputs");
  if (out->where != MDF_HOST)
    return fail(h, MDF_EINVAL, "fields_host_noalloc: outputs must be host arrays (where = MDF_HOST)");
  if (out->rho && !h->with_rho)
    return fail(h, MDF_EINVAL, "rho requested without the alpha = 0 set");
  if (fields_empty(out)) return MDF_OK;
  const size_t N = (size_t)h->N;
  const int d = h->d;
  double *const host[8] = {out->P, out->u, out->rho, out->G, out->div, out->S, out->sigma, out->omega};
  const size_t count[8] = {N, d * N, N, (size_t)d * d * N, N, nsym(d) * N, nsym(d) * N,
                           (size_t)(d == 2 ? 1 : 3) * N};
  size_t total = 0;
  for (int k = 0; k < 8; ++k)
    if (host[k]) total += count[k];
  if (total > kNoallocStageDoubles)
    return fail(h, MDF_EINVAL,
                "fields_host_noalloc: the requested fields need %zu doubles but the static "
                "staging buffer holds %zu (16 MiB); request fewer fields or use mdf_fields",
                total, kNoallocStageDoubles);
  double *stage = nullptr;
  mdf_status st = noalloc_stage_address(h, &stage);
  if (st != MDF_OK) return st;
  // Every requested field is written in full by the kernel, so no part of the
  // shared buffer has to be cleared first.
  DevArgs a = base_args(h);
  double **slot[8] = {&a.P, &a.u, &a.rho, &a.G, &a.div, &a.S, &a.sigma, &a.omega};
  double *p = stage;
  for (int k = 0; k < 8; ++k)
    if (host[k]) { *slot[k] = p; p += count[k]; }
  CU(h, launch_update(h, MODE_FIELDS, a));
  for (int k = 0; k < 8; ++k)
    if (host[k])
      CU(h, cudaMemcpyAsync(host[k], *slot[k], count[k] * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return MDF_OK;
}

// ---------------------------------------------------------------------------
// Slab decomposition: one lattice as k sub-domains along its last axis (y in
// 2D, z in 3D), each a handle of its own with one ghost layer on either side.
// After every update the only populations that cross a face are exchanged:
// for each set, the post-collision values of the one direction pointing
// across it, one layer (a row of x in 2D, an x-y plane in 3D) per face,
// copied device to device.  The ghost layers are updated with the rest and
// their results ignored: the next update of a real layer pulls from a ghost
// layer only the exchanged slot.  The per-node arithmetic is the undivided
// lattice's, so the two give the same bits.  This is the exchange a
// multi-GPU run would make between neighbouring ranks; here all sub-domains
// live on one GPU and share one stream.
// ---------------------------------------------------------------------------
struct mdf_slabs_s {
  int d = 0, k = 0, nloc = 0;  // sub-domains and real layers per sub-domain
  int nx = 0, ny = 0, nz = 0;  // global grid
  std::vector<mdf_t> h;
  cudaStream_t stream = nullptr;
  long long step = 0;
  std::string err = "no error";
};

namespace {

std::string g_slabs_create_error = "no error";

mdf_status sfail(mdf_slabs_t s, mdf_status st, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (s) s->err = msg;
  else g_slabs_create_error = msg;
  return st;
}

// Elements of one layer along the last axis, and the address of layer `l`
// of slot i of set a in buffer `buf` of handle h.
size_t layer_elems(const mdf_t h) { return h->d == 2 ? (size_t)h->px : (size_t)h->px * h->ny; }
char *layer_at(const mdf_t h, void *buf, int a, int i, int l) {
  const size_t el = storage_bytes(h->storage);
  return static_cast<char *>(buf) +
         (((size_t)a * h->q + i) * (size_t)h->plane + (size_t)l * layer_elems(h)) * el;
}

// Direction index of c = sg e_last for lattice (d, q).
int axis_dir(int d, int q, int sg) {
  if (d == 2) return q == 5 ? (sg > 0 ? 2 : 4) : (sg > 0 ? 1 : 3);
  return q == 7 ? (sg > 0 ? 5 : 6) : (sg > 0 ? 4 : 5);
}

mdf_status exchange(mdf_slabs_t S) {
  const int k = S->k;
  const size_t bytes = layer_elems(S->h[0]) * storage_bytes(S->h[0]->storage);
  const int up = axis_dir(S->d, S->h[0]->q, +1), dn = axis_dir(S->d, S->h[0]->q, -1);
  for (int s = 0; s < k; ++s) {
    mdf_t me = S->h[s], lo = S->h[(s + k - 1) % k], hi = S->h[(s + 1) % k];
    for (int a = 0; a < me->nsets; ++a) {
      // ghost layer 0 <- the lower neighbour's last real layer, moving up
      cudaError_t e = cudaMemcpyAsync(layer_at(me, me->cur, a, up, 0), layer_at(lo, lo->cur, a, up, S->nloc),
                                      bytes, cudaMemcpyDeviceToDevice, S->stream);
      // ghost layer nloc + 1 <- the upper neighbour's first real layer, moving down
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(layer_at(me, me->cur, a, dn, S->nloc + 1), layer_at(hi, hi->cur, a, dn, 1), bytes,
                            cudaMemcpyDeviceToDevice, S->stream);
      if (e != cudaSuccess) return sfail(S, MDF_ECUDA, "slab exchange: %s", cudaGetErrorString(e));
    }
  }
  return MDF_OK;
}

}  // namespace

extern "C" {

void mdf_slabs_destroy(mdf_slabs_t s) {
  if (!s) return;
  for (mdf_t h : s->h) mdf_destroy(h);
  delete s;
}

mdf_status mdf_slabs_create(mdf_slabs_t *out, const mdf_grid *g, int d, const mdf_rates *r,
                            const mdf_bc *bc, const mdf_opts *o, int k) {
  if (!out) return sfail(nullptr, MDF_EINVAL, "null handle pointer");
  *out = nullptr;
  if (!g || !r) return sfail(nullptr, MDF_EINVAL, "null grid or rates");
  if (d != 2 && d != 3) return sfail(nullptr, MDF_EINVAL, "d must be 2 or 3");
  const int n = d == 2 ? g->ny : g->nz;
  if (k < 1 || n % k != 0) return sfail(nullptr, MDF_EINVAL, "%d layers do not split into %d slabs", n, k);
  if (bc && (bc->wall[d - 1] || bc->lid))
    return sfail(nullptr, MDF_EUNSUPPORTED, "the split axis must be periodic (no walls or lid on it)");
  if (o && (o->inplace || o->storage == MDF_F16EQ || o->storage == MDF_BF16EQ))
    return sfail(nullptr, MDF_EUNSUPPORTED, "slabs take the two-buffer rest-shifted storage types");
  mdf_slabs_t S = new (std::nothrow) mdf_slabs_s;
  if (!S) return sfail(nullptr, MDF_ENOMEM, "host allocation");
  S->d = d; S->k = k; S->nloc = n / k;
  S->nx = g->nx; S->ny = g->ny; S->nz = g->nz;
  S->stream = o ? static_cast<cudaStream_t>(o->stream) : nullptr;
  mdf_grid gl = *g;
  if (d == 2) gl.ny = S->nloc + 2;
  else gl.nz = S->nloc + 2;
  for (int s = 0; s < k; ++s) {
    mdf_t h = nullptr;
    const mdf_status st = mdf_create(&h, &gl, d, r, bc, o);
    if (st != MDF_OK) {
      sfail(nullptr, st, "slab %d: %s", s, mdf_last_error(nullptr));
      mdf_slabs_destroy(S);
      return st;
    }
    // global index of local node 0: local layer 1 is global layer s nloc
    const long long L = d == 2 ? (long long)g->nx : (long long)g->nx * g->ny;
    h->key_base = ((long long)s * S->nloc - 1) * L;
    S->h.push_back(h);
  }
  *out = S;
  return MDF_OK;
}

mdf_status mdf_slabs_init(mdf_slabs_t S, const double *P, const double *u) {
  if (!S) return MDF_EINVAL;
  if (!P || !u) return sfail(S, MDF_EINVAL, "init: null P or u");
  const long long N = (long long)S->nx * S->ny * S->nz;
  const long long L = S->d == 2 ? S->nx : (long long)S->nx * S->ny;  // nodes per layer
  const int n = S->nloc * S->k, nl = S->nloc + 2;
  std::vector<double> Pl((size_t)(L * nl)), ul((size_t)(L * nl * S->d));
  for (int s = 0; s < S->k; ++s) {
    for (int l = 0; l < nl; ++l) {  // local layer l holds global layer s nloc + l - 1 (periodic)
      const long long gl = ((long long)s * S->nloc + l - 1 + n) % n;
      std::memcpy(&Pl[(size_t)(l * L)], P + gl * L, sizeof(double) * (size_t)L);
      for (int b = 0; b < S->d; ++b)
        std::memcpy(&ul[(size_t)(b * L * nl + l * L)], u + b * N + gl * L, sizeof(double) * (size_t)L);
    }
    const mdf_status st = mdf_init(S->h[s], Pl.data(), ul.data(), MDF_HOST);
    if (st != MDF_OK) return sfail(S, st, "slab %d init: %s", s, mdf_last_error(S->h[s]));
  }
  S->step = 0;
  return MDF_OK;
}

mdf_status mdf_slabs_step(mdf_slabs_t S, long long n) {
  if (!S) return MDF_EINVAL;
  if (n < 0) return sfail(S, MDF_EINVAL, "step: n < 0");
  for (long long t = 0; t < n; ++t) {
    for (mdf_t h : S->h) {
      const mdf_status st = one_update(h, MODE_STEP, nullptr);
      if (st != MDF_OK) return sfail(S, st, "slab update: %s", h->err.c_str());
    }
    const mdf_status st = exchange(S);
    if (st != MDF_OK) return st;
    ++S->step;
  }
  return MDF_OK;
}

mdf_status mdf_slabs_fields(mdf_slabs_t S, const mdf_fields_t *out) {
  if (!S) return MDF_EINVAL;
  if (!out || out->where != MDF_HOST) return sfail(S, MDF_EINVAL, "fields: host outputs only");
  const int d = S->d;
  const long long N = (long long)S->nx * S->ny * S->nz;
  const long long L = d == 2 ? S->nx : (long long)S->nx * S->ny;
  const long long Nl = L * (S->nloc + 2);
  const int nsymm = d == 2 ? 3 : 6;
  double *const dst[8] = {out->P, out->u, out->rho, out->G, out->div, out->S, out->sigma, out->omega};
  const int comps[8] = {1, d, 1, d * d, 1, nsymm, nsymm, d == 2 ? 1 : 3};
  std::vector<double> loc[8];
  mdf_fields_t lf{};
  lf.where = MDF_HOST;
  double **slot[8] = {&lf.P, &lf.u, &lf.rho, &lf.G, &lf.div, &lf.S, &lf.sigma, &lf.omega};
  for (int f = 0; f < 8; ++f)
    if (dst[f]) {
      loc[f].resize((size_t)(comps[f] * Nl));
      *slot[f] = loc[f].data();
    }
  for (int s = 0; s < S->k; ++s) {
    const mdf_status st = mdf_fields(S->h[s], &lf);
    if (st != MDF_OK) return sfail(S, st, "slab %d fields: %s", s, mdf_last_error(S->h[s]));
    for (int f = 0; f < 8; ++f) {
      if (!dst[f]) continue;
      for (int c = 0; c < comps[f]; ++c)  // real layers 1 .. nloc
        std::memcpy(dst[f] + c * N + (long long)s * S->nloc * L, loc[f].data() + c * Nl + L,
                    sizeof(double) * (size_t)(S->nloc * L));
    }
  }
  return MDF_OK;
}

const char *mdf_slabs_last_error(mdf_slabs_t S) { return S ? S->err.c_str() : g_slabs_create_error.c_str(); }

}  // extern "C"

// Host/device interface between the C-ABI layer (mdf_api.cu) and the
// per-lattice kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdf {

// Everything a kernel launch needs, as plain pointers and sizes.
struct DevArgs {
  const void *fin;               // current populations (post-collision, pre-stream)
  void *fout;                    // next populations
  const uint8_t *mask;           // link mask [plane] or null (periodic)
  const void *force;             // [d][plane] body force (compute type) or null
  int scheme2;                   // 1: Scheme II forcing (Eq. 2-3c, 2-7a) with a force set
  int aa;                        // 0: two buffers, pull; in-place AA pattern: 1 even, 2 odd phase
  const void *min;               // moments [K][plane] read (equilibrium-shifted storage)
  void *mout;                    // moments written
  int nx, ny, nz, px;            // grid and padded x pitch
  long long plane;               // px * ny * nz
  int with_rho;                  // 1: set 0 is the alpha = 0 set
  int vx;                        // x-nodes per thread of the update kernel (1: scalar)
  int block;                     // threads per block of the update kernel
  double s1, s2;                 // relaxation rates (s0 never acts: m0 = m0eq)
  float s1f, s2f;                // the same rates rounded to FP32 on the host
  double lid_u[3];               // lid velocity
  // derived-field outputs (dense [N] layout), each nullable
  double *P, *u, *rho, *G, *div, *S, *sigma, *omega;
  // init inputs (dense FP64 on the device); Gin [d][d][N] nullable
  const double *Pin, *uin, *Gin;
  // reductions
  double *partials;              // [blocks][k] block partial sums
  double *uprev;                 // [d][N] previous velocity (residual)
  double *result;                // [k] final sums
  int *nonfinite;                // set to 1 when a non-finite value is met
  // dithered rounding of FP32 storage: time step = *clock + tk; the node
  // key is that of global node index key_base + dense local index
  const int *clock;              // device step counter of the launch group
  int tk;                        // this launch's offset in its group
  long long key_base;            // global index of local node 0 (slabs)
};

enum Mode { MODE_STEP = 0, MODE_STEP_FIELDS = 1, MODE_FIELDS = 2 };
enum Storage { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2, ST_F64 = 3, ST_F16EQ = 4, ST_BF16EQ = 5 };
enum ReduceKind { RED_SUMS = 0, RED_RESIDUAL = 1 };

// Block width along x of the auxiliary kernels, and the largest block of the
// update kernels (their width is a launch parameter).
constexpr int kBlockX = 128;
constexpr int kMaxBlock = 256;
// Blocks of the grid-stride reduction pass (a multiple of the 152 SMs).
constexpr int kReduceBlocks = 152 * 4;
constexpr int kReduceThreads = 256;

// Per-lattice launchers (mdf_d2q5.cu, mdf_d3q7.cu).

cudaError_t launch_update_d2q5(int storage, int mode, bool walls, const DevArgs &a,
                               cudaStream_t s);
cudaError_t launch_init_d2q5(int storage, bool walls, const DevArgs &a, cudaStream_t s);
cudaError_t launch_reduce_d2q5(int storage, bool walls, int kind, const DevArgs &a,
                               cudaStream_t s);
cudaError_t launch_update_d3q7(int storage, int mode, bool walls, const DevArgs &a,
                               cudaStream_t s);
cudaError_t launch_init_d3q7(int storage, bool walls, const DevArgs &a, cudaStream_t s);
cudaError_t launch_reduce_d3q7(int storage, bool walls, int kind, const DevArgs &a,
                               cudaStream_t s);

cudaError_t launch_mask_d2q5(const int wall[3], int lid, const DevArgs &a, uint8_t *mask,
                             cudaStream_t s);
cudaError_t launch_mask_d3q7(const int wall[3], int lid, const DevArgs &a, uint8_t *mask,
                             cudaStream_t s);

// Lattices without a rest direction (mdf_d2q4.cu, mdf_d3q6.cu): the
// rest-shifted storage types only.
cudaError_t launch_update_d2q4(int storage, int mode, bool walls, const DevArgs &a,
                               cudaStream_t s);
cudaError_t launch_init_d2q4(int storage, bool walls, const DevArgs &a, cudaStream_t s);
cudaError_t launch_reduce_d2q4(int storage, bool walls, int kind, const DevArgs &a,
                               cudaStream_t s);
cudaError_t launch_mask_d2q4(const int wall[3], int lid, const DevArgs &a, uint8_t *mask,
                             cudaStream_t s);
cudaError_t launch_update_d3q6(int storage, int mode, bool walls, const DevArgs &a,
                               cudaStream_t s);
cudaError_t launch_init_d3q6(int storage, bool walls, const DevArgs &a, cudaStream_t s);
cudaError_t launch_reduce_d3q6(int storage, bool walls, int kind, const DevArgs &a,
                               cudaStream_t s);
cudaError_t launch_mask_d3q6(const int wall[3], int lid, const DevArgs &a, uint8_t *mask,
                             cudaStream_t s);

// The four launchers of one lattice.
struct LatticeLaunch {
  cudaError_t (*update)(int storage, int mode, bool walls, const DevArgs &a, cudaStream_t s);
  cudaError_t (*init)(int storage, bool walls, const DevArgs &a, cudaStream_t s);
  cudaError_t (*reduce)(int storage, bool walls, int kind, const DevArgs &a, cudaStream_t s);
  cudaError_t (*mask)(const int wall[3], int lid, const DevArgs &a, uint8_t *mask, cudaStream_t s);
};
inline const LatticeLaunch *lattice_launch(int d, int q) {
  static const LatticeLaunch d2q5{launch_update_d2q5, launch_init_d2q5, launch_reduce_d2q5, launch_mask_d2q5};
  static const LatticeLaunch d3q7{launch_update_d3q7, launch_init_d3q7, launch_reduce_d3q7, launch_mask_d3q7};
  static const LatticeLaunch d2q4{launch_update_d2q4, launch_init_d2q4, launch_reduce_d2q4, launch_mask_d2q4};
  static const LatticeLaunch d3q6{launch_update_d3q6, launch_init_d3q6, launch_reduce_d3q6, launch_mask_d3q6};
  if (d == 2) return q == 5 ? &d2q5 : q == 4 ? &d2q4 : nullptr;
  if (d == 3) return q == 7 ? &d3q7 : q == 6 ? &d3q6 : nullptr;
  return nullptr;
}

// Sets the device step counter read by the update kernels of a launch group.
cudaError_t launch_set_clock(int *clock, int value, cudaStream_t s);
// Second reduction pass: sums `nblocks` x `k` partials in a fixed order.
cudaError_t launch_reduce_final(const DevArgs &a, int nblocks, int k, cudaStream_t s);
// Dense FP64 [d][N] -> padded [d][plane] in FP32 (f64 = false) or FP64.
cudaError_t launch_pad_force(const double *src, void *dst, bool f64, int d, int nx, int ny,
                             int nz, int px, cudaStream_t s);

}  // namespace mdf

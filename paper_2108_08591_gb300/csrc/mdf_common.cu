// Lattice-independent helper kernels: the fixed-order second reduction pass,
// the padding of body-force fields and the device step counter.
#include "mdf_internal.h"

namespace mdf {

// Sums nblocks x k partials (row-major) into result[k] with one block; each
// thread walks a fixed stride and the block tree is fixed, so the result is
// bitwise reproducible.
__global__ void __launch_bounds__(kReduceThreads) k_reduce_final(const double *__restrict__ partials,
                                                                int nblocks, int k,
                                                                double *__restrict__ result) {
  __shared__ double sh[kReduceThreads];
  for (int c = 0; c < k; ++c) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(long long)b * k + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) result[c] = sh[0];
    __syncthreads();
  }
}

cudaError_t launch_reduce_final(const DevArgs &a, int nblocks, int k, cudaStream_t s) {
  k_reduce_final<<<1, kReduceThreads, 0, s>>>(a.partials, nblocks, k, a.result);
  return cudaGetLastError();
}

__global__ void k_set_clock(int *clock, int value) { *clock = value; }

cudaError_t launch_set_clock(int *clock, int value, cudaStream_t s) {
  k_set_clock<<<1, 1, 0, s>>>(clock, value);
  return cudaGetLastError();
}

template <class T>
__global__ void k_pad_force(const double *__restrict__ src, T *__restrict__ dst, int d, int nx,
                            int ny, int nz, int px) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const long long N = (long long)nx * ny * nz, plane = (long long)px * ny * nz;
  const long long n = ((long long)z * ny + y) * nx + x;
  const long long idx = ((long long)z * ny + y) * px + x;
  for (int b = 0; b < d; ++b) dst[b * plane + idx] = (T)src[b * N + n];
}

cudaError_t launch_pad_force(const double *src, void *dst, bool f64, int d, int nx, int ny, int nz,
                             int px, cudaStream_t s) {
  dim3 grid((unsigned)((nx + kBlockX - 1) / kBlockX), (unsigned)ny, (unsigned)nz);
  if (f64) k_pad_force<double><<<grid, kBlockX, 0, s>>>(src, (double *)dst, d, nx, ny, nz, px);
  else k_pad_force<float><<<grid, kBlockX, 0, s>>>(src, (float *)dst, d, nx, ny, nz, px);
  return cudaGetLastError();
}

}  // namespace mdf

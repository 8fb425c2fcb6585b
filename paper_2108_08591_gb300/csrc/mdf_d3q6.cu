// D3Q6 instantiations of the MDF-LBM kernels (one translation unit per
// lattice so that they compile in parallel).
#include "mdf_kernels.cuh"

namespace mdf {

cudaError_t launch_update_d3q6(int storage, int mode, bool walls, const DevArgs &a,
                               cudaStream_t s) {
  return update_lattice<D3Q6>(storage, mode, walls, a, s);
}

cudaError_t launch_init_d3q6(int storage, bool walls, const DevArgs &a, cudaStream_t s) {
  return init_lattice<D3Q6>(storage, walls, a, s);
}

cudaError_t launch_reduce_d3q6(int storage, bool walls, int kind, const DevArgs &a,
                               cudaStream_t s) {
  return reduce_lattice<D3Q6>(storage, walls, kind, a, s);
}

cudaError_t launch_mask_d3q6(const int wall[3], int lid, const DevArgs &a, uint8_t *mask,
                             cudaStream_t s) {
  return mask_lattice<D3Q6>(wall, lid, a, mask, s);
}

}  // namespace mdf

// D2Q4 instantiations of the MDF-LBM kernels (one translation unit per
// lattice so that they compile in parallel).
#include "mdf_kernels.cuh"

namespace mdf {

cudaError_t launch_update_d2q4(int storage, int mode, bool walls, const DevArgs &a,
                               cudaStream_t s) {
  return update_lattice<D2Q4>(storage, mode, walls, a, s);
}

cudaError_t launch_init_d2q4(int storage, bool walls, const DevArgs &a, cudaStream_t s) {
  return init_lattice<D2Q4>(storage, walls, a, s);
}

cudaError_t launch_reduce_d2q4(int storage, bool walls, int kind, const DevArgs &a,
                               cudaStream_t s) {
  return reduce_lattice<D2Q4>(storage, walls, kind, a, s);
}

cudaError_t launch_mask_d2q4(const int wall[3], int lid, const DevArgs &a, uint8_t *mask,
                             cudaStream_t s) {
  return mask_lattice<D2Q4>(wall, lid, a, mask, s);
}

}  // namespace mdf

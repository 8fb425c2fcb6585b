// D2Q5 instantiations of the MDF-LBM kernels (one translation unit per
// lattice so that they compile in parallel).
#include "mdf_kernels.cuh"

namespace mdf {

cudaError_t launch_update_d2q5(int storage, int mode, bool walls, const DevArgs &a,
                               cudaStream_t s) {
  return update_lattice<D2Q5>(storage, mode, walls, a, s);
}

cudaError_t launch_init_d2q5(int storage, bool walls, const DevArgs &a, cudaStream_t s) {
  return init_lattice<D2Q5>(storage, walls, a, s);
}

cudaError_t launch_reduce_d2q5(int storage, bool walls, int kind, const DevArgs &a,
                               cudaStream_t s) {
  return reduce_lattice<D2Q5>(storage, walls, kind, a, s);
}

cudaError_t launch_mask_d2q5(const int wall[3], int lid, const DevArgs &a, uint8_t *mask,
                             cudaStream_t s) {
  return mask_lattice<D2Q5>(wall, lid, a, mask, s);
}

}  // namespace mdf

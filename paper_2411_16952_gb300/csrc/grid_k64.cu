// Grid-form (tensor-core) sampler kernels for up to 64 modes, one tile buffer (shared memory).
#include "grid_impl.cuh"

namespace tkdv {
void grid_kernels_k64(GridKernels *t) { fill_grid_kernels<64, 1>(t); }
}  // namespace tkdv

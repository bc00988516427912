// Grid-form (tensor-core) sampler kernels for up to 32 modes: single-buffered
// tiles, three CTAs per SM.
#include "grid_impl.cuh"

namespace tkdv {
void grid_kernels_k32(GridKernels *t) { fill_grid_kernels<32, 1>(t); }
}  // namespace tkdv

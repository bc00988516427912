// Grid-form (tensor-core) sampler kernels for up to 16 modes, double-buffered tiles.
#include "grid_impl.cuh"

namespace tkdv {
void grid_kernels_k16(GridKernels *t) { fill_grid_kernels<16, 2>(t); }
}  // namespace tkdv

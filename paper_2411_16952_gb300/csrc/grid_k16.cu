// Grid-form (tensor-core) sampler kernels for up to 16 modes: four or two
// warpgroups per CTA sharing one copy of the basis (two where the grid has
// more than 128 points: every warpgroup holds N columns of tensor memory).
#include "grid_impl.cuh"

namespace tkdv {
void grid_kernels_k16(GridKernels *t) {
    fill_grid_variant<16, 4>(t, 0);
    fill_grid_variant<16, 2>(t, 1);
}
}  // namespace tkdv

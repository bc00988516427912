// Grid-form (tensor-core) sampler kernels for up to 32 modes: three
// warpgroups per CTA at 168 registers, four at 128 (the autotune times
// them), or two where the grid has more than 170 points.
#include "grid_impl.cuh"

namespace tkdv {
void grid_kernels_k32(GridKernels *t) {
    fill_grid_variant<32, 3>(t, 0);
    fill_grid_variant<32, 4>(t, 1);
    fill_grid_variant<32, 2>(t, 2);
}
}  // namespace tkdv

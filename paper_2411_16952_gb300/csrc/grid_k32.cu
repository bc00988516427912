// Grid-form (tensor-core) sampler kernels for up to 32 modes: four
// warpgroups per CTA at 128 registers, three at 168, or two where the grid
// has more than 128 points.  The autotune times every variant that fits.
#include "grid_impl.cuh"

namespace tkdv {
void grid_kernels_k32(GridKernels *t) {
    fill_grid_variant<32, 4>(t, 0);
    fill_grid_variant<32, 3>(t, 1);
    fill_grid_variant<32, 2>(t, 2);
}
}  // namespace tkdv

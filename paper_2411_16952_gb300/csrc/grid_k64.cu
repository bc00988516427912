// Grid-form (tensor-core) sampler kernels for up to 64 modes: two warpgroups
// per CTA (basis 64 KB, two 64 KB tiles of shared memory, all 512 TMEM
// columns).
#include "grid_impl.cuh"

namespace tkdv {
void grid_kernels_k64(GridKernels *t) { fill_grid_variant<64, 2>(t, 0); }
}  // namespace tkdv

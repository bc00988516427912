// Triad-sampler kernels for up to 64 modes: the launch variants with the
// per-lane accept path (the rest of the table is in sampler_k64.cu).
#include "sampler_impl.cuh"

namespace tkdv {
void triad_kernels_k64_lane(TriadKernels *t) { fill_triad_kernels_lane<64>(t); }
}  // namespace tkdv

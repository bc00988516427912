// Triad-sampler kernels for up to 4 modes (K <= 4; modes above K are masked).
#include "sampler_impl.cuh"

namespace tkdv {
void triad_kernels_k4(TriadKernels *t) { fill_triad_kernels<4>(t); }
}  // namespace tkdv

// Triad-sampler kernels for up to 16 modes (K <= 16; modes above K are masked).
#include "sampler_impl.cuh"

namespace tkdv {
void triad_kernels_k16(TriadKernels *t) { fill_triad_kernels<16>(t); }
}  // namespace tkdv

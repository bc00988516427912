// Triad-sampler kernels for up to 32 modes (K <= 32; modes above K are masked).
#include "sampler_impl.cuh"

namespace tkdv {
void triad_kernels_k32(TriadKernels *t) { fill_triad_kernels<32>(t); }
}  // namespace tkdv

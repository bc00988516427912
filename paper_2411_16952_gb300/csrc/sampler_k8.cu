// Triad-sampler kernels for up to 8 modes (K <= 8; modes above K are masked).
#include "sampler_impl.cuh"

namespace tkdv {
void triad_kernels_k8(TriadKernels *t) { fill_triad_kernels<8>(t); }
}  // namespace tkdv

// Triad-sampler kernels for up to 64 modes (K <= 64; modes above K are masked).
#include "sampler_impl.cuh"

namespace tkdv {
void triad_kernels_k64(TriadKernels *t) { fill_triad_kernels<64>(t); }
}  // namespace tkdv

// Triad-sampler kernels for up to 64 modes (K <= 64; modes above K are masked):
// the variants with the accept hand-off, SIR, FP64 pass and replay.  The
// per-lane accept variants compile in sampler_k64_lane.cu, in parallel.
#include "sampler_impl.cuh"

namespace tkdv {
void triad_kernels_k64(TriadKernels *t) {
    fill_triad_kernels_xfer<64>(t);
    triad_kernels_k64_lane(t);
}
}  // namespace tkdv

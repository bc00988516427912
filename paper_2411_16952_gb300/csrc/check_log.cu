// Exhaustive checks of the FP32 radius -2 ln u: every one of the 2^23 values of
// the uniform map against an FP64 logarithm, as the ratio of the error to the
// bound the accept guard band is built on (must not exceed 1).
//   rho_fast (one-thread form): kRhoAbsErr + kRhoRelErr rho
//   rho_log  (warp form):       kRhoLogRelErr rho
#include <cuda_runtime.h>

#include <cstring>

#include "sampler_impl.cuh"
#include "tkdv.h"

namespace tkdv {

template <bool LOG>
__global__ void __launch_bounds__(256) k_check_rho(unsigned long long *worst) {
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= (1u << 23)) return;
    const uint32_t w = m << 9;  // any word of bucket m
    const double u = (2.0 * (double)m + 1.0) * 0x1p-24;
    const double ref = -2.0 * log(u);
    const double got = LOG ? (double)rho_log(w) : (double)rho_fast(w);
    const double bound = LOG ? kRhoLogRelErr * ref : kRhoAbsErr + kRhoRelErr * ref;
    const double err = fabs(got - ref) / bound;
    const unsigned long long key =
        ((unsigned long long)__float_as_uint((float)err) << 32) | (unsigned long long)m;
    atomicMax(worst, key);
}

template <bool LOG>
int check_radius(double *max_ratio, uint32_t *worst_word) {
    if (!max_ratio) return TKDV_ERR_INVALID_ARG;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return TKDV_ERR_OOM;
    unsigned long long h = 0;
    cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        k_check_rho<LOG><<<(1u << 23) / 256, 256>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return TKDV_ERR_CUDA;
    const uint32_t bits = (uint32_t)(h >> 32);
    float f;
    memcpy(&f, &bits, 4);
    *max_ratio = f;
    if (worst_word) *worst_word = (uint32_t)(h & 0xFFFFFFFFu) << 9;
    return TKDV_OK;
}

}  // namespace tkdv

extern "C" int tkdv_check_radius_error(double *max_ratio, uint32_t *worst_word) {
    return tkdv::check_radius<false>(max_ratio, worst_word);
}

extern "C" int tkdv_check_radius_error_log(double *max_ratio, uint32_t *worst_word) {
    return tkdv::check_radius<true>(max_ratio, worst_word);
}

// Largest surface displacement of accepted fields on the 2K-point grid of
// Sec. V.D (the "1-in-m event" of Figs. 8-11 is the field with the largest
// such maximum among m accepted fields).  An opt-in pass over the kept
// records: one warp per record, each lane a few grid points.
#include <cuda_runtime.h>

#include <algorithm>

#include "tkdv_internal.h"

namespace tkdv {

// u(xi_j) = u0s sum_k (xh_k cos k xi_j + xh_{K+k} sin k xi_j) (Eq. 8 with
// Eq. 16), xi_j = -pi + pi j / K, so cos k xi_j = (-1)^k cos(pi k j / K) and
// sin k xi_j = (-1)^k sin(pi k j / K); the phases come from a table of
// cos, sin (pi m / K), m = 0..2K-1, and index k j mod 2K.
__global__ void __launch_bounds__(128) k_field_max(const unsigned char *__restrict__ ring, unsigned long long rec_bytes,
                                                   unsigned long long n, int K,
                                                   const PointConst *__restrict__ pts, float *umax, int *jmax) {
    __shared__ float s_c[2 * kKMax], s_s[2 * kKMax];
    const int G = 2 * K;
    for (int m = threadIdx.x; m < G; m += blockDim.x) {
        float sn, cs;
        sincospif((float)m / (float)K, &sn, &cs);
        s_c[m] = cs;
        s_s[m] = sn;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long r = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n;
         r += warps) {
        const unsigned char *rec = ring + r * rec_bytes;
        const uint32_t point = *reinterpret_cast<const uint32_t *>(rec + 8);
        const float *xh = reinterpret_cast<const float *>(rec + 32);
        float best = -INFINITY;
        int bj = 0;
        for (int j = lane; j < G; j += 32) {
            float acc = 0.f;
            int id = 0;
            for (int k = 1; k <= K; ++k) {
                id += j;
                if (id >= G) id -= G;
                const float t = fmaf(__ldg(&xh[k - 1]), s_c[id], __ldg(&xh[K + k - 1]) * s_s[id]);
                acc = (k & 1) ? acc - t : acc + t;
            }
            if (acc > best) {
                best = acc;
                bj = j;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ob > best || (ob == best && oj < bj)) {
                best = ob;
                bj = oj;
            }
        }
        if (lane == 0) {
            umax[r] = __ldg(&pts[point].u0s) * best;
            jmax[r] = bj;
        }
    }
}

cudaError_t launch_field_max(const unsigned char *ring, unsigned long long rec_bytes, unsigned long long n, int K,
                             const PointConst *pts, float *umax, int *jmax, cudaStream_t st) {
    if (!n) return cudaSuccess;
    const unsigned long long blocks = std::min<unsigned long long>((n + 3) / 4, 65535ull * 16);
    k_field_max<<<(unsigned)blocks, 128, 0, st>>>(ring, rec_bytes, n, K, pts, umax, jmax);
    return cudaGetLastError();
}

}  // namespace tkdv

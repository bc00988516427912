// grid_host.cu - host construction of the grid basis of the tensor-core form:
// row j is the mirror pair of grid points +-xi_j, xi_j = pi (2j + 1)/N,
// j = 0..N/2-1 (the N-point rectangle rule of Eq. 2, offset by half a step);
// column i of the cosine part (i < KA/2) holds -cos(k xi_j) and column
// KA/2 + i of the sine part -sqrt(3) sin(k xi_j), k = i + 1 (the factor makes
// the kernel's pair sum 2 C (C^2 + 3 S^2) one multiply shorter; the sign
// matches the kernel's rows, which hold the draw's components negated), zero
// for modes above K and for the padding; every value is split into BF16
// hi + lo.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "grid_impl.cuh"

namespace tkdv {
namespace {
uint16_t bf16_rn(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
float bf16_to_f(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
}  // namespace

void build_grid_image(int K, int kmax, int ka, int N, unsigned char *out) {
    const int half = N / 2, part = ka / 2;
    const size_t tile = (size_t)half * ka * 2;
    std::memset(out, 0, 2 * tile);
    for (int j = 0; j < half; ++j) {
        const double xi = M_PI * (double)(2 * j + 1) / (double)N;
        for (int i = 0; i < ka; ++i) {
            const int sine = i >= part, k = (i % part) + 1;
            double v = 0.0;
            if (k <= K && k <= kmax) v = sine ? -std::sqrt(3.0) * std::sin(k * xi) : -std::cos(k * xi);
            const uint16_t hi = bf16_rn((float)v);
            const uint16_t lo = bf16_rn((float)(v - (double)bf16_to_f(hi)));
            const uint32_t off = sw128_offset((uint32_t)j, (uint32_t)i, (uint32_t)half);
            std::memcpy(out + off, &hi, 2);
            std::memcpy(out + tile + off, &lo, 2);
        }
    }
}
}  // namespace tkdv

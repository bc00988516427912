// grid_host.cu - host construction of the grid basis of the tensor-core form:
// row j is grid point xi_j = -pi + 2 pi j / N (the rectangle rule of Eq. 2);
// column 8c + 2e + s is mode k = 4c + e + 1 with cos(k xi_j) (s = 0) or
// sin(k xi_j) (s = 1), zero for modes above K and for the padding columns;
// every value is split into BF16 hi + lo.
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
    const size_t tile = (size_t)N * ka * 2;
    std::memset(out, 0, 2 * tile);
    for (int j = 0; j < N; ++j) {
        const double xi = -M_PI + 2.0 * M_PI * (double)j / (double)N;
        for (int i = 0; i < ka; ++i) {
            double v = 0.0;
            const int c = i / 8, e = (i % 8) / 2, s = i % 2;
            const int k = 4 * c + e + 1;
            if (k <= K && k <= kmax) v = s ? std::sin(k * xi) : std::cos(k * xi);
            const uint16_t hi = bf16_rn((float)v);
            const uint16_t lo = bf16_rn((float)(v - (double)bf16_to_f(hi)));
            const uint32_t off = sw128_offset((uint32_t)j, (uint32_t)i, (uint32_t)N);
            std::memcpy(out + off, &hi, 2);
            std::memcpy(out + tile + off, &lo, 2);
        }
    }
}
}  // namespace tkdv

// tkdv_internal.h - structures shared by the host side of the library and its
// CUDA kernels (not part of the public C ABI, see include/tkdv.h for that).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "tkdv.h"

namespace tkdv {

constexpr int kKMax = 128;
constexpr int kMaxPoints = 64;
constexpr int kHistBins = 256;
constexpr int kExcBins = 26;  // exceed-bin e = number of thresholds 0.25 i sigma0 below u0
constexpr uint32_t kRefineCap = 1u << 22;
// grid form: accepted draws one warp holds until the end of its chunk (a
// chunk has at most 64 proposals per thread, so 2048 per warp)
constexpr uint32_t kAcceptSlab = 2048;

// Fixed-point scales of the u0^p moment sums (exact 64-bit integer sums).
constexpr float kQ1 = 268435456.0f;  // 2^28
constexpr float kQ2 = 16777216.0f;   // 2^24
constexpr float kQ3 = 1048576.0f;    // 2^20
constexpr float kQ4 = 65536.0f;      // 2^16
// Fixed-point scale of the per-mode spectrum sums (s_k <= 1: 2^36 accepts per point fit).
constexpr float kSpecScale = 268435456.0f;  // 2^28
// Error bound of the FP32 radius -2 ln u on the fast path (rho_fast):
// |rho_fast - rho| <= kRhoAbsErr + kRhoRelErr * rho for every value of the map.
constexpr double kRhoAbsErr = 0x1p-21;
constexpr double kRhoRelErr = 0x1p-21;
// The radius of the warp form (65..128 modes), -2 logf(u), has only a relative
// error: |rho_log - rho| <= kRhoLogRelErr * rho for every value of the map.
constexpr double kRhoLogRelErr = 0x1p-22;

// Per-point constants, built on the host from the precompute (alpha*, sigma_k,
// log M) and read by every proposal of that point.
struct PointConst {
    float sigma[kKMax];     // sigma_k (k = 1..K), 0 beyond K (masks the mode out)
    float act[kKMax];       // 1 for k <= K, else 0
    double sigma_d[kKMax];  // sigma_k in FP64 for the guard-band recomputation
    // log f/(M g) = cS * S + cH * T + cQ * ln Q - logM, where for xhat = x/|x|
    //   S = sum k^2 s_k            (H2 = E0 S, Eq. 20)
    //   T = sum_n Re(conj(v_n) sum_{k<n} v_k v_{n-k}), v_k = xh_k - i xh_{K+k}
    //       (H3 = 2 pi (E0/2pi)^{3/2} T, Eq. 42)
    //   Q = sum_k s_k / sigma_k^2  (Eq. 33 times 2; = 1 + alpha* beta' S/K^3 for Eq. 40)
    float cS, cH, cQ, logM_f;
    double cS_d, cH_d, cQ_d, logM;
    float u0s;          // u(0) = u0s * sum_k xh_k, u0s = 2 sqrt(E0/2pi)   (Eq. 8)
    float h3s;          // H3 = h3s * T, h3s = 2 pi (E0/2pi)^{3/2}
    float E0;
    float hist_a, hist_b;  // histogram bin = floor(u0 * hist_a + hist_b)
    float exc_a;           // exceed bin = ceil(u0 * exc_a) for u0 > 0
    float guard_abs, guard_rel, guard_h;  // FP32 decision guard (point_table.cpp)
    uint32_t point_id;
    int K;
    float guard_e, guard_q;  // per-draw guard terms for the radius error (point_table.cpp)
    double sir_c;            // SIR: copies per unit exp(log f/(Mg))
    float sir_lnc;           // ln sir_c
    float pad2;
};

// Statistics of one point on the device: only integers, so that the result
// does not depend on the order in which CTAs add to it.
struct StatBlock {
    unsigned long long n_prop, n_acc, n_near, n_refined, n_viol, n_dropped;
    unsigned long long maxd_key;  // order-preserving key of the largest FP32 delta
    unsigned long long q[4];      // sum of round(u0^p * kQScale[p-1]) (two's complement)
    unsigned long long hist[kHistBins];
    unsigned long long exc[kExcBins];
    unsigned long long n_fallback;  // guard-band proposals decided in FP32 (queue full)
    unsigned long long pad[2];
    unsigned long long spec[kKMax];  // sum of round(s_k * kSpecScale), s_k = xh_k^2 + xh_{K+k}^2
    unsigned long long n_kept;       // SIR: proposals with at least one copy
    double sir[7];                   // SIR: sum w, w^2, w S, w u0^p (p = 1..4), w = exp(delta), FP32 terms
};

struct RefineItem {
    unsigned long long idx;
    uint32_t point;
    uint32_t pad;
};

// An accepted draw of the grid form waiting for its outputs.
struct AcceptItem {
    unsigned long long idx;
    float T;      // H3 / (2 pi (E0/2pi)^{3/2}) from the grid contraction
    float delta;  // log f/(Mg) of the FP32 path
};

// Device buffers of one handle.
struct DevBufs {
    const PointConst *pts;
    StatBlock *stats;
    unsigned char *ring;             // records, rec_bytes apart
    unsigned long long *ring_count;  // accepted so far (may exceed capacity)
    RefineItem *refine;              // guard-band proposals of the current run
    uint32_t *counters;              // [0] chunk counter, [1] refine count
    uint32_t *status;                // bit flags (kStatus*)
    unsigned long long ring_cap;
    uint32_t rec_bytes;
    uint32_t refine_cap;
    int sir;  // 1: the FP64 pass draws SIR copy numbers instead of accept bits
    AcceptItem *accs;   // grid form: one slab of acc_slab accepted draws per warp of the launch
    uint32_t acc_slab;
};

constexpr uint32_t kStatusRefineOverflow = 1u;
constexpr uint32_t kStatusDeadline = 2u;
constexpr uint32_t kStatusMbarTimeout = 4u;
constexpr uint32_t kStatusBadArg = 8u;

// Round keys of Philox4x32-10 for the run's key (k0, k1): round r uses
// (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85) mod 2^32, r = 0..9.  Passed with the
// kernel arguments, so that the rounds take their keys as constant operands
// instead of recomputing the key schedule for every block.
struct RoundKeys {
    uint32_t k[20];
};
inline RoundKeys round_keys(uint32_t k0, uint32_t k1) {
    RoundKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk.k[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    return rk;
}

// Arguments of one run (passed by value; the graph updates them per run).
struct RunArgs {
    unsigned long long idx0[kMaxPoints];
    unsigned long long count[kMaxPoints];
    uint32_t chunk_prefix[kMaxPoints + 1];  // cumulative chunk counts
    uint32_t chunk;                          // proposals per chunk
    int n_points;
    unsigned long long deadline_ns;          // 0: none; else per-CTA budget in ns
    float *trace;                            // grid form: (log f/(Mg), T) of point 0's first trace_n
    unsigned long long trace_n;              // proposals, or null
    RoundKeys rk;                            // Philox round keys of the run's seed
};

// Kernel table of one KMAX instantiation of the triad sampler.
struct TriadKernels {
    // [uniform][variant]: 0: 128 threads; 1: 256 threads; 2: 256 threads held
    // to 128 registers (two CTAs per SM); 3..5: the same without the accept
    // hand-off (one-thread form only)
    const void *main[2][6];
    int n_variants;  // variants present (6, or 3 for the warp form)
    const void *sir[2];  // SIR form of the sampler (256 threads), [uniform]
    const void *refine[2];
    const void *replay[2];
    int replay_per_block;  // indices one replay CTA of 128 threads handles
    int xfer_bytes_per_thread;  // dynamic shared memory per thread of variants 0..2 (0: none)
};
void triad_kernels_k4(TriadKernels *t);
void triad_kernels_k8(TriadKernels *t);
void triad_kernels_k16(TriadKernels *t);
void triad_kernels_k32(TriadKernels *t);
void triad_kernels_k64(TriadKernels *t);
void triad_kernels_k64_lane(TriadKernels *t);  // variants 3..5 of the 64-mode table
// 65..128 modes: one warp per batch of four proposals (sampler_k128.cu).
void triad_kernels_k128(TriadKernels *t);

// Kernel table of one KMAX instantiation of the grid (tensor-core) sampler.
constexpr int kGridVariants = 3;
struct GridKernels {
    const void *main[kGridVariants][2];  // [variant][uniform]
    int nwg[kGridVariants];              // warpgroups (tiles, TMEM accumulator pairs) per CTA of each variant
    int n_variants;
    int kmax;                            // modes per part of a tile row
    int ka;                              // contraction length (multiple of 64): [cosine part | sine part]
};
void grid_kernels_k16(GridKernels *t);
void grid_kernels_k32(GridKernels *t);
void grid_kernels_k64(GridKernels *t);
// BF16 hi/lo image of the grid basis (N/2 mirror pairs of grid points as
// rows), already in the 128B-swizzled K-major layout of shared memory: bytes
// [0, (N/2)*KA*2) hi, [(N/2)*KA*2, N*KA*2) lo.
void build_grid_image(int K, int kmax, int ka, int N, unsigned char *out);

constexpr int kTriadVariantThreads[6] = {128, 256, 256, 128, 256, 256};

inline size_t record_bytes(int K) {
    size_t b = 32 + 8 * (size_t)K;
    return (b + 15) & ~(size_t)15;
}

// Host: proposal variances sigma_k^2 (Eq. 25, learned corrections applied)
// and alpha*; returns a TKDV_ status.  s2 has K entries.
int proposal_variances(int K, const tkdv_point &q, double *alpha, double *s2);
// Host: the kernels' constant table of one point (coefficients, scales, guard).
void fill_point_const(int K, const tkdv_point &q, const double *s2, double logM, bool grid, PointConst &c);
// Largest displacement of n kept records on the 2K-point grid (fields.cu).
cudaError_t launch_field_max(const unsigned char *ring, unsigned long long rec_bytes, unsigned long long n, int K,
                             const PointConst *pts, float *umax, int *jmax, cudaStream_t st);

}  // namespace tkdv

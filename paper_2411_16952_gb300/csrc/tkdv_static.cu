// tkdv_static.cu - sampler_run_static(): one sampler run that allocates no
// memory at all, for callers that cannot call cudaMalloc.
//
// Who needs it: code whose device memory belongs to another allocator (a
// framework that reserved the whole device pool up front, so cudaMalloc
// fails or fragments it), latency-critical loops where cudaMalloc/cudaFree
// would synchronise the device, and plugin hosts whose rules forbid device
// allocation.  The regular handle API (sampler_create_ex) allocates its
// buffers with cudaMalloc; this entry point instead keeps its scratch in the
// file-scope array below, which every GPU that loads this library holds
// until the process exits.
//
// The run itself is the same persistent sampler and FP64 guard-band kernels
// as sampler_run_ranges(), launched on pointers into that array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/tkdv.h"
#include "tkdv_internal.h"

using namespace tkdv;

namespace {

// Scratch layout: [header | guard-band queue].  The header holds the point's
// constant table, its statistics block, the two run counters, the record
// counter and the status word.
struct StaticHeader {
    PointConst pc;
    StatBlock stats;
    uint32_t counters[2];
    unsigned long long ring_count;
    uint32_t status;
    uint32_t pad;
};

constexpr size_t kHeaderBytes = (sizeof(StaticHeader) + 255) & ~(size_t)255;
constexpr size_t kQueueBytes = (size_t)TKDV_STATIC_MAX_PROPOSALS * sizeof(RefineItem);
constexpr size_t kScratchBytes = kHeaderBytes + kQueueBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::once_flag g_once[kMaxDevices];
unsigned char *g_scratch_ptr[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];

// Same per-point table as the handle API builds (point_table.cpp), built
// without any allocation.
int fill_point(int K, const tkdv_point &q, PointConst &c, double &alpha) {
    if (!(q.E0 > 0) || !std::isfinite(q.E0)) return TKDV_ERR_INVALID_ARG;
    if (!(q.beta_p >= 0) || !std::isfinite(q.beta_p)) return TKDV_ERR_INVALID_ARG;
    if (!std::isfinite(q.r)) return TKDV_ERR_INVALID_ARG;
    if (q.proposal < 0 || q.proposal > 2) return TKDV_ERR_INVALID_ARG;
    if (!q.override_logM || !std::isfinite(q.logM))
        return TKDV_ERR_INVALID_ARG;
    if (q.proposal == TKDV_PROPOSAL_LEARNED && !q.log_var_correction)
        return TKDV_ERR_INVALID_ARG;
    double s2[kKMax];
    const int rc = proposal_variances(K, q, &alpha, s2);
    if (rc != TKDV_OK) return rc;
    fill_point_const(K, q, s2, q.logM, false, c);
    return TKDV_OK;
}

}  // namespace

extern "C" int sampler_run_static(int K, const tkdv_point *point, uint64_t idx0, uint64_t n_proposals,
                                  uint64_t seed, void *records, uint64_t capacity, uint64_t *n_records,
                                  tkdv_stats *stats, void *cuda_stream) {
    if (K < 1 || K > kKMax) return TKDV_ERR_INVALID_ARG;
    if (!point) return TKDV_ERR_INVALID_ARG;
    if (n_proposals > TKDV_STATIC_MAX_PROPOSALS) return TKDV_ERR_TOO_LARGE;
    if (capacity > 0 && !records) return TKDV_ERR_INVALID_ARG;
    PointConst pc;
    double alpha = 1.0;
    int rc = fill_point(K, *point, pc, alpha);
    if (rc) return rc;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return TKDV_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return TKDV_ERR_UNSUPPORTED;
    // Once per device, with that device current: the device address of the
    // scratch array (its name in host code is only a stand-in for it).
    std::call_once(g_once[dev], [dev]() {
        void *p = nullptr;
        g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_static_scratch);
        g_scratch_ptr[dev] = (unsigned char *)p;
    });
    if (g_scratch_err[dev] != cudaSuccess || !g_scratch_ptr[dev])
        return TKDV_ERR_CUDA;
    unsigned char *base = g_scratch_ptr[dev];
    StaticHeader *hdr = (StaticHeader *)base;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    TriadKernels kt{};
    int kmax = 128;
    for (int m : {4, 8, 16, 32, 64, 128})
        if (K <= m) {
            kmax = m;
            break;
        }
    switch (kmax) {
        case 4: triad_kernels_k4(&kt); break;
        case 8: triad_kernels_k8(&kt); break;
        case 16: triad_kernels_k16(&kt); break;
        case 32: triad_kernels_k32(&kt); break;
        case 64: triad_kernels_k64(&kt); break;
        default: triad_kernels_k128(&kt); break;
    }
    const int uni = point->proposal == TKDV_PROPOSAL_UNIFORM ? 1 : 0;
    const void *fn = kt.main[uni][kmax == 128 ? 2 : 1];  // warp form: two CTAs per SM
    int sms = 0, nb = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the triad form's accept hand-off: dynamic shared memory beyond the 48 KB default
    const size_t dyn = (size_t)256 * kt.xfer_bytes_per_thread;
    if (e == cudaSuccess && dyn)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess && dyn)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, 256, dyn);
    if (e != cudaSuccess) return TKDV_ERR_CUDA;
    const int ctas = std::max(1, nb) * sms;

    DevBufs B{};
    B.pts = &hdr->pc;
    B.stats = &hdr->stats;
    B.ring = (unsigned char *)records;
    B.ring_count = &hdr->ring_count;
    B.refine = (RefineItem *)(base + kHeaderBytes);
    B.counters = hdr->counters;
    B.status = &hdr->status;
    B.ring_cap = records ? capacity : 0;
    B.rec_bytes = (uint32_t)record_bytes(K);
    B.refine_cap = TKDV_STATIC_MAX_PROPOSALS;

    RunArgs A;
    std::memset(&A, 0, sizeof(A));
    A.n_points = 1;
    A.idx0[0] = idx0;
    A.count[0] = n_proposals;
    unsigned long long chunk = (n_proposals + 8ull * ctas - 1) / (8ull * ctas);
    chunk = (chunk + 255) / 256 * 256;
    chunk = std::max(256ull, std::min(256ull * 64ull, chunk));
    A.chunk = (uint32_t)chunk;
    A.chunk_prefix[0] = 0;
    A.chunk_prefix[1] = (uint32_t)((n_proposals + chunk - 1) / chunk);
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    A.rk = round_keys(k0, k1);

    // The array keeps the previous call's contents: clear the header (the
    // statistics, counters and status must start at zero), then upload the
    // point table.  The queue needs no clearing (its count is in the header).
    e = cudaMemsetAsync(base, 0, sizeof(StaticHeader), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hdr->pc, &pc, sizeof(pc), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return TKDV_ERR_CUDA;
    if (n_proposals > 0) {
        void *margs[] = {&B, &A, &k0, &k1};
        e = cudaLaunchKernel(fn, dim3(ctas), dim3(256), margs, dyn, st);
        if (e == cudaSuccess) {
            void *rargs[] = {&B, &k0, &k1};
            e = cudaLaunchKernel(kt.refine[uni], dim3(sms * 4), dim3(128), rargs, 0, st);
        }
        if (e != cudaSuccess) return TKDV_ERR_CUDA;
    }
    StatBlock sb;
    unsigned long long ring_count = 0;
    uint32_t status = 0;
    e = cudaMemcpyAsync(&sb, &hdr->stats, sizeof(sb), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ring_count, &hdr->ring_count, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &hdr->status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return TKDV_ERR_CUDA;
    if (n_records) *n_records = std::min<unsigned long long>(ring_count, B.ring_cap);
    if (stats) {
        tkdv_stats &o = *stats;
        std::memset(&o, 0, sizeof(o));
        o.n_proposals = sb.n_prop;
        o.n_accepted = sb.n_acc;
        o.n_near_threshold = sb.n_near;
        o.n_refined = sb.n_refined;
        o.n_envelope_violations = sb.n_viol;
        o.n_dropped = sb.n_dropped;
        o.n_fallback = sb.n_fallback;
        if (sb.maxd_key == 0) {
            o.max_delta = -INFINITY;
        } else {
            uint32_t k = (uint32_t)sb.maxd_key;
            uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
            float f;
            std::memcpy(&f, &b, 4);
            o.max_delta = f;
        }
        o.logM = point->logM;
        o.alpha_star = alpha;
        const double qs[4] = {kQ1, kQ2, kQ3, kQ4};
        for (int q = 0; q < 4; ++q) o.sum_u0[q] = (double)(long long)sb.q[q] / qs[q];
        const double n = (double)sb.n_acc;
        if (n > 0) {
            const double m1 = o.sum_u0[0] / n, m2 = o.sum_u0[1] / n, m3 = o.sum_u0[2] / n, m4 = o.sum_u0[3] / n;
            o.mean = m1;
            o.var = m2 - m1 * m1;
            o.skew = (m3 - 3 * m1 * m2 + 2 * m1 * m1 * m1) / std::pow(o.var, 1.5);
            o.kurt = (m4 - 4 * m1 * m3 + 6 * m1 * m1 * m2 - 3 * m1 * m1 * m1 * m1) / (o.var * o.var);
        } else {
            o.mean = o.var = o.skew = o.kurt = NAN;
        }
        for (int b = 0; b < kHistBins; ++b) o.hist[b] = sb.hist[b];
        const double ucap = std::sqrt(2.0 * K * point->E0 / M_PI);
        o.hist_lo = -ucap;
        o.hist_hi = ucap;
        for (int i = 0; i < TKDV_N_EXCEED; ++i) {
            unsigned long long t = 0;
            for (int j = i + 1; j < kExcBins; ++j) t += sb.exc[j];
            o.exceed[i] = t;
        }
        for (int m = 0; m < K && m < TKDV_KMAX; ++m) o.spectrum[m] = (double)sb.spec[m] / (double)kSpecScale;
    }
    if (status & kStatusDeadline) return TKDV_ERR_TIMEOUT;
    return TKDV_OK;
}

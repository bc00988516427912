// tkdv_api.cu - the C ABI of include/tkdv.h: handle life cycle, per-point
// precompute, the launch of one run (memset -> persistent sampler -> FP64
// guard-band pass, as one CUDA graph), statistics and records.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tkdv.h"
#include "tkdv_internal.h"

using namespace tkdv;

namespace {

thread_local std::string g_create_error;

struct Launch {
    int threads = 256;
    int ctas = 0;
    int variant = 1;  // triad form: index into TriadKernels::main[][variant]
    int form = TKDV_H3_TRIAD_F32;
};

}  // namespace

struct tkdv_sampler {
    int K = 0, kmax = 0, n_points = 0;
    tkdv_options opt{};
    std::vector<tkdv_point> pts;
    std::vector<double> alpha, logM;
    std::vector<std::vector<double>> sigma2;
    std::vector<PointConst> pc;            // table of the current form (uploaded)
    std::vector<PointConst> pc_triad, pc_grid;  // both forms' tables (the grid guard is wider)
    bool grid_ok = false;                  // the grid form's resources exist (grid mode, or AUTO on sm_10x)
    std::vector<unsigned long long> next_idx;
    bool all_uniform = false;
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevBufs dev{};
    void *d_pts = nullptr, *d_stats = nullptr, *d_ring = nullptr, *d_ring_count = nullptr,
         *d_refine = nullptr, *d_counters = nullptr, *d_status = nullptr, *d_accs = nullptr;
    size_t rec_bytes = 0;
    TriadKernels kt{};
    GridKernels kg{};
    int grid_N = 0;
    void *d_bimg = nullptr;   // grid form: BF16 hi/lo basis image
    size_t dyn_smem[kGridVariants] = {};  // grid form: dynamic shared memory per CTA of each variant
    bool gvalid[kGridVariants] = {};      // grid form: the variant fits (TMEM, shared memory) for this grid_N
    int gfirst = 0;                       // grid form: the default variant (the first that fits)
    float *trace = nullptr;   // grid form: optional per-proposal trace (device)
    unsigned long long trace_n = 0;
    Launch launch;
    unsigned long long deadline_ns = 0;
    // graph of one run: memset(counters) -> sampler -> refine
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t n_main = nullptr, n_refine = nullptr;
    Launch graph_launch;
    // kernel arguments (the graph nodes point at copies made at update time)
    RunArgs args{};
    uint32_t key0 = 0, key1 = 0;
    std::string err;
};

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            h->err = std::string(#call) + " failed: " + cudaGetErrorString(e_);              \
            return e_ == cudaErrorMemoryAllocation ? TKDV_ERR_OOM : TKDV_ERR_CUDA;            \
        }                                                                                     \
    } while (0)

namespace {

int fail(tkdv_sampler *h, int code, const std::string &msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return code;
}

int kmax_for(int K) {
    for (int m : {4, 8, 16, 32, 64, 128})
        if (K <= m) return m;
    return 0;
}

// Per-point precompute and the constant table of one point.
int build_point(tkdv_sampler *h, int p, std::string &msg) {
    const tkdv_point &q = h->pts[p];
    const int K = h->K;
    if (!(q.E0 > 0) || !std::isfinite(q.E0)) {
        msg = "point " + std::to_string(p) + ": E0 must be > 0";
        return TKDV_ERR_INVALID_ARG;
    }
    if (!(q.beta_p >= 0) || !std::isfinite(q.beta_p)) {
        msg = "point " + std::to_string(p) + ": beta' must be >= 0";
        return TKDV_ERR_INVALID_ARG;
    }
    if (!std::isfinite(q.r)) {
        msg = "point " + std::to_string(p) + ": C3/C2 must be finite";
        return TKDV_ERR_INVALID_ARG;
    }
    if (q.proposal < 0 || q.proposal > 2) {
        msg = "point " + std::to_string(p) + ": unknown proposal";
        return TKDV_ERR_INVALID_ARG;
    }
    if (q.proposal == TKDV_PROPOSAL_LEARNED && !q.log_var_correction) {
        msg = "point " + std::to_string(p) + ": learned proposal needs log_var_correction";
        return TKDV_ERR_INVALID_ARG;
    }
    double alpha = 1.0;
    std::vector<double> s2(K, 1.0);
    {
        const int rc = proposal_variances(K, q, &alpha, s2.data());
        if (rc == TKDV_ERR_NO_ALPHA) {
            msg = "point " + std::to_string(p) + ": no root alpha* of F (beta' >= K^2 sum 1/k^2)";
            return rc;
        }
        if (rc != TKDV_OK) {
            msg = "point " + std::to_string(p) + ": invalid proposal (non-finite log-variance correction?)";
            return rc;
        }
    }
    double lm = q.logM;
    if (!q.override_logM) {
        int rc = tkdv_log_M(K, q.beta_p, q.E0, q.r, q.proposal == TKDV_PROPOSAL_UNIFORM ? nullptr : s2.data(),
                            &lm);
        if (rc != TKDV_OK) {
            msg = "point " + std::to_string(p) + ": envelope search failed";
            return rc;
        }
    } else if (!std::isfinite(lm)) {
        msg = "point " + std::to_string(p) + ": overridden log M is not finite";
        return TKDV_ERR_INVALID_ARG;
    }
    h->alpha[p] = alpha;
    h->logM[p] = lm;
    h->sigma2[p] = s2;

    fill_point_const(K, q, s2.data(), lm, false, h->pc_triad[p]);
    fill_point_const(K, q, s2.data(), lm, true, h->pc_grid[p]);
    h->pc[p] = h->opt.h3_mode == TKDV_H3_GRID_BF16X3 ? h->pc_grid[p] : h->pc_triad[p];
    return TKDV_OK;
}

bool is_grid(const tkdv_sampler *h) { return h->launch.form == TKDV_H3_GRID_BF16X3; }

// Threads per CTA of launch variant `variant` of the current form.
int variant_threads(const tkdv_sampler *h, int variant) {
    return is_grid(h) ? 128 * h->kg.nwg[variant] : kTriadVariantThreads[variant];
}

// Switch the form of the next runs (TKDV_H3_AUTO handles): its point table
// and its default launch shape; the graph is rebuilt on the next run.
int set_form(tkdv_sampler *h, int form) {
    h->launch.form = form;
    h->pc = form == TKDV_H3_GRID_BF16X3 ? h->pc_grid : h->pc_triad;
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(h->d_pts, h->pc.data(), sizeof(PointConst) * h->n_points, cudaMemcpyHostToDevice));
    if (form == TKDV_H3_GRID_BF16X3) {
        h->launch.variant = h->gfirst;
        h->launch.threads = variant_threads(h, h->gfirst);
    } else {
        h->launch.threads = 256;
        h->launch.variant = h->kmax == 128 ? 2 : 1;
    }
    return TKDV_OK;
}

const void *main_fn(const tkdv_sampler *h, int variant) {
    const int uni = h->all_uniform ? 1 : 0;
    if (is_grid(h)) return h->kg.main[variant][uni];
    if (h->opt.sir) return h->kt.sir[uni];  // one form (256 threads)
    return h->kt.main[uni][variant];
}

// Dynamic shared memory of one CTA of the current form in launch variant
// `variant` with `threads` threads: the grid form's tiles, or the triad
// form's accept hand-off (variants 0..2; none in SIR runs and in the warp form).
size_t main_dyn_smem(const tkdv_sampler *h, int variant, int threads) {
    if (is_grid(h)) return h->dyn_smem[variant];
    if (h->opt.sir || variant >= 3) return 0;
    return (size_t)threads * (size_t)h->kt.xfer_bytes_per_thread;
}

// TMEM columns one grid-form CTA of launch variant `variant` allocates:
// N per warpgroup (its C and S accumulators), rounded up to a power of two.
int grid_tmem_cols(const tkdv_sampler *h, int variant) {
    int c = 32;
    while (c < h->grid_N * h->kg.nwg[variant]) c <<= 1;
    return c;
}



// Largest number of resident CTAs per SM for the handle's form.
int max_ctas_per_sm(tkdv_sampler *h, int variant, int threads, int *out) {
    int nb = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, main_fn(h, variant), threads,
                                                     main_dyn_smem(h, variant, threads)));
    if (is_grid(h)) {
        // The grid kernel's residency follows from its own limits: shared
        // memory (with the per-block reservation), allocated registers, and
        // the 512 TMEM columns of an SM.  (The occupancy query above has been
        // seen to answer one CTA where two are resident.)
        cudaFuncAttributes fa{};
        int smem_sm = 0, resv = 0, regs_sm = 0;
        CK(cudaFuncGetAttributes(&fa, main_fn(h, variant)));
        CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device));
        CK(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, h->device));
        CK(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, h->device));
        const size_t smem_blk = h->dyn_smem[variant] + fa.sharedSizeBytes + (size_t)resv;
        const int regs_thr = (fa.numRegs + 7) / 8 * 8;
        const int regs_blk = ((regs_thr * 32 + 255) / 256 * 256) * ((threads + 31) / 32);
        int by_smem = (int)((size_t)smem_sm / smem_blk);
        int by_regs = regs_blk > 0 ? regs_sm / regs_blk : 1;
        int by_tmem = 512 / grid_tmem_cols(h, variant);
        const int own = std::max(1, std::min(by_smem, std::min(by_regs, by_tmem)));
        if (std::getenv("TKDV_AUTOTUNE_LOG"))
            std::fprintf(stderr, "tkdv occupancy: query %d, shared memory %d, registers %d (%d/thread), TMEM %d\n",
                         nb, by_smem, by_regs, fa.numRegs, by_tmem);
        nb = own;
    }
    *out = nb;
    return TKDV_OK;
}

int set_default_launch(tkdv_sampler *h) {
    const int thr = h->launch.threads;
    int nb = 0;
    int rc = max_ctas_per_sm(h, h->launch.variant, thr, &nb);
    if (rc) return rc;
    if (nb < 1) return fail(h, TKDV_ERR_CUDA, "sampler kernel does not fit on an SM");
    int per_sm = h->opt.ctas_per_sm > 0 ? std::min(h->opt.ctas_per_sm, nb) : nb;
    h->launch.ctas = per_sm * h->num_sms;
    return TKDV_OK;
}

// RunArgs for explicit ranges.
int build_args(tkdv_sampler *h, const unsigned long long *idx0, const unsigned long long *count,
               uint64_t seed) {
    RunArgs &a = h->args;
    std::memset(&a, 0, sizeof(a));
    a.n_points = h->n_points;
    unsigned long long total = 0;
    for (int p = 0; p < h->n_points; ++p) {
        a.idx0[p] = idx0[p];
        a.count[p] = count[p];
        total += count[p];
    }
    // about 8 chunks per persistent worker (a CTA of the triad form, a
    // warpgroup of the grid form), between 1 and 64 proposals per thread
    const bool grid = is_grid(h);
    const unsigned long long thr = grid ? 128ull : (unsigned long long)h->launch.threads;
    const unsigned long long workers =
        (unsigned long long)h->launch.ctas * (grid ? (unsigned long long)h->kg.nwg[h->launch.variant] : 1ull);
    unsigned long long target = (total + 8ull * workers - 1) / (8ull * workers);
    target = (target + thr - 1) / thr * thr;
    target = std::max(thr, std::min(thr * 64ull, target));
    a.chunk = (uint32_t)target;
    unsigned long long acc = 0;
    a.chunk_prefix[0] = 0;
    for (int p = 0; p < h->n_points; ++p) {
        acc += (count[p] + a.chunk - 1) / a.chunk;
        if (acc >= 0xFFFFFFF0ull) return fail(h, TKDV_ERR_INVALID_ARG, "run too large (> 2^32 chunks)");
        a.chunk_prefix[p + 1] = (uint32_t)acc;
    }
    a.deadline_ns = h->deadline_ns;
    a.trace = h->trace;
    a.trace_n = h->trace ? h->trace_n : 0ull;
    h->key0 = (uint32_t)seed;
    h->key1 = (uint32_t)(seed >> 32);
    a.rk = round_keys(h->key0, h->key1);
    return TKDV_OK;
}

int refine_grid(tkdv_sampler *h) { return std::max(1, h->num_sms * 4); }

int build_graph(tkdv_sampler *h) {
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    if (h->graph) {
        cudaGraphDestroy(h->graph);
        h->graph = nullptr;
    }
    CK(cudaGraphCreate(&h->graph, 0));
    cudaMemsetParams ms{};
    ms.dst = h->d_counters;
    ms.value = 0;
    ms.elementSize = 4;
    ms.width = 4;
    ms.height = 1;
    ms.pitch = 0;
    cudaGraphNode_t n_ms;
    CK(cudaGraphAddMemsetNode(&n_ms, h->graph, nullptr, 0, &ms));
    const int uni = h->all_uniform ? 1 : 0;
    const unsigned char *bimg = (const unsigned char *)h->d_bimg;
    int gN = h->grid_N;
    void *margs[] = {&h->dev, &h->args, &h->key0, &h->key1, &bimg, &gN};
    cudaKernelNodeParams kp{};
    kp.func = (void *)main_fn(h, h->launch.variant);
    kp.gridDim = dim3(h->launch.ctas);
    kp.blockDim = dim3(h->launch.threads);
    kp.sharedMemBytes = (unsigned)main_dyn_smem(h, h->launch.variant, h->launch.threads);
    kp.kernelParams = margs;
    CK(cudaGraphAddKernelNode(&h->n_main, h->graph, &n_ms, 1, &kp));
    void *rargs[] = {&h->dev, &h->key0, &h->key1};
    cudaKernelNodeParams rp{};
    rp.func = (void *)h->kt.refine[uni];
    rp.gridDim = dim3(refine_grid(h));
    rp.blockDim = dim3(128);
    rp.kernelParams = rargs;
    CK(cudaGraphAddKernelNode(&h->n_refine, h->graph, &h->n_main, 1, &rp));
    CK(cudaGraphInstantiate(&h->exec, h->graph, 0));
    h->graph_launch = h->launch;
    return TKDV_OK;
}

int enqueue(tkdv_sampler *h) {
    const int uni = h->all_uniform ? 1 : 0;
    if (h->opt.use_graph) {
        if (!h->exec || h->graph_launch.ctas != h->launch.ctas || h->graph_launch.threads != h->launch.threads ||
            h->graph_launch.variant != h->launch.variant || h->graph_launch.form != h->launch.form) {
            int rc = build_graph(h);
            if (rc) return rc;
        }
        const unsigned char *bimg = (const unsigned char *)h->d_bimg;
        int gN = h->grid_N;
        void *margs[] = {&h->dev, &h->args, &h->key0, &h->key1, &bimg, &gN};
        cudaKernelNodeParams kp{};
        kp.func = (void *)main_fn(h, h->launch.variant);
        kp.gridDim = dim3(h->launch.ctas);
        kp.blockDim = dim3(h->launch.threads);
        kp.sharedMemBytes = (unsigned)main_dyn_smem(h, h->launch.variant, h->launch.threads);
        kp.kernelParams = margs;
        CK(cudaGraphExecKernelNodeSetParams(h->exec, h->n_main, &kp));
        void *rargs[] = {&h->dev, &h->key0, &h->key1};
        cudaKernelNodeParams rp{};
        rp.func = (void *)h->kt.refine[uni];
        rp.gridDim = dim3(refine_grid(h));
        rp.blockDim = dim3(128);
        rp.kernelParams = rargs;
        CK(cudaGraphExecKernelNodeSetParams(h->exec, h->n_refine, &rp));
        CK(cudaGraphLaunch(h->exec, h->stream));
        return TKDV_OK;
    }
    CK(cudaMemsetAsync(h->d_counters, 0, 16, h->stream));
    const unsigned char *bimg = (const unsigned char *)h->d_bimg;
    int gN = h->grid_N;
    void *margs[] = {&h->dev, &h->args, &h->key0, &h->key1, &bimg, &gN};
    CK(cudaLaunchKernel(main_fn(h, h->launch.variant), dim3(h->launch.ctas), dim3(h->launch.threads), margs,
                        main_dyn_smem(h, h->launch.variant, h->launch.threads), h->stream));
    void *rargs[] = {&h->dev, &h->key0, &h->key1};
    CK(cudaLaunchKernel(h->kt.refine[uni], dim3(refine_grid(h)), dim3(128), rargs, 0, h->stream));
    return TKDV_OK;
}

int run_ranges(tkdv_sampler *h, const unsigned long long *idx0, const unsigned long long *count,
               uint64_t seed) {
    unsigned long long total = 0;
    for (int p = 0; p < h->n_points; ++p) total += count[p];
    if (total == 0) return TKDV_OK;
    int rc = build_args(h, idx0, count, seed);
    if (rc) return rc;
    return enqueue(h);
}

int check_status(tkdv_sampler *h) {
    uint32_t st = 0;
    CK(cudaMemcpy(&st, h->d_status, 4, cudaMemcpyDeviceToHost));
    if (st) CK(cudaMemset(h->d_status, 0, 4));
    if (st & (kStatusDeadline | kStatusMbarTimeout))
        return fail(h, TKDV_ERR_TIMEOUT,
                    (st & kStatusDeadline) ? "run stopped at its deadline" : "device wait timed out");
    if (st & kStatusRefineOverflow)
        h->err = "FP64 guard-band queue overflowed; the overflow was decided in FP32 (see n_fallback)";
    return TKDV_OK;
}

void free_all(tkdv_sampler *h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (void *p : {h->d_pts, h->d_stats, h->d_ring, h->d_ring_count, h->d_refine, h->d_counters, h->d_status,
                    h->d_bimg, h->d_accs})
        if (p) cudaFree(p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

}  // namespace

extern "C" {

size_t tkdv_record_bytes(int K) { return record_bytes(K); }

int sampler_create(int K, double beta_p, double E0, double r, int proposal, tkdv_sampler **out) {
    tkdv_point p{};
    p.beta_p = beta_p;
    p.E0 = E0;
    p.r = r;
    p.proposal = proposal;
    tkdv_options o{};
    o.K = K;
    o.h3_mode = TKDV_H3_TRIAD_F32;
    o.sample_capacity = 1ull << 20;
    o.use_graph = 1;
    return sampler_create_ex(&p, 1, &o, out);
}

int sampler_create_ex(const tkdv_point *points, int n_points, const tkdv_options *opt, tkdv_sampler **out) {
    if (!out) return fail(nullptr, TKDV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!points || !opt) return fail(nullptr, TKDV_ERR_INVALID_ARG, "points/options NULL");
    if (n_points < 1 || n_points > kMaxPoints)
        return fail(nullptr, TKDV_ERR_INVALID_ARG, "n_points must be in 1..64");
    if (opt->K < 1 || opt->K > kKMax) return fail(nullptr, TKDV_ERR_INVALID_ARG, "K must be in 1..128");
    if (opt->h3_mode != TKDV_H3_TRIAD_F32 && opt->h3_mode != TKDV_H3_GRID_BF16X3 && opt->h3_mode != TKDV_H3_AUTO)
        return fail(nullptr, TKDV_ERR_INVALID_ARG, "unknown h3_mode");
    // AUTO: the grid form is a candidate where it exists (K <= 64, not SIR)
    const bool want_grid = opt->h3_mode == TKDV_H3_GRID_BF16X3 ||
                           (opt->h3_mode == TKDV_H3_AUTO && opt->K <= 64 && !opt->sir);
    int gridN = 0;
    if (want_grid) {
        gridN = opt->grid_N ? opt->grid_N : ((3 * opt->K + 1 + 31) / 32) * 32;
        if (gridN % 32 != 0 || gridN <= 3 * opt->K || gridN > 256)
            return fail(nullptr, TKDV_ERR_INVALID_ARG,
                        "grid_N must be a multiple of 32, larger than 3K and at most 256");
    }
    if (opt->threads_per_cta != 0 && opt->threads_per_cta != 128 && opt->threads_per_cta != 256)
        return fail(nullptr, TKDV_ERR_INVALID_ARG, "threads_per_cta must be 0, 128 or 256");
    if (opt->sir != 0 && opt->sir != 1) return fail(nullptr, TKDV_ERR_INVALID_ARG, "sir must be 0 or 1");
    if (opt->sir && opt->h3_mode == TKDV_H3_GRID_BF16X3)
        return fail(nullptr, TKDV_ERR_UNSUPPORTED, "SIR runs use the triad form");
    if (opt->sir && opt->K > 64) return fail(nullptr, TKDV_ERR_UNSUPPORTED, "SIR runs need K <= 64");
    if (opt->sir)
        for (int p = 0; p < n_points; ++p)
            if (!(points[p].sir_c > 0) || !std::isfinite(points[p].sir_c))
                return fail(nullptr, TKDV_ERR_INVALID_ARG, "SIR: every point needs sir_c > 0");
    tkdv_sampler *h = new tkdv_sampler();
    h->K = opt->K;
    h->kmax = kmax_for(opt->K);
    h->grid_N = gridN;
    h->n_points = n_points;
    h->opt = *opt;
    h->pts.assign(points, points + n_points);
    h->alpha.assign(n_points, 1.0);
    h->logM.assign(n_points, 0.0);
    h->sigma2.assign(n_points, {});
    h->pc.assign(n_points, PointConst{});
    h->pc_triad.assign(n_points, PointConst{});
    h->pc_grid.assign(n_points, PointConst{});
    h->next_idx.assign(n_points, 0ull);
    h->all_uniform = true;
    for (int p = 0; p < n_points; ++p) {
        std::string msg;
        int rc = build_point(h, p, msg);
        if (rc) {
            delete h;
            return fail(nullptr, rc, msg);
        }
        if (points[p].proposal != TKDV_PROPOSAL_UNIFORM) h->all_uniform = false;
    }
    switch (h->kmax) {
        case 4: triad_kernels_k4(&h->kt); break;
        case 8: triad_kernels_k8(&h->kt); break;
        case 16: triad_kernels_k16(&h->kt); break;
        case 32: triad_kernels_k32(&h->kt); break;
        case 64: triad_kernels_k64(&h->kt); break;
        default: triad_kernels_k128(&h->kt); break;
    }
    auto bail = [&](int rc) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return rc;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        h->err = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return bail(TKDV_ERR_CUDA);
    }
    // the triad form's accept hand-off may exceed the 48 KB default
    if (h->kt.xfer_bytes_per_thread > 0) {
        for (int u = 0; u < 2 && e == cudaSuccess; ++u)
            for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
                e = cudaFuncSetAttribute(h->kt.main[u][v], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTriadVariantThreads[v] * h->kt.xfer_bytes_per_thread);
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(h->kt.main[u][v], cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared);
            }
        if (e != cudaSuccess) {
            h->err = std::string("triad kernel shared memory: ") + cudaGetErrorString(e);
            return bail(TKDV_ERR_CUDA);
        }
    }
    h->launch.threads = opt->threads_per_cta ? opt->threads_per_cta : 256;
    h->launch.variant = h->launch.threads == 128 ? 0 : 1;
    // the warp form (K > 64) fits two 256-thread CTAs per SM at 128 registers
    if (h->kmax == 128 && h->launch.threads == 256) h->launch.variant = 2;
    if (opt->sir) {
        h->launch.threads = 256;
        h->launch.variant = 1;
    }
    bool grid_here = want_grid;
    if (want_grid) {
        int major = 0;
        e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device);
        if (e != cudaSuccess || major != 10) {
            if (opt->h3_mode == TKDV_H3_GRID_BF16X3) {
                h->err = "the tensor-core grid form needs an sm_10x (tcgen05) device";
                return bail(TKDV_ERR_UNSUPPORTED);
            }
            grid_here = false;  // AUTO on another device: the triad form only
        }
    }
    if (grid_here) {
        if (h->K <= 16)
            grid_kernels_k16(&h->kg);
        else if (h->K <= 32)
            grid_kernels_k32(&h->kg);
        else
            grid_kernels_k64(&h->kg);
        h->grid_ok = true;
        h->launch.form = TKDV_H3_GRID_BF16X3;
        h->pc = h->pc_grid;
        const size_t btile = (size_t)(gridN / 2) * h->kg.ka * 2, atile = (size_t)128 * h->kg.ka * 2;
        // a variant fits if its warpgroups' accumulators (N columns each) fit
        // the 512 TMEM columns of an SM and its tiles the shared memory
        int smem_optin = 0;
        e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
        h->gfirst = -1;
        for (int v = 0; v < h->kg.n_variants && e == cudaSuccess; ++v) {
            h->dyn_smem[v] = 2 * btile + (size_t)h->kg.nwg[v] * 2 * atile + 1024;
            cudaFuncAttributes fa{};
            e = cudaFuncGetAttributes(&fa, h->kg.main[v][0]);
            if (e != cudaSuccess) break;
            h->gvalid[v] = h->kg.nwg[v] * gridN <= 512 && h->dyn_smem[v] + fa.sharedSizeBytes <= (size_t)smem_optin;
            if (!h->gvalid[v]) continue;
            if (h->gfirst < 0) h->gfirst = v;
            for (int u = 0; u < 2 && e == cudaSuccess; ++u) {
                e = cudaFuncSetAttribute(h->kg.main[v][u], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)h->dyn_smem[v]);
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(h->kg.main[v][u], cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared);
            }
        }
        if (e != cudaSuccess) {
            h->err = std::string("grid kernel shared memory: ") + cudaGetErrorString(e);
            return bail(TKDV_ERR_CUDA);
        }
        if (h->gfirst < 0) {
            h->err = "no grid-form launch fits this grid_N";
            return bail(TKDV_ERR_UNSUPPORTED);
        }
        h->launch.variant = h->gfirst;
        h->launch.threads = variant_threads(h, h->gfirst);
        std::vector<unsigned char> img(2 * btile);
        build_grid_image(h->K, h->kg.kmax, h->kg.ka, gridN, img.data());
        e = cudaMalloc(&h->d_bimg, img.size());
        if (e == cudaSuccess) e = cudaMemcpy(h->d_bimg, img.data(), img.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            h->err = std::string("grid basis: ") + cudaGetErrorString(e);
            return bail(e == cudaErrorMemoryAllocation ? TKDV_ERR_OOM : TKDV_ERR_CUDA);
        }
    }
    h->rec_bytes = record_bytes(h->K);
    const unsigned long long cap = opt->sample_capacity;
    auto alloc = [&](void **p, size_t bytes) -> int {
        cudaError_t ee = cudaMalloc(p, bytes ? bytes : 16);
        if (ee != cudaSuccess) {
            h->err = std::string("cudaMalloc: ") + cudaGetErrorString(ee);
            return ee == cudaErrorMemoryAllocation ? TKDV_ERR_OOM : TKDV_ERR_CUDA;
        }
        return TKDV_OK;
    };
    int rc;
    if ((rc = alloc(&h->d_pts, sizeof(PointConst) * n_points))) return bail(rc);
    if ((rc = alloc(&h->d_stats, sizeof(StatBlock) * n_points))) return bail(rc);
    if ((rc = alloc(&h->d_ring, h->rec_bytes * cap))) return bail(rc);
    if ((rc = alloc(&h->d_ring_count, 8))) return bail(rc);
    if ((rc = alloc(&h->d_refine, sizeof(RefineItem) * (size_t)kRefineCap))) return bail(rc);
    if ((rc = alloc(&h->d_counters, 16))) return bail(rc);
    if ((rc = alloc(&h->d_status, 4))) return bail(rc);
    if (opt->cuda_stream) {
        h->stream = (cudaStream_t)opt->cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            h->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            return bail(TKDV_ERR_CUDA);
        }
        h->own_stream = true;
    }
    e = cudaMemcpy(h->d_pts, h->pc.data(), sizeof(PointConst) * n_points, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->d_stats, 0, sizeof(StatBlock) * n_points);
    if (e == cudaSuccess) e = cudaMemset(h->d_ring_count, 0, 8);
    if (e == cudaSuccess) e = cudaMemset(h->d_counters, 0, 16);
    if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, 4);
    if (e != cudaSuccess) {
        h->err = std::string("initialising device buffers: ") + cudaGetErrorString(e);
        return bail(TKDV_ERR_CUDA);
    }
    h->dev.pts = (const PointConst *)h->d_pts;
    h->dev.stats = (StatBlock *)h->d_stats;
    h->dev.ring = (unsigned char *)h->d_ring;
    h->dev.ring_count = (unsigned long long *)h->d_ring_count;
    h->dev.refine = (RefineItem *)h->d_refine;
    h->dev.counters = (uint32_t *)h->d_counters;
    h->dev.status = (uint32_t *)h->d_status;
    h->dev.ring_cap = cap;
    h->dev.rec_bytes = (uint32_t)h->rec_bytes;
    h->dev.refine_cap = kRefineCap;
    h->dev.sir = opt->sir;
    if ((rc = set_default_launch(h))) return bail(rc);
    if (h->grid_ok) {
        // one slab of accepted draws per warp of the largest grid-form launch
        size_t warps = 0;
        const int form0 = h->launch.form;
        h->launch.form = TKDV_H3_GRID_BF16X3;
        for (int v = 0; v < h->kg.n_variants; ++v) {
            if (!h->gvalid[v]) continue;
            int nb = 0;
            if ((rc = max_ctas_per_sm(h, v, variant_threads(h, v), &nb))) return bail(rc);
            warps = std::max(warps, (size_t)std::max(nb, 1) * h->num_sms * h->kg.nwg[v] * 4);
        }
        h->launch.form = form0;
        if ((rc = alloc(&h->d_accs, warps * kAcceptSlab * sizeof(AcceptItem)))) return bail(rc);
        h->dev.accs = (AcceptItem *)h->d_accs;
        h->dev.acc_slab = kAcceptSlab;
    }
    *out = h;
    return TKDV_OK;
}

int sampler_run(tkdv_sampler *h, uint64_t n_proposals, uint64_t seed) {
    if (!h) return TKDV_ERR_INVALID_ARG;
    std::vector<uint64_t> b(h->n_points, n_proposals);
    return sampler_run_budgets(h, b.data(), seed);
}

int sampler_run_budgets(tkdv_sampler *h, const uint64_t *budgets, uint64_t seed) {
    if (!h || !budgets) return TKDV_ERR_INVALID_ARG;
    std::vector<unsigned long long> i0(h->n_points), c(h->n_points);
    for (int p = 0; p < h->n_points; ++p) {
        i0[p] = h->next_idx[p];
        c[p] = budgets[p];
    }
    int rc = run_ranges(h, i0.data(), c.data(), seed);
    if (rc) return rc;
    for (int p = 0; p < h->n_points; ++p) h->next_idx[p] += budgets[p];
    return TKDV_OK;
}

int sampler_run_ranges(tkdv_sampler *h, const uint64_t *idx0, const uint64_t *count, uint64_t seed) {
    if (!h || !idx0 || !count) return TKDV_ERR_INVALID_ARG;
    std::vector<unsigned long long> i0(idx0, idx0 + h->n_points), c(count, count + h->n_points);
    return run_ranges(h, i0.data(), c.data(), seed);
}

int sampler_sync(tkdv_sampler *h) {
    if (!h) return TKDV_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    return check_status(h);
}

int sampler_set_trace(tkdv_sampler *h, void *dev_buf, uint64_t n) {
    if (!h || (n && !dev_buf)) return TKDV_ERR_INVALID_ARG;
    if (!is_grid(h)) return fail(h, TKDV_ERR_UNSUPPORTED, "the trace is written by the grid form only");
    h->trace = n ? (float *)dev_buf : nullptr;
    h->trace_n = n;
    return TKDV_OK;
}

int sampler_set_deadline_ns(tkdv_sampler *h, uint64_t ns) {
    if (!h) return TKDV_ERR_INVALID_ARG;
    h->deadline_ns = ns;
    return TKDV_OK;
}

int sampler_stats(tkdv_sampler *h, tkdv_stats *out, int n_out) {
    if (!h || !out || n_out < 0 || n_out > h->n_points) return TKDV_ERR_INVALID_ARG;
    int rc = sampler_sync(h);
    std::vector<StatBlock> sb(h->n_points);
    CK(cudaMemcpy(sb.data(), h->d_stats, sizeof(StatBlock) * h->n_points, cudaMemcpyDeviceToHost));
    for (int p = 0; p < n_out; ++p) {
        const StatBlock &s = sb[p];
        tkdv_stats &o = out[p];
        std::memset(&o, 0, sizeof(o));
        o.n_proposals = s.n_prop;
        o.n_accepted = s.n_acc;
        o.n_near_threshold = s.n_near;
        o.n_refined = s.n_refined;
        o.n_envelope_violations = s.n_viol;
        o.n_dropped = s.n_dropped;
        o.n_fallback = s.n_fallback;
        if (s.maxd_key == 0) {
            o.max_delta = -INFINITY;
        } else {
            uint32_t k = (uint32_t)s.maxd_key;
            uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
            float f;
            std::memcpy(&f, &b, 4);
            o.max_delta = f;
        }
        o.logM = h->logM[p];
        o.alpha_star = h->alpha[p];
        const double qs[4] = {kQ1, kQ2, kQ3, kQ4};
        for (int q = 0; q < 4; ++q) o.sum_u0[q] = (double)(long long)s.q[q] / qs[q];
        const double n = (double)s.n_acc;
        if (n > 0) {
            const double m1 = o.sum_u0[0] / n, m2 = o.sum_u0[1] / n, m3 = o.sum_u0[2] / n, m4 = o.sum_u0[3] / n;
            o.mean = m1;
            o.var = m2 - m1 * m1;
            const double c3 = m3 - 3 * m1 * m2 + 2 * m1 * m1 * m1;
            const double c4 = m4 - 4 * m1 * m3 + 6 * m1 * m1 * m2 - 3 * m1 * m1 * m1 * m1;
            o.skew = c3 / std::pow(o.var, 1.5);
            o.kurt = c4 / (o.var * o.var);
        } else {
            o.mean = o.var = o.skew = o.kurt = NAN;
        }
        for (int b = 0; b < kHistBins; ++b) o.hist[b] = s.hist[b];
        const double ucap = std::sqrt(2.0 * h->K * h->pts[p].E0 / M_PI);
        o.hist_lo = -ucap;
        o.hist_hi = ucap;
        for (int i = 0; i < TKDV_N_EXCEED; ++i) {
            unsigned long long t = 0;
            for (int e = i + 1; e < kExcBins; ++e) t += s.exc[e];
            o.exceed[i] = t;
        }
        for (int m = 0; m < h->K && m < TKDV_KMAX; ++m) o.spectrum[m] = (double)s.spec[m] / (double)kSpecScale;
        o.n_kept = s.n_kept;
        o.sir_sum_w = s.sir[0];
        o.sir_sum_w2 = s.sir[1];
        o.sir_sum_wS = s.sir[2];
        for (int q = 0; q < 4; ++q) o.sir_sum_w_u0[q] = s.sir[3 + q];
    }
    return rc;
}

int sampler_samples(tkdv_sampler *h, void *dst, int dst_on_device, uint64_t max_records, uint64_t *n_out) {
    if (!h || (!dst && max_records) || !n_out) return TKDV_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    unsigned long long cnt = 0;
    CK(cudaMemcpy(&cnt, h->d_ring_count, 8, cudaMemcpyDeviceToHost));
    unsigned long long n = std::min<unsigned long long>(cnt, h->dev.ring_cap);
    n = std::min<unsigned long long>(n, max_records);
    if (n) CK(cudaMemcpy(dst, h->d_ring, n * h->rec_bytes, dst_on_device ? cudaMemcpyDeviceToDevice
                                                                           : cudaMemcpyDeviceToHost));
    *n_out = n;
    return TKDV_OK;
}

int sampler_field_maxima(tkdv_sampler *h, uint64_t max_records, double *umax, int32_t *jmax, uint64_t *n_out) {
    if (!h || !n_out || (max_records && !umax)) return TKDV_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    unsigned long long cnt = 0;
    CK(cudaMemcpy(&cnt, h->d_ring_count, 8, cudaMemcpyDeviceToHost));
    unsigned long long n = std::min<unsigned long long>(cnt, h->dev.ring_cap);
    n = std::min<unsigned long long>(n, max_records);
    *n_out = n;
    if (!n) return TKDV_OK;
    float *d_u = nullptr;
    int *d_j = nullptr;
    if (cudaMalloc(&d_u, 4 * n) != cudaSuccess) return fail(h, TKDV_ERR_OOM, "field maxima: out of device memory");
    if (cudaMalloc(&d_j, 4 * n) != cudaSuccess) {
        cudaFree(d_u);
        return fail(h, TKDV_ERR_OOM, "field maxima: out of device memory");
    }
    cudaError_t e = launch_field_max((const unsigned char *)h->d_ring, h->rec_bytes, n, h->K,
                                     (const PointConst *)h->d_pts, d_u, d_j, h->stream);
    std::vector<float> hu(n);
    std::vector<int> hj(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpy(hu.data(), d_u, 4 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hj.data(), d_j, 4 * n, cudaMemcpyDeviceToHost);
    cudaFree(d_u);
    cudaFree(d_j);
    if (e != cudaSuccess) return fail(h, TKDV_ERR_CUDA, cudaGetErrorString(e));
    for (unsigned long long i = 0; i < n; ++i) {
        umax[i] = hu[i];
        if (jmax) jmax[i] = hj[i];
    }
    return TKDV_OK;
}

int sampler_reset(tkdv_sampler *h) {
    if (!h) return TKDV_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemset(h->d_stats, 0, sizeof(StatBlock) * h->n_points));
    CK(cudaMemset(h->d_ring_count, 0, 8));
    CK(cudaMemset(h->d_status, 0, 4));
    std::fill(h->next_idx.begin(), h->next_idx.end(), 0ull);
    return TKDV_OK;
}

int sampler_point_info(tkdv_sampler *h, int p, double *alpha_star, double *logM, double *sigma2) {
    if (!h || p < 0 || p >= h->n_points) return TKDV_ERR_INVALID_ARG;
    if (alpha_star) *alpha_star = h->alpha[p];
    if (logM) *logM = h->logM[p];
    if (sigma2)
        for (int k = 0; k < h->K; ++k) sigma2[k] = h->sigma2[p][k];
    return TKDV_OK;
}

int sampler_replay(tkdv_sampler *h, int p, const uint64_t *idx, uint64_t n, uint64_t seed, double *out) {
    if (!h || p < 0 || p >= h->n_points || (!idx && n) || (!out && n)) return TKDV_ERR_INVALID_ARG;
    if (n == 0) return TKDV_OK;
    const size_t row = 8 + 2 * (size_t)h->K;
    void *d_idx = nullptr, *d_out = nullptr;
    CK(cudaMalloc(&d_idx, 8 * n));
    cudaError_t e = cudaMalloc(&d_out, sizeof(double) * row * n);
    if (e != cudaSuccess) {
        cudaFree(d_idx);
        return fail(h, TKDV_ERR_OOM, "replay buffers");
    }
    const int uni = h->all_uniform ? 1 : 0;
    const PointConst *P = h->dev.pts + p;
    unsigned long long nn = n;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    void *args[] = {(void *)&P, &d_idx, &nn, &k0, &k1, &d_out};
    e = cudaMemcpyAsync(d_idx, idx, 8 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaLaunchKernel(h->kt.replay[uni], dim3((unsigned)((n + h->kt.replay_per_block - 1) / h->kt.replay_per_block)),
                             dim3(128), args, 0, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(double) * row * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d_idx);
    cudaFree(d_out);
    if (e != cudaSuccess) return fail(h, TKDV_ERR_CUDA, std::string("replay: ") + cudaGetErrorString(e));
    return TKDV_OK;
}

int sampler_autotune(tkdv_sampler *h, uint64_t calib_proposals, double *best_us) {
    if (!h || calib_proposals == 0) return TKDV_ERR_INVALID_ARG;
    const int saved_graph = h->opt.use_graph;
    h->opt.use_graph = 0;
    std::vector<unsigned long long> i0(h->n_points, 1ull << 62), c(h->n_points, calib_proposals);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    Launch best = h->launch;
    float best_ms = 1e30f;
    // TKDV_H3_AUTO with both forms available: time both and keep the faster
    std::vector<int> forms = {h->launch.form};
    if (h->opt.h3_mode == TKDV_H3_AUTO && h->grid_ok) forms = {TKDV_H3_GRID_BF16X3, TKDV_H3_TRIAD_F32};
    for (int form : forms) {
        if (form != h->launch.form) {
            const int rcf = set_form(h, form);
            if (rcf) return rcf;
        }
        std::vector<int> var_list;
        const int nvar = is_grid(h) ? h->kg.n_variants : h->kt.n_variants;
        for (int v = 0; v < nvar; ++v)
            if (!is_grid(h) || h->gvalid[v]) var_list.push_back(v);
        if (h->opt.sir) var_list = {1};
        for (int var : var_list) {
            const int thr = variant_threads(h, var);
            int nb = 0;
            const int rc0 = max_ctas_per_sm(h, var, thr, &nb);
            if (rc0) return rc0;
            for (int per = 1; per <= nb; ++per) {
                h->launch.threads = thr;
                h->launch.variant = var;
                h->launch.ctas = per * h->num_sms;
                float ms_best = 1e30f;
                for (int rep = 0; rep < 5; ++rep) {  // the first warms up; best of four
                    CK(cudaEventRecord(e0, h->stream));
                    const int rc = run_ranges(h, i0.data(), c.data(), 0x5EEDull + rep);
                    if (rc) return rc;
                    CK(cudaEventRecord(e1, h->stream));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    if (rep > 0) ms_best = std::min(ms_best, ms);
                }
                if (std::getenv("TKDV_AUTOTUNE_LOG"))
                    std::fprintf(stderr, "tkdv autotune: form %s variant %d threads %d ctas/SM %d -> %.3f ms\n",
                                 is_grid(h) ? "grid" : "triad", var, thr, per, (double)ms_best);
                if (ms_best < best_ms) {
                    best_ms = ms_best;
                    best = h->launch;
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best.form != h->launch.form) {
        const int rcf = set_form(h, best.form);
        if (rcf) return rcf;
    }
    h->launch = best;
    h->opt.use_graph = saved_graph;
    if (best_us) *best_us = best_ms * 1000.0;
    return sampler_reset(h);
}

int sampler_set_launch(tkdv_sampler *h, int variant, int ctas_per_sm) {
    if (!h || ctas_per_sm < 0) return TKDV_ERR_INVALID_ARG;
    bool ok;
    if (is_grid(h))
        ok = variant >= 0 && variant < h->kg.n_variants && h->gvalid[variant];
    else if (h->opt.sir)
        ok = variant == 1;
    else
        ok = variant >= 0 && variant < h->kt.n_variants;
    if (!ok) return fail(h, TKDV_ERR_INVALID_ARG, "no such launch variant for this handle's form");
    const int thr = variant_threads(h, variant);
    int nb = 0;
    const int rc = max_ctas_per_sm(h, variant, thr, &nb);
    if (rc) return rc;
    if (nb < 1) return fail(h, TKDV_ERR_CUDA, "sampler kernel does not fit on an SM");
    if (ctas_per_sm > nb) return fail(h, TKDV_ERR_INVALID_ARG, "ctas_per_sm above the occupancy maximum");
    h->launch.threads = thr;
    h->launch.variant = variant;
    h->launch.ctas = (ctas_per_sm ? ctas_per_sm : nb) * h->num_sms;
    return TKDV_OK;
}

int sampler_h3_form(const tkdv_sampler *h) {
    if (!h) return TKDV_ERR_INVALID_ARG;
    return h->launch.form;
}

int sampler_batch_run(const tkdv_point *points, int n_points, const tkdv_options *opt, const uint64_t *budgets,
                      uint64_t seed, tkdv_stats *out) {
    if (!budgets || !out) return fail(nullptr, TKDV_ERR_INVALID_ARG, "budgets/out NULL");
    tkdv_sampler *h = nullptr;
    int rc = sampler_create_ex(points, n_points, opt, &h);
    if (rc) return rc;
    rc = sampler_run_budgets(h, budgets, seed);
    if (!rc) rc = sampler_stats(h, out, n_points);
    if (rc) g_create_error = h->err;
    sampler_destroy(h);
    return rc;
}

int sampler_launch_config(tkdv_sampler *h, int *ctas, int *threads_per_cta, uint32_t *chunk) {
    if (!h) return TKDV_ERR_INVALID_ARG;
    if (ctas) *ctas = h->launch.ctas;
    if (threads_per_cta) *threads_per_cta = h->launch.threads;
    if (chunk) *chunk = h->args.chunk;
    return TKDV_OK;
}

const char *sampler_last_error(const tkdv_sampler *h) {
    return h ? h->err.c_str() : g_create_error.c_str();
}

void sampler_destroy(tkdv_sampler *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

}  // extern "C"

// sampler_k128.cu - the rejection sampler for 65..128 modes (Sec. IV.B of
// Moore & Foerster, arXiv 2411.16952, at the K = 128 of Fig. 7): one warp per
// batch of four proposals, the batch's state in shared memory.
//
// At K = 128 one proposal holds 256 floats, too many for one thread's
// registers, and the double sum of Eq. (42) has 4096 distinct triads.  So a
// warp draws four proposals at once: lane L makes modes 2j, 2j+1 for the
// Philox blocks j = L and L + 32 of every proposal (the stream rule of the
// one-thread sampler, so both forms draw the same states), writes the scaled
// pairs (x_m, y_m) to shared memory and keeps its share of |x|^2, S|x|^2,
// Q|x|^2, u(0) and the smallest radius word, which warp reductions complete.
//
// The double sum, for v_k = x_k - i y_k,
//   T = sum_{k, l >= 1, k + l <= K} Re(v_k v_l conj(v_{k+l})),
// is cut into 8 x 8 tiles of (k, l) pairs over blocks kb <= lb of eight
// modes: a tile with kb < lb stands for (k, l) and (l, k) and has weight 2;
// a diagonal tile holds all ordered pairs of its block and has weight 1.  The
// 72 tiles with kb + lb <= 15 hold every pair with k + l <= 128; modes above
// K read as zero, which removes the pairs with k + l > K.  A batch has
// 4 x 72 = 288 tiles, nine rounds of one tile per lane with every lane on the
// same instruction stream.  A tile loads its 8 + 8 modes and the 15 sums
// k + l, sums the products of each anti-diagonal i + j = d in packed FP32
//   P1 = sum (x_k x_l, y_k y_l),  P2 = sum (y_k x_l, x_k y_l)
// and weights them by v_{k+l} once per anti-diagonal.  Every term passes
// through at most 50 roundings (8 in P, 31 in the tile, 3 over rounds, 5 in
// the warp reduction, 3 in the scaling), within the chain of 64 the decision
// guard of point_table.cpp allows the warp form, so the guard band and the
// FP64 pass (k_refine_warp) keep every accept decision exact.  The radius is
// rho_log, the full-precision logarithm, whose error is purely relative: the
// guard needs no per-draw radius terms and is about ten times narrower than
// it would be with the fast radius, so that about 0.15 % of the draws at
// K = 128 reach the FP64 pass.
//
// Shared-memory layout: proposal q of a warp at word q * kWS, mode m at word
// m + m/8 (one pad word per block of eight), so that lanes reading the same
// mode of consecutive blocks hit distinct banks.  Modes K..135 stay zero.
#include "sampler_impl.cuh"

namespace tkdv {
namespace {

constexpr int kWK = 128;                      // modes of the layout
constexpr int kWQ = 4;                        // proposals per warp batch
constexpr int kWS = 153;                      // float2 words per proposal (mode 135 at word 151)
constexpr int kWTiles = 72;                   // tiles per proposal
constexpr int kWRounds = kWQ * kWTiles / 32;  // tile rounds per batch (9)
static_assert(kWQ * kWTiles == 32 * kWRounds, "tiles must fill whole rounds");

__device__ __forceinline__ int wpos(int m) { return m + (m >> 3); }

// Tile t of a batch: proposal q = t / 72 and the (kb, lb) pair number t % 72
// in the order kb = 0..7, lb = kb..15-kb.  x: word offsets of the k and l
// blocks; y: word offset of block kb + lb, q << 16, weight << 24.
__device__ uint2 tile_entry(int t) {
    const int q = t / kWTiles;
    int f = t % kWTiles, kb = 0;
    while (f >= 16 - 2 * kb) {
        f -= 16 - 2 * kb;
        ++kb;
    }
    const int lb = kb + f;
    const uint32_t base = (uint32_t)(q * kWS);
    uint2 e;
    e.x = (base + 9u * kb) | ((base + 9u * lb) << 16);
    e.y = (base + 9u * (kb + lb)) | ((uint32_t)q << 16) | ((kb < lb ? 2u : 1u) << 24);
    return e;
}

// sum over the tile's pairs of Re(v_k v_l conj(v_{k+l})), unweighted.
__device__ __forceinline__ float tile_sum(const float2 *sv, uint32_t ko, uint32_t lo, uint32_t no) {
    f32x2_t A[8], As[8], Bv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float2 a = sv[ko + i];
        A[i] = pk2(a.x, a.y);
        As[i] = pk2(a.y, a.x);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float2 b = sv[lo + j];
        Bv[j] = pk2(b.x, b.y);
    }
    f32x2_t P1[15], P2[15];
#pragma unroll
    for (int d = 0; d < 15; ++d) P1[d] = P2[d] = 0ull;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            P1[i + j] = fma2(A[i], Bv[j], P1[i + j]);
            P2[i + j] = fma2(As[i], Bv[j], P2[i + j]);
        }
    }
    float t = 0.f;
#pragma unroll
    for (int d = 0; d < 15; ++d) {
        // k + l = 8 (kb + lb) + d + 2, i.e. mode 8 (kb + lb) + d + 1
        const float2 vn = sv[no + (d + 1) + ((d + 1) >> 3)];
        float a0, a1, b0, b1;
        upk2(P1[d], a0, a1);
        upk2(P2[d], b0, b1);
        t = fmaf(vn.x, a0 - a1, t);
        t = fmaf(vn.y, b0 + b1, t);
    }
    return t;
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;  // the same value in every lane (each level adds a commuting pair)
}

__device__ __forceinline__ float sel4(const float *a, int q) {
    return q == 0 ? a[0] : q == 1 ? a[1] : q == 2 ? a[2] : a[3];
}

// One batch of the fast path: the four proposals' draws, reductions and T.
// On return every lane holds the values of proposal ql = lane & 3.
struct WEval {
    float nrm2, Sraw, zz, u0raw, T;
    uint32_t wmin;
};

template <bool UNIF>
__device__ __forceinline__ WEval warp_batch(float2 *sv, const uint2 *s_tab, const float *sig, const float *act,
                                            int K, const uint32_t *lo, const uint32_t *hi, uint32_t vmask,
                                            uint32_t pid, uint32_t k0, uint32_t k1, int lane) {
    float nrm2[kWQ], Sraw[kWQ], zz[kWQ], u0raw[kWQ];
    uint32_t wmin[kWQ];
#pragma unroll
    for (int q = 0; q < kWQ; ++q) {
        nrm2[q] = Sraw[q] = zz[q] = u0raw[q] = 0.f;
        wmin[q] = 0xFFFFFFFFu;
    }
    // Steps 1-3: lane L makes the Philox blocks L and L + 32 of every proposal.
    // The radius is rho_log (purely relative error), so the outputs of
    // accepted draws need no second pass and the guard no per-draw terms.
#pragma unroll
    for (int i = 0; i < 2 * kWQ; ++i) {
        const int q = i >> 1;
        const int j = lane + 32 * (i & 1);
        if (((vmask >> q) & 1u) && 2 * j < K) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)j, lo[q], hi[q], pid), k0, k1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = 2 * j + h;
                const float s = UNIF ? act[m] : sig[m];
                const float rho = rho_log(h ? w.z : w.x);
                const float a = (-s * rho) * rsqrt_approx(rho);
                float sn, cs;
                sincos_approx(angle_f(h ? w.w : w.y), sn, cs);
                const float xm = a * cs, ym = a * sn;
                if (m < K) wmin[q] = min(wmin[q], h ? w.z : w.x);
                sv[q * kWS + wpos(m)] = make_float2(xm, ym);
                const float sk = (s * s) * rho;
                nrm2[q] += sk;
                Sraw[q] = fmaf((float)((m + 1) * (m + 1)), sk, Sraw[q]);
                zz[q] += s > 0.f ? rho : 0.f;
                u0raw[q] += xm;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kWQ; ++q) {
        nrm2[q] = wsum(nrm2[q]);
        Sraw[q] = wsum(Sraw[q]);
        zz[q] = wsum(zz[q]);
        u0raw[q] = wsum(u0raw[q]);
        wmin[q] = __reduce_min_sync(0xffffffffu, wmin[q]);
    }
    __syncwarp();
    // Step 4: nine rounds of one tile per lane.
    float Tq[kWQ] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int r = 0; r < kWRounds; ++r) {
        const uint2 e = s_tab[r * 32 + lane];
        const float t = tile_sum(sv, e.x & 0xFFFFu, e.x >> 16, e.y & 0xFFFFu) * (float)(e.y >> 24);
        const int q = (int)((e.y >> 16) & 0xFFu);
#pragma unroll
        for (int qq = 0; qq < kWQ; ++qq) Tq[qq] += q == qq ? t : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kWQ; ++q) Tq[q] = wsum(Tq[q]);
    const int ql = lane & 3;
    WEval ev;
    ev.nrm2 = sel4(nrm2, ql);
    ev.Sraw = sel4(Sraw, ql);
    ev.zz = sel4(zz, ql);
    ev.u0raw = sel4(u0raw, ql);
    ev.T = sel4(Tq, ql);
    ev.wmin = ql == 0 ? wmin[0] : ql == 1 ? wmin[1] : ql == 2 ? wmin[2] : wmin[3];
    return ev;
}

// Steps 5-6 for the lane's proposal (the formulas of eval_fast).
template <bool UNIF>
__device__ __forceinline__ Fast warp_eval(const WEval &ev, const Scal &c, uint32_t wacc) {
    Fast f;
    const float inv2 = rcp_rn(ev.nrm2);
    f.inv = rsqrt_approx(ev.nrm2);
    f.S = ev.Sraw * inv2;
    f.T = ev.T * (inv2 * f.inv);
    const float tS = c.cS * f.S;
    const float tH = c.cH * f.T;
    const float tQ = UNIF ? 0.f : c.cQ * logf(ev.zz * inv2);
    f.delta = ((tS + tH) + tQ) - c.logM;
    f.lnU = -0.5f * rho_fast(wacc);
    f.d = f.lnU - f.delta;
    // the warp form's guard has no per-draw radius terms (guard_e = guard_q = 0)
    f.guard = c.ga + c.gr * (fabsf(tS) + fabsf(tQ) + fabsf(tH) + fabsf(f.lnU) + fabsf(c.logM)) + c.gh;
    return f;
}

// Shared state common to the sampler and the replay kernel: tile table,
// proposal variances and the warps' state slabs (zeroed: modes above K).
template <int NW>
struct WShared {
    uint2 tab[32 * kWRounds];
    float sig[kWK], act[kWK];
    float2 v[NW][kWQ * kWS];
};

template <int NW>
__device__ void wshared_init(WShared<NW> &sh, int tid, int nt) {
    for (int t = tid; t < 32 * kWRounds; t += nt) sh.tab[t] = tile_entry(t);
    float2 *v = &sh.v[0][0];
    for (int e = tid; e < NW * kWQ * kWS; e += nt) v[e] = make_float2(0.f, 0.f);
}

// ---- FP64 pass of the warp form -------------------------------------------
// The same draw and formulas as eval64 (sampler_impl.cuh), spread over a warp:
// lane L makes the modes of Philox blocks L and L + 32 into the slab sx (FP64
// pairs, zero from K on), and the double sum of Eq. (42), folded,
//   T = sum_{n=2}^{K} Re(conj(v_n) W_n),
//   W_n = 2 sum_{k < n-k} v_k v_{n-k} + [n even] v_{n/2}^2,
// takes rows n and 131 - n as one loop of 64 pairs (n = 3..65): two such
// loops per lane, and row 2 on lane 31.  Rows above K read v_n = 0.  Every
// lane returns the proposal's values.
__device__ __forceinline__ double wsum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void row_end(const double2 *sx, int n, double A, double B, double &t) {
    A *= 2.0;
    B *= 2.0;
    if ((n & 1) == 0) {
        const double2 h = sx[n / 2 - 1];
        A = fma(h.x, h.x, A);
        A = fma(-h.y, h.y, A);
        B = fma(2.0 * h.x, h.y, B);
    }
    const double2 vn = sx[n - 1];
    t = fma(vn.x, A, t);
    t = fma(vn.y, B, t);
}

// rows n1 < n2 with (n1 - 1)/2 + (n2 - 1)/2 = 64 folded pairs
__device__ __forceinline__ void fold_pair(const double2 *sx, int n1, int n2, double &t) {
    const int len1 = (n1 - 1) / 2;
    double A = 0.0, B = 0.0;
    int n = n1, k = 1;
    for (int i = 0; i < 64; ++i) {
        if (i == len1) {
            row_end(sx, n1, A, B, t);
            A = 0.0;
            B = 0.0;
            n = n2;
            k = 1;
        }
        const double2 a = sx[k - 1], b = sx[n - k - 1];
        A = fma(a.x, b.x, A);
        A = fma(-a.y, b.y, A);
        B = fma(a.x, b.y, B);
        B = fma(a.y, b.x, B);
        ++k;
    }
    row_end(sx, n2, A, B, t);
}

template <bool UNIF>
__device__ __noinline__ void eval64_warp(const PointConst *P, unsigned long long idx, uint32_t k0, uint32_t k1,
                                         double2 *sx, int lane, Out64 &o, double &inv_out) {
    const int K = P->K;
    const uint32_t lo = (uint32_t)idx, hi = (uint32_t)(idx >> 32), pid = P->point_id;
    double nrm2 = 0.0, Sraw = 0.0, zz = 0.0, u0raw = 0.0;
    __syncwarp();  // earlier readers of the slab are done
    for (int jj = 0; jj < 2; ++jj) {
        const int j = lane + 32 * jj;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (2 * j < K) w = philox4x32_10(make_uint4((uint32_t)j, lo, hi, pid), k0, k1);
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * j + h;
            double2 v = make_double2(0.0, 0.0);
            if (m < K) {
                const double u1 = u01d_ext(h ? w.z : w.x, 2u * (uint32_t)m, lo, hi, pid, k0, k1);
                const double u2 = u01d(h ? w.w : w.y);
                const double rho = -2.0 * log(u1);
                const double rad = sqrt(rho);
                double sn, cs;
                sincospi(2.0 * u2, &sn, &cs);
                const double sg = UNIF ? 1.0 : P->sigma_d[m];
                v.x = sg * rad * cs;
                v.y = sg * rad * sn;
                const double sk = v.x * v.x + v.y * v.y;
                nrm2 += sk;
                Sraw += (double)((m + 1) * (m + 1)) * sk;
                zz += rho;
                u0raw += v.x;
            }
            sx[m] = v;
        }
    }
    __syncwarp();
    double t = 0.0;
    fold_pair(sx, 3 + lane, 128 - lane, t);
    if (lane < 31)
        fold_pair(sx, 35 + lane, 96 - lane, t);
    else
        row_end(sx, 2, 0.0, 0.0, t);
    const double T = wsum_d(t);
    nrm2 = wsum_d(nrm2);
    Sraw = wsum_d(Sraw);
    zz = wsum_d(zz);
    u0raw = wsum_d(u0raw);
    const double inv = 1.0 / sqrt(nrm2);
    const double inv2 = inv * inv;
    o.S = Sraw * inv2;
    o.T = T * inv2 * inv;
    double delta = P->cS_d * o.S + P->cH_d * o.T;
    if (!UNIF) delta += P->cQ_d * log(zz * inv2);
    delta -= P->logM;
    const uint32_t wa = accept_word(lo, hi, pid, K, k0, k1);
    o.delta = delta;
    o.u = u01d_ext(wa, 4u * (uint32_t)((K + 1) / 2), lo, hi, pid, k0, k1);
    o.lnU = log(o.u);
    o.accept = o.lnU < delta;
    o.near = fabs(o.lnU - delta) < 1e-6;
    o.H2 = (float)((double)P->E0 * o.S);
    o.H3 = (float)((double)P->h3s * o.T);
    o.u0 = (float)((double)P->u0s * u0raw * inv);
    inv_out = inv;
}

// FP64 decision of the guard-band proposals, one warp per queued proposal.
template <bool UNIF>
__global__ void __launch_bounds__(128) k_refine_warp(DevBufs B, uint32_t k0, uint32_t k1) {
    __shared__ double2 s_x[4][kWK];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double2 *sx = s_x[warp];
    const uint32_t n = min(*(volatile uint32_t *)&B.counters[1], B.refine_cap);
    for (uint32_t i = blockIdx.x * 4u + (uint32_t)warp; i < n; i += gridDim.x * 4u) {
        const RefineItem it = B.refine[i];
        const PointConst *P = B.pts + it.point;
        StatBlock *st = B.stats + it.point;
        Out64 o;
        double inv;
        eval64_warp<UNIF>(P, it.idx, k0, k1, sx, lane, o, inv);
        if (lane == 0) {
            atomicAdd(&st->n_refined, 1ull);
            atomicMax(&st->maxd_key, (unsigned long long)fkey((float)o.delta));
            if (o.near) atomicAdd(&st->n_near, 1ull);
            if (o.delta > 0.0) atomicAdd(&st->n_viol, 1ull);
        }
        if (!o.accept) continue;  // the same in every lane
        const int K = P->K;
        unsigned long long slot = 0;
        if (lane == 0) {
            atomicAdd(&st->n_acc, 1ull);
            const float u0 = o.u0, u2 = u0 * u0;
            atomicAdd(&st->hist[hist_bin(u0, __ldg(&P->hist_a), __ldg(&P->hist_b))], 1ull);
            atomicAdd(&st->exc[exc_bin(u0, __ldg(&P->exc_a))], 1ull);
            atomicAdd(&st->q[0], (unsigned long long)__float2ll_rn(u0 * kQ1));
            atomicAdd(&st->q[1], (unsigned long long)__float2ll_rn(u2 * kQ2));
            atomicAdd(&st->q[2], (unsigned long long)__float2ll_rn(u2 * u0 * kQ3));
            atomicAdd(&st->q[3], (unsigned long long)__float2ll_rn(u2 * u2 * kQ4));
            slot = atomicAdd(B.ring_count, 1ull);
            if (slot >= B.ring_cap) atomicAdd(&st->n_dropped, 1ull);
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        unsigned char *rec = slot < B.ring_cap ? B.ring + slot * B.rec_bytes : nullptr;
        float *xh = rec ? reinterpret_cast<float *>(rec + 32) : nullptr;
        for (int m = lane; m < K; m += 32) {
            const double2 v = sx[m];
            const float xf = (float)(v.x * inv), yf = (float)(v.y * inv);
            atomicAdd(&st->spec[m], (unsigned long long)__float2ull_rn(fmaf(xf, xf, yf * yf) * kSpecScale));
            if (xh) {
                xh[m] = xf;
                xh[K + m] = yf;
            }
        }
        if (rec && lane == 0) {
            *reinterpret_cast<unsigned long long *>(rec) = it.idx;
            uint32_t *h = reinterpret_cast<uint32_t *>(rec + 8);
            h[0] = it.point;
            h[1] = 1u | (o.near ? 2u : 0u);
            float *f = reinterpret_cast<float *>(rec + 16);
            f[0] = o.H2;
            f[1] = o.H3;
            f[2] = o.u0;
            f[3] = (float)o.delta;
        }
    }
}

template <bool UNIF, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_sample_warp(const __grid_constant__ DevBufs B, const __grid_constant__ RunArgs A, uint32_t k0, uint32_t k1) {
    constexpr int NW = NT / 32;
    __shared__ WShared<NW> sh;
    __shared__ uint32_t s_hist[kHistBins];
    __shared__ uint32_t s_exc[kExcBins];
    __shared__ unsigned long long s_q[4];
    __shared__ unsigned long long s_spec[kWK];
    __shared__ uint32_t s_cnt[4];  // accepted, envelope violations, dropped, fallbacks
    __shared__ uint32_t s_maxd;
    __shared__ uint32_t s_chunk;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ql = lane & 3;
    wshared_init<NW>(sh, tid, NT);
    for (int e = tid; e < kHistBins; e += NT) s_hist[e] = 0;
    for (int e = tid; e < kWK; e += NT) s_spec[e] = 0ull;
    if (tid < kExcBins) s_exc[tid] = 0;
    if (tid < 4) {
        s_q[tid] = 0ull;
        s_cnt[tid] = 0;
    }
    if (tid == 0) s_maxd = 0;
    float2 *sv = sh.v[warp];
    const uint32_t total = A.chunk_prefix[A.n_points];
    const unsigned long long t0 = A.deadline_ns ? globaltimer_ns() : 0ull;

    for (;;) {
        if (tid == 0) {
            uint32_t c = atomicAdd(&B.counters[0], 1u);
            if (A.deadline_ns && c < total && globaltimer_ns() - t0 > A.deadline_ns) {
                atomicOr(B.status, kStatusDeadline);
                c = total;
            }
            s_chunk = c;
        }
        __syncthreads();
        const uint32_t c = s_chunk;
        if (c >= total) break;
        int p = 0;
        while (p + 1 < A.n_points && A.chunk_prefix[p + 1] <= c) ++p;
        const unsigned long long local = (unsigned long long)(c - A.chunk_prefix[p]) * A.chunk;
        const unsigned long long left = A.count[p] - local;
        const uint32_t n_here = left < A.chunk ? (uint32_t)left : A.chunk;
        const unsigned long long base = A.idx0[p] + local;
        const PointConst *P = B.pts + p;
        for (int e = tid; e < kWK; e += NT) {
            sh.sig[e] = __ldg(&P->sigma[e]);
            sh.act[e] = __ldg(&P->act[e]);
        }
        const Scal sc = load_scal(P);
        __syncthreads();

        float maxd = -INFINITY;
        for (uint32_t i0 = (uint32_t)warp * kWQ; i0 < n_here; i0 += (uint32_t)NW * kWQ) {
            uint32_t lo[kWQ], hi[kWQ], vmask = 0;
#pragma unroll
            for (int q = 0; q < kWQ; ++q) {
                const unsigned long long idx = base + i0 + q;
                lo[q] = (uint32_t)idx;
                hi[q] = (uint32_t)(idx >> 32);
                if (i0 + q < n_here) vmask |= 1u << q;
            }
            const WEval ev = warp_batch<UNIF>(sv, sh.tab, sh.sig, sh.act, sc.K, lo, hi, vmask, sc.pid, k0, k1, lane);
            const uint32_t lq = ql == 0 ? lo[0] : ql == 1 ? lo[1] : ql == 2 ? lo[2] : lo[3];
            const uint32_t hq = ql == 0 ? hi[0] : ql == 1 ? hi[1] : ql == 2 ? hi[2] : hi[3];
            const uint32_t wa = accept_word(lq, hq, sc.pid, sc.K, k0, k1);
            const Fast f = warp_eval<UNIF>(ev, sc, wa);
            const bool valid = lane < kWQ && ((vmask >> lane) & 1u);
            const bool tail = min(ev.wmin, wa) < kTailBucket;
            bool defer = valid && (fabsf(f.d) < f.guard || tail);
            if (valid && !tail) maxd = fmaxf(maxd, f.delta);

            const unsigned md = __ballot_sync(0xffffffffu, defer);
            if (md) {
                const int leader = __ffs(md) - 1;
                uint32_t slot0 = 0;
                if (lane == leader) slot0 = atomicAdd(&B.counters[1], (uint32_t)__popc(md));
                slot0 = __shfl_sync(0xffffffffu, slot0, leader);
                if (defer) {
                    const uint32_t slot = slot0 + __popc(md & ((1u << lane) - 1u));
                    if (slot < B.refine_cap) {
                        RefineItem it;
                        it.idx = ((unsigned long long)hq << 32) | lq;
                        it.point = (uint32_t)p;
                        it.pad = 0;
                        B.refine[slot] = it;
                    } else {  // queue full: decide in FP32 and flag the run
                        atomicOr(B.status, kStatusRefineOverflow);
                        atomicAdd(&s_cnt[3], 1u);
                        defer = false;
                    }
                }
            }
            const bool acc = valid && !defer && f.d < 0.f;
            if (valid && !defer && f.delta > 0.f) atomicAdd(&s_cnt[1], 1u);

            unsigned ma = __ballot_sync(0xffffffffu, acc);
            while (ma) {  // rare: the whole warp writes each accepted record
                const int q = __ffs(ma) - 1;
                ma &= ma - 1;
                const float inv = __shfl_sync(0xffffffffu, f.inv, q);
                const float u0 = __shfl_sync(0xffffffffu, sc.u0s * ev.u0raw * f.inv, q);
                unsigned long long slot = 0;
                if (lane == 0) {
                    slot = atomicAdd(B.ring_count, 1ull);
                    atomicAdd(&s_cnt[0], 1u);
                }
                slot = __shfl_sync(0xffffffffu, slot, 0);
                unsigned char *rec = slot < B.ring_cap ? B.ring + slot * B.rec_bytes : nullptr;
                const float sc2 = (inv * inv) * kSpecScale;
                float *xh = rec ? reinterpret_cast<float *>(rec + 32) : nullptr;
#pragma unroll
                for (int cc = 0; cc < kWK / 32; ++cc) {
                    const int m = lane + 32 * cc;
                    if (m < sc.K) {
                        const float2 v = sv[q * kWS + wpos(m)];
                        atomicAdd(&s_spec[m], (unsigned long long)__float2ull_rn(fmaf(v.x, v.x, v.y * v.y) * sc2));
                        if (xh) {
                            xh[m] = v.x * inv;
                            xh[sc.K + m] = v.y * inv;
                        }
                    }
                }
                if (lane == q) {
                    tally_accepted(u0, sc.ha, sc.hb, sc.ea, s_hist, s_exc, s_q);
                    if (rec) {
                        *reinterpret_cast<unsigned long long *>(rec) = ((unsigned long long)hq << 32) | lq;
                        uint32_t *h = reinterpret_cast<uint32_t *>(rec + 8);
                        h[0] = (uint32_t)p;
                        h[1] = 0u;
                        float *fr = reinterpret_cast<float *>(rec + 16);
                        fr[0] = sc.E0 * f.S;
                        fr[1] = sc.h3s * f.T;
                        fr[2] = u0;
                        fr[3] = f.delta;
                    } else {
                        atomicAdd(&s_cnt[2], 1u);
                    }
                }
            }
            __syncwarp();  // the next batch overwrites the slab
        }
        // chunk done: flush this CTA's partials into the point's StatBlock
        uint32_t key = fkey(maxd);
        key = __reduce_max_sync(0xffffffffu, key);
        if (lane == 0 && maxd > -INFINITY) atomicMax(&s_maxd, key);
        __syncthreads();
        StatBlock *st = B.stats + p;
        for (int e = tid; e < kHistBins; e += NT) {
            if (s_hist[e]) {
                atomicAdd(&st->hist[e], (unsigned long long)s_hist[e]);
                s_hist[e] = 0;
            }
        }
        if (tid < kExcBins && s_exc[tid]) {
            atomicAdd(&st->exc[tid], (unsigned long long)s_exc[tid]);
            s_exc[tid] = 0;
        }
        if (tid < 4 && s_q[tid]) {
            atomicAdd(&st->q[tid], s_q[tid]);
            s_q[tid] = 0ull;
        }
        for (int e = tid; e < kWK; e += NT) {
            if (s_spec[e]) {
                atomicAdd(&st->spec[e], s_spec[e]);
                s_spec[e] = 0ull;
            }
        }
        if (tid == 0) {
            atomicAdd(&st->n_prop, (unsigned long long)n_here);
            if (s_cnt[0]) atomicAdd(&st->n_acc, (unsigned long long)s_cnt[0]);
            if (s_cnt[1]) atomicAdd(&st->n_viol, (unsigned long long)s_cnt[1]);
            if (s_cnt[2]) atomicAdd(&st->n_dropped, (unsigned long long)s_cnt[2]);
            if (s_cnt[3]) atomicAdd(&st->n_fallback, (unsigned long long)s_cnt[3]);
            if (s_maxd) atomicMax(&st->maxd_key, (unsigned long long)s_maxd);
            s_cnt[0] = s_cnt[1] = s_cnt[2] = s_cnt[3] = 0;
            s_maxd = 0;
        }
        __syncthreads();
    }
}

// Replay: per-proposal outputs of listed indices, four per warp (the same
// batch code as the sampler).  out row: [delta, lnU, accept, flags, H2, H3,
// u0, S, xhat(2K)].
constexpr int kReplayWarps = 4;

template <bool UNIF>
__global__ void __launch_bounds__(32 * kReplayWarps) k_replay_warp(const PointConst *P, const unsigned long long *idx,
                                                                   unsigned long long n, uint32_t k0, uint32_t k1,
                                                                   double *out) {
    __shared__ WShared<kReplayWarps> sh;
    __shared__ double2 s_x[kReplayWarps][kWK];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, ql = lane & 3;
    wshared_init<kReplayWarps>(sh, tid, 32 * kReplayWarps);
    for (int e = tid; e < kWK; e += 32 * kReplayWarps) {
        sh.sig[e] = P->sigma[e];
        sh.act[e] = P->act[e];
    }
    __syncthreads();
    const Scal sc = load_scal(P);
    const int K = sc.K;
    const unsigned long long b0 = ((unsigned long long)blockIdx.x * kReplayWarps + warp) * kWQ;
    if (b0 >= n) return;  // whole warps leave together
    float2 *sv = sh.v[warp];
    uint32_t lo[kWQ], hi[kWQ], vmask = 0;
#pragma unroll
    for (int q = 0; q < kWQ; ++q) {
        const unsigned long long i = b0 + q < n ? b0 + q : n - 1;
        const unsigned long long id = idx[i];
        lo[q] = (uint32_t)id;
        hi[q] = (uint32_t)(id >> 32);
        if (b0 + q < n) vmask |= 1u << q;
    }
    const WEval ev = warp_batch<UNIF>(sv, sh.tab, sh.sig, sh.act, K, lo, hi, vmask, sc.pid, k0, k1, lane);
    const uint32_t lq = ql == 0 ? lo[0] : ql == 1 ? lo[1] : ql == 2 ? lo[2] : lo[3];
    const uint32_t hq = ql == 0 ? hi[0] : ql == 1 ? hi[1] : ql == 2 ? hi[2] : hi[3];
    const uint32_t wa = accept_word(lq, hq, sc.pid, K, k0, k1);
    const Fast f = warp_eval<UNIF>(ev, sc, wa);
    const bool valid = lane < kWQ && ((vmask >> lane) & 1u);
    const bool slow = fabsf(f.d) < f.guard || min(ev.wmin, wa) < kTailBucket;
    const size_t rowlen = 8 + 2 * (size_t)K;
    if (valid && !slow) {
        double *row = out + (b0 + lane) * rowlen;
        {
            row[0] = f.delta;
            row[1] = f.lnU;
            row[2] = f.d < 0.f ? 1.0 : 0.0;
            row[3] = 0.0;
            row[4] = sc.E0 * f.S;
            row[5] = sc.h3s * f.T;
            row[6] = sc.u0s * ev.u0raw * f.inv;
            row[7] = f.S;
        }
    }
    // the proposals of the FP64 pass, one after the other on the whole warp
    unsigned ms = __ballot_sync(0xffffffffu, valid && slow);
    while (ms) {
        const int q = __ffs(ms) - 1;
        ms &= ms - 1;
        const unsigned long long id =
            ((unsigned long long)__shfl_sync(0xffffffffu, hq, q) << 32) | __shfl_sync(0xffffffffu, lq, q);
        Out64 o;
        double inv;
        eval64_warp<UNIF>(P, id, k0, k1, s_x[warp], lane, o, inv);
        double *row = out + (b0 + q) * rowlen;
        if (lane == 0) {
            row[0] = o.delta;
            row[1] = o.lnU;
            row[2] = o.accept;
            row[3] = 1.0 + (o.near ? 2.0 : 0.0);
            row[4] = o.H2;
            row[5] = o.H3;
            row[6] = o.u0;
            row[7] = o.S;
        }
        for (int m = lane; m < K; m += 32) {
            const double2 v = s_x[warp][m];
            row[8 + m] = (float)(v.x * inv);
            row[8 + K + m] = (float)(v.y * inv);
        }
    }
    // projected state of the proposals decided in FP32, written by the warp
    const unsigned mf = __ballot_sync(0xffffffffu, valid && !slow);
    for (int q = 0; q < kWQ; ++q) {
        if (!((mf >> q) & 1u)) continue;
        const float inv = __shfl_sync(0xffffffffu, f.inv, q);
        double *row = out + (b0 + q) * rowlen;
        for (int m = lane; m < K; m += 32) {
            const float2 v = sv[q * kWS + wpos(m)];
            row[8 + m] = v.x * inv;
            row[8 + K + m] = v.y * inv;
        }
    }
}

}  // namespace

void triad_kernels_k128(TriadKernels *t) {
    t->main[0][0] = (const void *)k_sample_warp<false, 128, 1>;
    t->main[0][1] = (const void *)k_sample_warp<false, 256, 1>;
    t->main[0][2] = (const void *)k_sample_warp<false, 256, 2>;
    t->main[1][0] = (const void *)k_sample_warp<true, 128, 1>;
    t->main[1][1] = (const void *)k_sample_warp<true, 256, 1>;
    t->main[1][2] = (const void *)k_sample_warp<true, 256, 2>;
    t->sir[0] = t->sir[1] = nullptr;  // SIR runs use the one-thread form (K <= 64)
    t->refine[0] = (const void *)k_refine_warp<false>;
    t->refine[1] = (const void *)k_refine_warp<true>;
    t->replay[0] = (const void *)k_replay_warp<false>;
    t->replay[1] = (const void *)k_replay_warp<true>;
    t->replay_per_block = 32 * kReplayWarps / 32 * kWQ;
    t->xfer_bytes_per_thread = 0;
    t->n_variants = 3;
}

}  // namespace tkdv

// grid_impl.cuh - the grid form of H3 on the 5th-generation tensor cores.
//
// Eq. (2) gives H3 = (1/6) int u^3.  On N equispaced points the rectangle rule
// integrates a trigonometric polynomial of degree below N exactly, whatever
// the offset of the grid, and u^3 has degree 3K < N.  The grid here is
// xi = +-xi_j, xi_j = pi (2j + 1)/N, j = 0..N/2-1 (the N-point grid offset by
// half a step), so that its points come in mirror pairs.  With the cosine and
// sine parts of the raw scaled normals,
//   C_j = sum_k x_k cos(k xi_j),   S_j = sum_k y_k sin(k xi_j),
// u(+-xi_j) is proportional to C_j +- S_j, and a pair contributes
//   (C + S)^3 + (C - S)^3 = 2 C (C^2 + 3 S^2),
// so that
//   H3 = (pi/(3N)) sum_{all N points} u^3,  u = 2 sqrt(E0/2pi) U/|x|,
// needs two contractions of K terms onto N/2 columns instead of one of 2K
// terms onto N: half the multiply-adds of the plain grid contraction.
//
// On the tensor cores, for a tile of 128 proposals:
//   C = Xc Bc,  S' = Xs Bs,  Xc, Xs: 128 x K,  Bc, Bs: K x N/2,
// with Bs holding sqrt(3) sin, so that S' = sqrt(3) S and a pair sums as
// 2 C (C^2 + S'^2) (one packed multiply fewer per two pairs),
// each as three BF16 products with FP32 accumulation in tensor memory:
// X = Xh + Xl, B = Bh + Bl, XB ~ Xh Bh + Xh Bl + Xl Bh (the dropped Xl Bl
// term is 2^-16 relative).  The A tile holds a row per proposal in the
// contraction order [cosine part | sine part], each part KA/2 columns (mode
// k at column k - 1 of its part), BF16 in the 128-byte-swizzled K-major
// layout; B holds the N/2 grid pairs as rows in the same column order.
//
// CTA = NWG warpgroups of 128 threads.  B (hi and lo) is loaded once per CTA
// and shared; every warpgroup owns one A tile (hi and lo), one pair of TMEM
// accumulators (C and S, N/2 columns each) and one mbarrier, and runs its own
// persistent loop over chunks of proposal indices:
//   1. each thread makes its proposal (Philox, Box-Muller, sigma scaling: the
//      values of the triad form with the signs of the components flipped,
//      the two modes of a Philox block in packed FP32 pairs) and writes its
//      row of Xh and Xl (the basis is negated to match);
//   2. after a warpgroup barrier one thread issues the 2 x 3 x K/16
//      tcgen05.mma (M = 128, N = N/2, K = 16) and commits them to the
//      warpgroup's mbarrier;
//   3. every thread waits (bounded) on the mbarrier, reads its own TMEM lane
//      (its proposal's C_j and S'_j) and sums 2 C (C^2 + S'^2);
//   4. the decision is that of the triad form; an accepted draw's index,
//      T and log f/(Mg) go to its warp's slab in global memory, and at the
//      end of the chunk the warp makes the outputs of its slab 32 draws at a
//      time (the draw again with the accurate radius for the record's state,
//      u(0) and spectrum), so that the hot loop never runs a divergent redraw.
// While one warpgroup waits for its products, the others produce.
#pragma once

#include <cuda_bf16.h>

#include "sampler_impl.cuh"

namespace tkdv {

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Barrier of one warpgroup (named barrier 1 + g, 128 threads).
__device__ __forceinline__ void wg_sync(int g) {
    asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after ~2 s of %globaltimer and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t addr, uint32_t parity) {
    if (mbar_try_wait(addr, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(addr, parity)) return true;
        if ((it & 255u) == 255u && globaltimer_ns() - t0 > 2000000000ull) return false;
    }
}

__device__ __forceinline__ void tmem_alloc(uint32_t smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_dst), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (tmem) (+)= A (smem desc) * B (smem desc), BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major, 128B-swizzled operand tile
// whose 8-row groups are 1024 bytes apart (tile base 1024-byte aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024u >> 4) << 32;          // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, col) of a K-major SW128 tile with `rows` rows:
// 64 BF16 columns per 128-byte swizzle atom, atoms `rows * 128` bytes apart.
__host__ __device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t col, uint32_t rows) {
    const uint32_t atom = col >> 6, c = col & 63u, chunk = c >> 3;
    return atom * rows * 128u + (row >> 3) * 1024u + (row & 7u) * 128u + ((chunk ^ (row & 7u)) << 4) + (c & 7u) * 2u;
}

template <int KMAX>
struct GridShape {
    static constexpr int KA = (2 * KMAX + 63) / 64 * 64;  // contraction columns: [cosine part | sine part]
    static constexpr int PART = KA / 2;                   // columns of each part (mode k at column k - 1)
    static constexpr int KSTEPS = (KMAX + 15) / 16;       // 16-column MMA steps per part
    static constexpr int A_TILE = 128 * KA * 2;           // bytes of one BF16 tile (hi or lo)
};

// The two Box-Muller pairs of one Philox block (radius words w.x, w.z, angle
// words w.y, w.w; scales s = (s_m, s_m+1)), with the multiplications and
// additions of the two modes as packed pairs: rho as rho_fast gives it,
// rr = rsqrt_approx(rho), and (x, y) = s sqrt(rho) (cos, sin) of the reduced
// angle 2 pi (u2 - 1/2).  These are the values of box_muller_f32<false> with
// the signs of x and y flipped; the grid basis carries the same flip (its
// values are negated), so that the products C and S' are unchanged.
__device__ __forceinline__ void box_muller2(const uint4 w, f32x2_t s, f32x2_t &rho, f32x2_t &rr, f32x2_t &x,
                                            f32x2_t &y) {
    constexpr float kLn4 = 1.38629436111989061883f, k2Pi = 6.28318530717958647692f;
    const f32x2_t f1 = pk2(one_m(w.x), one_m(w.z));
    float u0, u1;
    upk2(add2(f1, pk2(-0x1.fffffep-1f, -0x1.fffffep-1f)), u0, u1);  // u01f of w.x, w.z
    float l0, l1;
    upk2(mul2(pk2(lg2_approx(u0), lg2_approx(u1)), pk2(-kLn4, -kLn4)), l0, l1);
    const float r0 = fmaxf(l0, 0x1p-25f), r1 = fmaxf(l1, 0x1p-25f);  // rho_fast
    rho = pk2(r0, r1);
    rr = pk2(rsqrt_approx(r0), rsqrt_approx(r1));
    const f32x2_t a = mul2(mul2(s, rho), rr);
    const f32x2_t f2 = pk2(one_m(w.y), one_m(w.w));
    float t0, t1;  // angle_f of w.y, w.w
    upk2(fma2(pk2(k2Pi, k2Pi), add2(f2, pk2(-1.5f, -1.5f)), pk2(k2Pi * 0x1p-24f, k2Pi * 0x1p-24f)), t0, t1);
    float sn0, cs0, sn1, cs1;
    sincos_approx(t0, sn0, cs0);
    sincos_approx(t1, sn1, cs1);
    x = mul2(a, pk2(cs0, cs1));
    y = mul2(a, pk2(sn0, sn1));
}

// Pack 8 floats into BF16 hi and lo halves (x = hi + lo + O(2^-16 x)); the
// residuals x - hi (exact in FP32) of a pair by one packed subtraction.
__device__ __forceinline__ void split8(const float *v, uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        const uint32_t hb = *reinterpret_cast<const uint32_t *>(&hh);
        f32x2_t rr;
        asm("sub.rn.f32x2 %0, %1, %2;"
            : "=l"(rr)
            : "l"(pk2(v[2 * q], v[2 * q + 1])), "l"(pk2(__uint_as_float(hb << 16), __uint_as_float(hb & 0xFFFF0000u))));
        float r0, r1;
        upk2(rr, r0, r1);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(r0, r1);
        h[q] = hb;
        l[q] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Per-warpgroup shared state: the point being sampled and the statistics
// partials of the current chunk (flushed to the point's StatBlock at its end).
template <int KMAX>
struct GridWG {
    uint32_t hist[kHistBins];
    uint32_t exc[kExcBins];
    unsigned long long q[4];
    unsigned long long spec[KMAX];
    uint32_t cnt[4];  // accepted, envelope violations, dropped, fallbacks
    uint32_t maxd;
    uint32_t chunk;
    uint32_t abort;
    float sig[KMAX], act[KMAX];
    // mode_consts of the point by pairs of modes (2j, 2j + 1) = Philox block
    // j: (s, s', s^2, s'^2) and ((m+1)^2 s^2, (m+2)^2 s'^2, act, act')
    float4 mp[KMAX / 2][2];
};

// One row of a tile between its draw and its decision.
struct GridRow {
    unsigned long long idx;
    float nrm2, Sraw, zz, esum;
    bool valid;
    bool tail;  // a radius word in the lowest bucket of the uniform map
};

// ---- the persistent grid-form sampler --------------------------------------
// Dynamic shared memory (1024-byte aligned): [B hi | B lo | NWG x (A hi | A lo)].
// (A second A tile per warpgroup, drawing tile t+1 before waiting for the
// products of tile t, measured 8 % slower at three warpgroups than one tile
// with the product-free decision terms made before the wait.)
template <int KMAX, bool UNIF, int NWG, int UNR>
__global__ void __launch_bounds__(128 * NWG, 1)
    k_sample_grid(const __grid_constant__ DevBufs B, const __grid_constant__ RunArgs A, uint32_t k0, uint32_t k1,
                  const unsigned char *__restrict__ bimg, int gridN) {
    using GS = GridShape<KMAX>;
    constexpr int KA = GS::KA, PART = GS::PART, KSTEPS = GS::KSTEPS, ATILE = GS::A_TILE;
    extern __shared__ unsigned char dyn_smem[];
    __shared__ GridWG<KMAX> s_wg[NWG];
    __shared__ __align__(8) unsigned long long s_mbar[NWG];  // the tile's products are in TMEM (MMA commit)
    __shared__ uint32_t s_tmem;
    __shared__ uint32_t s_abort;  // any warpgroup's device wait gave up: every warpgroup stops

    const int g = threadIdx.x >> 7, t = threadIdx.x & 127, lane = t & 31;
    GridWG<KMAX> &W = s_wg[g];
    const int half = gridN >> 1;                      // grid pairs = columns of C and of S
    const uint32_t btile = (uint32_t)half * KA * 2;  // bytes of one B tile (hi or lo)
    const uint32_t base = (smem_u32(dyn_smem) + 1023u) & ~1023u;
    unsigned char *gbase = dyn_smem + (base - smem_u32(dyn_smem));
    const uint32_t b_hi = base, b_lo = base + btile;
    const uint32_t a_hi = base + 2 * btile + (uint32_t)g * 2u * ATILE, a_lo = a_hi + ATILE;
    unsigned char *ga_hi = gbase + 2 * btile + (uint32_t)g * 2u * ATILE;
    unsigned char *ga_lo = ga_hi + ATILE;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(bimg);
        uint4 *dst = reinterpret_cast<uint4 *>(gbase);
        for (uint32_t i = threadIdx.x; i < 2 * btile / 16; i += 128 * NWG) dst[i] = __ldg(src + i);
    }
    for (int e = t; e < kHistBins; e += 128) W.hist[e] = 0;
    for (int e = t; e < KMAX; e += 128) W.spec[e] = 0ull;
    if (t < kExcBins) W.exc[t] = 0;
    if (t < 4) {
        W.q[t] = 0ull;
        W.cnt[t] = 0;
    }
    if (t == 0) {
        W.maxd = 0;
        W.abort = 0;
    }
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int w = 0; w < NWG; ++w) mbar_init(smem_u32(&s_mbar[w]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // TMEM: per warpgroup C (N/2 columns) and S (N/2 columns)
    uint32_t tcols = 32;
    while (tcols < (uint32_t)(NWG * gridN)) tcols <<= 1;
    if (threadIdx.x < 32) {
        tmem_alloc(smem_u32(&s_tmem), tcols);
        tmem_relinquish();
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_c = s_tmem + (uint32_t)(g * gridN);
    const uint32_t tmem_s = tmem_c + (uint32_t)half;
    const uint32_t lane_off = ((uint32_t)(t >> 5) * 32u) << 16;
    const uint32_t idesc = idesc_bf16_f32(128, half);
    const uint32_t mbar = smem_u32(&s_mbar[g]);
    uint32_t phase = 0;
    bool pending = false;  // an MMA commit of this warpgroup not yet waited for
    // this warp's slab: room for the accepted draws of one chunk (at most
    // chunk / 4 proposals per warp)
    AcceptItem *slab = B.accs + ((size_t)(blockIdx.x * NWG + g) * 4 + (size_t)(t >> 5)) * B.acc_slab;
    const float tscale = 8.f / (3.f * (float)gridN);  // T = (4/(3N)) sum U^3/|x|^3, sum U^3 = 2 sum C (C^2 + 3 S^2)

    const uint32_t total = A.chunk_prefix[A.n_points];
    const unsigned long long t0 = A.deadline_ns ? globaltimer_ns() : 0ull;
    for (;;) {
        if (t == 0) {
            uint32_t c = atomicAdd(&B.counters[0], 1u);
            if (A.deadline_ns && c < total && globaltimer_ns() - t0 > A.deadline_ns) {
                atomicOr(B.status, kStatusDeadline);
                c = total;
            }
            if (*(volatile uint32_t *)&s_abort) c = total;
            W.chunk = c;
        }
        wg_sync(g);
        const uint32_t c = W.chunk;
        if (c >= total) break;
        int p = 0;
        while (p + 1 < A.n_points && A.chunk_prefix[p + 1] <= c) ++p;
        const unsigned long long local = (unsigned long long)(c - A.chunk_prefix[p]) * A.chunk;
        const unsigned long long left = A.count[p] - local;
        const uint32_t n_here = left < A.chunk ? (uint32_t)left : A.chunk;
        const unsigned long long cbase = A.idx0[p] + local;
        const PointConst *P = B.pts + p;
        if (t < KMAX) {
            W.sig[t] = __ldg(&P->sigma[t]);
            W.act[t] = __ldg(&P->act[t]);
        }
        if (t < KMAX / 2) {
            const float4 a = mode_consts<UNIF>(__ldg(&P->sigma[2 * t]), __ldg(&P->act[2 * t]), 2 * t);
            const float4 b = mode_consts<UNIF>(__ldg(&P->sigma[2 * t + 1]), __ldg(&P->act[2 * t + 1]), 2 * t + 1);
            W.mp[t][0] = make_float4(a.x, b.x, a.y, b.y);
            W.mp[t][1] = make_float4(a.z, b.z, a.w, b.w);
        }
        const Scal sc = load_scal(P);
        wg_sync(g);
        float maxd = -INFINITY;
        uint32_t nacc = 0;  // accepted draws of this warp in this chunk (the same in every lane)

        const uint32_t n_tiles = (n_here + 127u) / 128u;
        // ---- 3./4. the products and the decision of one row
        auto consume = [&](const GridRow &r) {
            const unsigned long long idx = r.idx;
            const uint32_t lo = (uint32_t)idx, hi = (uint32_t)(idx >> 32);
            const bool valid = r.valid, tail_r = r.tail;
            const float nrm2 = r.nrm2, Sraw = r.Sraw, zz = r.zz, esum = r.esum;
            // the terms of the decision that do not need the products, made
            // while the tensor cores work: 1/|x|^2, S, ln Q, the accept word
            const float inv2 = rcp_rn(nrm2);
            const float inv = rsqrt_approx(nrm2);
            const float S = Sraw * inv2;
            const float tS = sc.cS * S;
            const float tQ = UNIF ? 0.f : sc.cQ * logf(zz * inv2);
            const uint32_t wa = PhiloxRow(lo, hi, sc.pid, A.rk.k).block((uint32_t)((sc.K + 1) / 2)).x;
            const float lnU = -0.5f * rho_fast(wa);
            // ---- 3. wait for the products, sum 2 C (C^2 + 3 S^2) of this row
            float cube = 0.f;
            bool ok = false;
            if (pending && !W.abort) {  // after a timeout of this warpgroup no thread waits again
                ok = mbar_wait_bounded(mbar, phase);
                if (ok) {
                    phase ^= 1u;
                    pending = false;
                    tc_fence_after();
                    // 16 columns of C and of S per wait (32 per wait spilled
                    // and measured slower at every launch shape: 5.57e9 against
                    // 5.81e9 proposals/s at 64 modes, 12.04e9 against 12.17e9
                    // with three warpgroups at 32)
                    f32x2_t acc[2] = {0ull, 0ull};
                    auto cube_sum = [&](const float *cv, const float *sv, int n) {
#pragma unroll
                        for (int e = 0; e < n; e += 2) {
                            const f32x2_t C2 = pk2(cv[e], cv[e + 1]), S2 = pk2(sv[e], sv[e + 1]);
                            const f32x2_t q = fma2(S2, S2, mul2(C2, C2));  // C^2 + 3 S^2
                            acc[(e >> 1) & 1] = fma2(C2, q, acc[(e >> 1) & 1]);
                        }
                    };
                    int cb = 0;
                    for (; cb < half; cb += 16) {
                        float cv[16], sv[16];
                        tmem_ld16(tmem_c + lane_off + (uint32_t)cb, cv);
                        tmem_ld16(tmem_s + lane_off + (uint32_t)cb, sv);
                        tmem_wait_ld();
                        cube_sum(cv, sv, 16);
                    }
                    float a0, a1, b0, b1;
                    upk2(acc[0], a0, a1);
                    upk2(acc[1], b0, b1);
                    cube = (a0 + a1) + (b0 + b1);
                    tc_fence_before();
                } else {
                    atomicOr(B.status, kStatusMbarTimeout);
                    W.abort = 1;
                    s_abort = 1;
                }
            }
            // ---- 4. decision
            const bool usable = valid && ok;
            const float T = cube * tscale * (inv2 * inv);
            const float tH = sc.cH * T;
            const float delta = ((tS + tH) + tQ) - sc.logM;
            const float d = lnU - delta;
            const float guard = fmaf(
                sc.ge * esum, inv,
                fmaf(sc.gq, inv2, sc.ga + sc.gr * (fabsf(tS) + fabsf(tQ) + fabsf(tH) + fabsf(lnU) + fabsf(sc.logM)) + sc.gh));
            // a radius or accept word in the lowest bucket: FP64 pass (refined tail)
            const bool tail = tail_r || wa < kTailBucket;
            bool defer = usable && (fabsf(d) < guard || tail);
            if (usable && !tail) maxd = fmaxf(maxd, delta);
            const unsigned long long li = idx - A.idx0[p];
            if (A.trace && p == 0 && usable && li < A.trace_n) {
                // a draw with a refined tail word is decided in FP64 only: NaN here
                A.trace[2 * li] = tail ? __int_as_float(0x7fc00000) : delta;
                A.trace[2 * li + 1] = tail ? __int_as_float(0x7fc00000) : T;
            }
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
                        it.idx = idx;
                        it.point = (uint32_t)p;
                        it.pad = 0;
                        B.refine[slot] = it;
                    } else {
                        atomicOr(B.status, kStatusRefineOverflow);
                        atomicAdd(&W.cnt[3], 1u);
                        defer = false;
                    }
                }
            }
            const bool acc = usable && !defer && d < 0.f;
            if (usable && !defer && delta > 0.f) atomicAdd(&W.cnt[1], 1u);
            // accepted draws: (index, T, log f/(Mg)) to this warp's slab
            const unsigned ma = __ballot_sync(0xffffffffu, acc);
            if (ma) {
                if (acc) {
                    AcceptItem it;
                    it.idx = idx;
                    it.T = T;
                    it.delta = delta;
                    slab[nacc + __popc(ma & ((1u << lane) - 1u))] = it;
                }
                nacc += (uint32_t)__popc(ma);
            }
        };
        for (uint32_t trip = 0; trip < n_tiles; ++trip) {
            GridRow cur;
            {  // ---- 1. this thread's row of the tile
                const uint32_t i = trip * 128u + (uint32_t)t;
                const unsigned long long idx = cbase + i;
                const uint32_t lo = (uint32_t)idx, hi = (uint32_t)(idx >> 32);
                // ---- 1. the row of X: eight modes (four Philox blocks) at a time,
                // cosine values to part 0 and sine values to part 1 of the row
                // the mode sums over even and odd modes in packed pairs
                f32x2_t nrm2p = 0ull, Srawp = 0ull, zzp = 0ull, esump = 0ull;
                uint32_t wmin = 0xFFFFFFFFu;
                const PhiloxRow prow(lo, hi, sc.pid, A.rk.k);
#pragma unroll(UNR)
                for (int c8 = 0; c8 < KMAX / 8; ++c8) {
                    float vx[8], vy[8];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = 4 * c8 + jj;
                        const uint4 w = prow.block((uint32_t)j);
                        const float4 c0 = W.mp[j][0], c1 = W.mp[j][1];
                        const f32x2_t s2 = pk2(c0.x, c0.y);
                        f32x2_t rho2, rr2, x2, y2;
                        box_muller2(w, s2, rho2, rr2, x2, y2);
                        upk2(x2, vx[2 * jj], vx[2 * jj + 1]);
                        upk2(y2, vy[2 * jj], vy[2 * jj + 1]);
                        wmin = min(wmin, min(w.x, w.z));
                        esump = fma2(s2, rr2, esump);
                        nrm2p = fma2(pk2(c0.z, c0.w), rho2, nrm2p);
                        Srawp = fma2(pk2(c1.x, c1.y), rho2, Srawp);
                        zzp = fma2(pk2(c1.z, c1.w), rho2, zzp);  // the active modes' squared radii
                    }
                    uint4 hx, lx, hy, ly;
                    split8(vx, hx, lx);
                    split8(vy, hy, ly);
                    const uint32_t ox = sw128_offset((uint32_t)t, (uint32_t)(8 * c8), 128u);
                    const uint32_t oy = sw128_offset((uint32_t)t, (uint32_t)(PART + 8 * c8), 128u);
                    *reinterpret_cast<uint4 *>(ga_hi + ox) = hx;
                    *reinterpret_cast<uint4 *>(ga_lo + ox) = lx;
                    *reinterpret_cast<uint4 *>(ga_hi + oy) = hy;
                    *reinterpret_cast<uint4 *>(ga_lo + oy) = ly;
                }
                float e0, e1;
                cur.idx = idx;
                cur.valid = i < n_here;
                upk2(nrm2p, e0, e1);
                cur.nrm2 = e0 + e1;
                upk2(Srawp, e0, e1);
                cur.Sraw = e0 + e1;
                upk2(zzp, e0, e1);
                cur.zz = e0 + e1;
                upk2(esump, e0, e1);
                cur.esum = e0 + e1;
                cur.tail = wmin < kTailBucket;
            }
            {  // ---- 2. after the warpgroup barrier one thread issues the contraction of the tile
                fence_async_smem();
                wg_sync(g);
                const bool run_mma = W.abort == 0;
                if (run_mma) {
                    if (t == 0) {
                        tc_fence_after();
#pragma unroll
                        for (int part = 0; part < 2; ++part) {
                            const uint32_t dt = part ? tmem_s : tmem_c;
#pragma unroll
                            for (int ks = 0; ks < KSTEPS; ++ks) {
                                const uint32_t kcol = (uint32_t)(part * PART + 16 * ks);
                                const uint32_t koff = (kcol & 63u) * 2u;  // bytes into the swizzle atom
                                const uint32_t aat = (kcol >> 6) * 128u * 128u;
                                const uint32_t bat = (kcol >> 6) * (uint32_t)half * 128u;
                                const uint64_t dah = sw128_desc(a_hi + aat + koff), dal = sw128_desc(a_lo + aat + koff);
                                const uint64_t dbh = sw128_desc(b_hi + bat + koff), dbl = sw128_desc(b_lo + bat + koff);
                                umma_bf16(dt, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                                umma_bf16(dt, dah, dbl, idesc, 1u);
                                umma_bf16(dt, dal, dbh, idesc, 1u);
                            }
                        }
                        umma_commit(mbar);
                    }
                    pending = true;
                }
            }
            consume(cur);
        }

        // ---- outputs of this warp's accepted draws of the chunk, 32 at a time:
        // the draw again with the accurate radius (rho_acc) for the state,
        // u(0), H2 and the spectrum; H3 from the grid contraction
        __syncwarp();  // the slab entries other lanes wrote
        if (lane == 0 && nacc) atomicAdd(&W.cnt[0], nacc);
        for (uint32_t b0 = 0; b0 < nacc; b0 += 32) {
            const bool has = b0 + (uint32_t)lane < nacc;
            const unsigned mh = __ballot_sync(0xffffffffu, has);
            unsigned long long slot0 = 0;
            if (lane == 0) slot0 = atomicAdd(B.ring_count, (unsigned long long)__popc(mh));
            slot0 = __shfl_sync(0xffffffffu, slot0, 0);
            unsigned long long qv[4] = {0ull, 0ull, 0ull, 0ull};  // u0 power sums, summed over the warp first
            if (has) {
                const AcceptItem it = slab[b0 + lane];
                const uint32_t ilo = (uint32_t)it.idx, ihi = (uint32_t)(it.idx >> 32);
                const DrawSums dr = acc_draw_sums<KMAX, UNIF>(W.sig, W.act, ilo, ihi, sc.pid, k0, k1);
                const float inv2 = rcp_rn(dr.nrm2);
                const float inv = rsqrt_approx(dr.nrm2);
                const float u0 = sc.u0s * dr.u0raw * inv;
                atomicAdd(&W.hist[hist_bin(u0, sc.ha, sc.hb)], 1u);
                atomicAdd(&W.exc[exc_bin(u0, sc.ea)], 1u);
                const float u2 = u0 * u0;
                qv[0] = (unsigned long long)__float2ll_rn(u0 * kQ1);
                qv[1] = (unsigned long long)__float2ll_rn(u2 * kQ2);
                qv[2] = (unsigned long long)__float2ll_rn(u2 * u0 * kQ3);
                qv[3] = (unsigned long long)__float2ll_rn(u2 * u2 * kQ4);
                const unsigned long long slot = slot0 + __popc(mh & ((1u << lane) - 1u));
                unsigned char *rec = nullptr;
                if (slot < B.ring_cap) {
                    rec = B.ring + slot * B.rec_bytes;
                    write_header(rec, it.idx, (uint32_t)p, 0u, sc.E0 * (dr.Sraw * inv2), sc.h3s * it.T, u0, it.delta);
                } else {
                    atomicAdd(&W.cnt[2], 1u);
                }
                acc_draw_emit<KMAX, UNIF>(W.sig, W.act, ilo, ihi, sc.pid, k0, k1, inv, inv2, sc.K,
                                          rec ? reinterpret_cast<float *>(rec + 32) : nullptr, W.spec,
                                          lane % ((KMAX + 1) / 2));
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {  // fixed-point sums: exact in any order
                unsigned long long v = qv[e];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0 && v) atomicAdd(&W.q[e], v);
            }
        }

        // chunk done: flush this warpgroup's partials into the point's StatBlock
        uint32_t key = fkey(maxd);
        key = __reduce_max_sync(0xffffffffu, key);
        if (lane == 0 && maxd > -INFINITY) atomicMax(&W.maxd, key);
        wg_sync(g);
        StatBlock *st = B.stats + p;
        for (int e = t; e < kHistBins; e += 128) {
            if (W.hist[e]) {
                atomicAdd(&st->hist[e], (unsigned long long)W.hist[e]);
                W.hist[e] = 0;
            }
        }
        if (t < kExcBins && W.exc[t]) {
            atomicAdd(&st->exc[t], (unsigned long long)W.exc[t]);
            W.exc[t] = 0;
        }
        if (t < 4 && W.q[t]) {
            atomicAdd(&st->q[t], W.q[t]);
            W.q[t] = 0ull;
        }
        for (int e = t; e < KMAX; e += 128) {
            if (W.spec[e]) {
                atomicAdd(&st->spec[e], W.spec[e]);
                W.spec[e] = 0ull;
            }
        }
        if (t == 0) {
            atomicAdd(&st->n_prop, (unsigned long long)n_here);
            if (W.cnt[0]) atomicAdd(&st->n_acc, (unsigned long long)W.cnt[0]);
            if (W.cnt[1]) atomicAdd(&st->n_viol, (unsigned long long)W.cnt[1]);
            if (W.cnt[2]) atomicAdd(&st->n_dropped, (unsigned long long)W.cnt[2]);
            if (W.cnt[3]) atomicAdd(&st->n_fallback, (unsigned long long)W.cnt[3]);
            if (W.maxd) atomicMax(&st->maxd_key, (unsigned long long)W.maxd);
            W.cnt[0] = W.cnt[1] = W.cnt[2] = W.cnt[3] = 0;
            W.maxd = 0;
        }
        wg_sync(g);
    }
    // a commit that timed out may still land: wait for it (bounded) before
    // the accumulator columns are released
    if (pending) (void)mbar_wait_bounded(mbar, phase);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(s_tmem, tcols);
}

template <int KMAX>
void fill_grid_kernels_nwg(GridKernels *t, int variant, const void *g0, const void *g1, int nwg) {
    t->main[variant][0] = g0;
    t->main[variant][1] = g1;
    t->nwg[variant] = nwg;
    if (variant + 1 > t->n_variants) t->n_variants = variant + 1;
    t->kmax = KMAX;
    t->ka = GridShape<KMAX>::KA;
}

// Variant v of the KMAX grid kernels with NWG warpgroups per CTA; the
// producer loop over groups of eight modes unrolled UNR times (measured at 32
// modes: 4, the whole loop, for four and three warpgroups, 11.34e9 against
// 11.00e9 proposals/s with 2 at four; 2 for two warpgroups, at 32 and at 64
// modes, where 4 measured 2 % and 5 % slower).
template <int KMAX, int NWG, int UNR = (NWG >= 3 ? 4 : 2)>
void fill_grid_variant(GridKernels *t, int variant) {
    fill_grid_kernels_nwg<KMAX>(t, variant, (const void *)k_sample_grid<KMAX, false, NWG, UNR>,
                                (const void *)k_sample_grid<KMAX, true, NWG, UNR>, NWG);
}

}  // namespace tkdv

// grid_impl.cuh - the grid form of H3 on the 5th-generation tensor cores.
//
// Eq. (2) gives H3 = (1/6) int u^3; on the N-point grid xi_j = -pi + 2 pi j/N
// with N > 3K the rectangle rule is exact, so for a tile of 128 proposals
//   U = X B,   X: 128 x 2K (raw scaled normals, [cos | sin] halves),
//              B: 2K x N  (B[k][j] = cos(k xi_j), B[K+k][j] = sin(k xi_j)),
//   H3 = (pi/(3N)) sum_j (2 sqrt(E0/2pi) U_j / |x|)^3.
// The contraction runs as three BF16 products with FP32 accumulation in
// tensor memory: X = Xh + Xl, B = Bh + Bl, U ~ Xh Bh + Xh Bl + Xl Bh
// (the dropped Xl Bl term is 2^-16 relative).
//
// CTA = one warpgroup of 128 threads; each tile has 128 rows (proposals):
//   1. every thread makes its proposal (Philox, Box-Muller, sigma scaling as
//      in the triad form) and writes its row of Xh and Xl (BF16) into a
//      128B-swizzled K-major shared-memory tile.  The contraction index is
//      ordered so that each 16-byte chunk holds (x_k, y_k) of four
//      consecutive modes: column 8c + 2e + s is mode 4c + e + 1, cosine
//      (s = 0) or sine (s = 1) half;
//   2. after a CTA barrier one thread issues 3 * (KA/16) tcgen05.mma
//      (M = 128, N = grid points, K = 16 each) into one of the CTA's TMEM
//      accumulators and commits them to that accumulator's mbarrier;
//   3. every thread waits (bounded) on the mbarrier, reads its own TMEM lane
//      with tcgen05.ld (32 columns at a time), and sums U_j^3;
//   4. the decision, statistics and records are those of the triad form.
// B (hi and lo) is built on the host once per handle, already in the
// swizzled layout, and copied into shared memory when a CTA starts.
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

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
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
    static constexpr int KA = (2 * KMAX + 63) / 64 * 64;  // contraction length, whole swizzle atoms
    static constexpr int A_TILE = 128 * KA * 2;           // bytes of one BF16 tile (hi or lo)
};

// Pack 8 floats into BF16 hi and lo halves (x = hi + lo + O(2^-16 x)).
__device__ __forceinline__ void split8(const float *v, uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        const float r0 = v[2 * q] - __low2float(hh), r1 = v[2 * q + 1] - __high2float(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(r0, r1);
        h[q] = *reinterpret_cast<const uint32_t *>(&hh);
        l[q] = *reinterpret_cast<const uint32_t *>(&ll);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// ---- the persistent grid-form sampler --------------------------------------
// One warpgroup (128 threads) per CTA.  With NBUF = 2 the BF16 tiles and the
// TMEM accumulators are double-buffered: after the MMAs of tile t are issued
// the threads finish tile t-1 (wait, TMEM read, decision) and then make tile
// t+1, so the tensor-core work of one tile overlaps the generation of the
// next within the CTA.  With NBUF = 1 a CTA waits for its own MMAs and the
// overlap comes from the other CTAs on the SM: for K <= 32 that layout holds
// three CTAs per SM (168 registers, 512 TMEM columns / 128) where the
// double-buffered one held two, and measured 24 % more proposals per second.
// Dynamic shared memory: [B hi | B lo | NBUF x (A hi | A lo)], 1024-byte
// aligned.
struct GridPending {
    unsigned long long idx;
    float nrm2, Sraw, zz, esum;
    bool valid;
    bool tail;  // a radius word in the lowest bucket of the uniform map
};

template <int KMAX, bool UNIF, int NBUF>
__global__ void __launch_bounds__(128, NBUF == 2 ? 2 : (KMAX <= 32 ? 3 : 1))
    k_sample_grid(const __grid_constant__ DevBufs B, const __grid_constant__ RunArgs A, uint32_t k0, uint32_t k1,
                  const unsigned char *__restrict__ bimg, int gridN) {
    constexpr int NT = 128;
    constexpr int KA = GridShape<KMAX>::KA;
    constexpr int ATILE = GridShape<KMAX>::A_TILE;
    extern __shared__ unsigned char dyn_smem[];
    __shared__ uint32_t s_hist[kHistBins];
    __shared__ uint32_t s_exc[kExcBins];
    __shared__ unsigned long long s_q[4];
    __shared__ unsigned long long s_spec[KMAX];
    __shared__ uint32_t s_cnt[4];
    __shared__ uint32_t s_maxd;
    __shared__ uint32_t s_chunk;
    __shared__ uint32_t s_abort;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) unsigned long long s_mbar[NBUF];
    __shared__ float s_sig[KMAX], s_act[KMAX];

    const int tid = threadIdx.x, lane = tid & 31, row = tid;
    const uint32_t btile = (uint32_t)gridN * KA * 2;  // bytes of one B tile
    const uint32_t base = (smem_u32(dyn_smem) + 1023u) & ~1023u;
    unsigned char *gbase = dyn_smem + (base - smem_u32(dyn_smem));
    const uint32_t b_hi = base, b_lo = base + btile;
    const uint32_t a0 = base + 2 * btile;  // A buffer b: hi at a0 + 2 b ATILE, lo at + ATILE

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(bimg);
        uint4 *dst = reinterpret_cast<uint4 *>(gbase);
        for (uint32_t i = tid; i < 2 * btile / 16; i += NT) dst[i] = __ldg(src + i);
        uint4 *az = reinterpret_cast<uint4 *>(gbase + 2 * btile);
        for (uint32_t i = tid; i < (uint32_t)NBUF * 2 * ATILE / 16; i += NT) az[i] = make_uint4(0, 0, 0, 0);
    }
    for (int e = tid; e < kHistBins; e += NT) s_hist[e] = 0;
    for (int e = tid; e < KMAX; e += NT) s_spec[e] = 0ull;
    if (tid < kExcBins) s_exc[tid] = 0;
    if (tid < 4) {
        s_q[tid] = 0ull;
        s_cnt[tid] = 0;
    }
    if (tid == 0) {
        s_maxd = 0;
        s_abort = 0;
        for (int b = 0; b < NBUF; ++b) mbar_init(smem_u32(&s_mbar[b]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t tcols = 32;
    while (tcols < (uint32_t)gridN) tcols <<= 1;
    if (tid < 32) {
        tmem_alloc(smem_u32(&s_tmem), tcols * NBUF);
        tmem_relinquish();
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem0 = s_tmem;
    const uint32_t lane_off = ((uint32_t)(tid >> 5) * 32u) << 16;
    const uint32_t idesc = idesc_bf16_f32(128, gridN);
    uint32_t phase[NBUF];
#pragma unroll
    for (int b = 0; b < NBUF; ++b) phase[b] = 0;
    bool waits_pending[NBUF];
#pragma unroll
    for (int b = 0; b < NBUF; ++b) waits_pending[b] = false;
    const float tscale = 4.f / (3.f * (float)gridN);  // T = (4/(3N)) sum U^3 / |x|^3

    const uint32_t total = A.chunk_prefix[A.n_points];
    const unsigned long long t0 = A.deadline_ns ? globaltimer_ns() : 0ull;
    for (;;) {
        if (tid == 0) {
            uint32_t c = atomicAdd(&B.counters[0], 1u);
            if (A.deadline_ns && c < total && globaltimer_ns() - t0 > A.deadline_ns) {
                atomicOr(B.status, kStatusDeadline);
                c = total;
            }
            if (s_abort) c = total;
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
        const unsigned long long cbase = A.idx0[p] + local;
        const PointConst *P = B.pts + p;
        if (tid < KMAX) {
            s_sig[tid] = __ldg(&P->sigma[tid]);
            s_act[tid] = __ldg(&P->act[tid]);
        }
        const Scal sc = load_scal(P);
        __syncthreads();
        float maxd = -INFINITY;

        // Finish one tile: wait for its MMAs, read U from TMEM, decide.
        auto consume = [&](const GridPending &g, int b) {
            float cube = 0.f;
            bool ok = false;
            if (waits_pending[b]) {
                ok = mbar_wait_bounded(smem_u32(&s_mbar[b]), phase[b]);
                if (ok) {
                    phase[b] ^= 1u;
                    waits_pending[b] = false;
                    tc_fence_after();
                    const uint32_t taddr = tmem0 + (uint32_t)b * tcols + lane_off;
                    // sum of U^3 in four packed accumulators (columns e mod 8),
                    // so that no single chain of dependent FMAs is long
                    f32x2_t cq[4] = {0ull, 0ull, 0ull, 0ull};
                    for (int cb = 0; cb < gridN; cb += 32) {
                        float u[32];
                        tmem_ld32(taddr + (uint32_t)cb, u);
                        tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 32; e += 2) {
                            const f32x2_t uu = pk2(u[e], u[e + 1]);
                            cq[(e >> 1) & 3] = fma2(mul2(uu, uu), uu, cq[(e >> 1) & 3]);
                        }
                    }
                    float c[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) upk2(cq[q], c[2 * q], c[2 * q + 1]);
                    cube = ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
                    tc_fence_before();
                } else {
                    atomicOr(B.status, kStatusMbarTimeout);
                    s_abort = 1;
                }
            }
            const bool usable = g.valid && ok;
            const uint32_t lo = (uint32_t)g.idx, hi = (uint32_t)(g.idx >> 32);
            const float inv2 = 1.f / g.nrm2;
            const float inv = rsqrtf(g.nrm2);
            const float S = g.Sraw * inv2;
            const float T = cube * tscale * (inv2 * inv);
            const float tS = sc.cS * S;
            const float tH = sc.cH * T;
            const float tQ = UNIF ? 0.f : sc.cQ * logf(g.zz * inv2);
            const float delta = ((tS + tH) + tQ) - sc.logM;
            const uint32_t wa = accept_word(lo, hi, sc.pid, sc.K, k0, k1);
            const float lnU = -0.5f * rho_fast(wa);
            const float d = lnU - delta;
            const float guard = fmaf(
                sc.ge * g.esum, inv,
                fmaf(sc.gq, inv2, sc.ga + sc.gr * (fabsf(tS) + fabsf(tQ) + fabsf(tH) + fabsf(lnU) + fabsf(sc.logM)) + sc.gh));
            // a radius or accept word in the lowest bucket: FP64 pass (refined tail)
            const bool tail = g.tail || wa < kTailBucket;
            bool defer = usable && (fabsf(d) < guard || tail);
            if (usable && !tail) maxd = fmaxf(maxd, delta);
            const unsigned long long li = g.idx - A.idx0[p];
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
                        it.idx = g.idx;
                        it.point = (uint32_t)p;
                        it.pad = 0;
                        B.refine[slot] = it;
                    } else {
                        atomicOr(B.status, kStatusRefineOverflow);
                        atomicAdd(&s_cnt[3], 1u);
                        defer = false;
                    }
                }
            }
            const bool acc = usable && !defer && d < 0.f;
            if (usable && !defer && delta > 0.f) atomicAdd(&s_cnt[1], 1u);
            const unsigned ma = __ballot_sync(0xffffffffu, acc);
            if (ma) {
                const int leader = __ffs(ma) - 1;
                unsigned long long slot0 = 0;
                if (lane == leader) {
                    slot0 = atomicAdd(B.ring_count, (unsigned long long)__popc(ma));
                    atomicAdd(&s_cnt[0], (uint32_t)__popc(ma));
                }
                slot0 = __shfl_sync(0xffffffffu, slot0, leader);
                if (acc) {
                    const unsigned long long slot = slot0 + __popc(ma & ((1u << lane) - 1u));
                    unsigned char *rec = nullptr;
                    if (slot < B.ring_cap)
                        rec = B.ring + slot * B.rec_bytes;
                    else
                        atomicAdd(&s_cnt[2], 1u);
                    // the grid form keeps no projected state: emit_accepted draws it again
                    emit_accepted<KMAX, UNIF>(P, g.idx, (uint32_t)p, k0, k1, s_sig, s_act, s_hist, s_exc, s_q,
                                              s_spec, rec);
                }
            }
        };

        GridPending prev;
        prev.valid = false;
        prev.tail = false;
        bool have_prev = false;
        int b = 0;
        // one extra trip with NBUF = 2 finishes the last tile (a single call
        // site of consume keeps the code, and its instruction-cache footprint, small)
        const uint32_t n_trips = (n_here + NT - 1) / NT + (NBUF == 2 ? 1u : 0u);
        for (uint32_t trip = 0; trip < n_trips; ++trip) {
            const bool produce = trip * NT < n_here;
            const uint32_t i0 = trip * NT;
            const uint32_t i = i0 + (uint32_t)tid;
            GridPending cur;
            cur.valid = produce && i < n_here;
            cur.tail = false;
            cur.idx = cbase + i;
            if (produce) {
                const uint32_t lo = (uint32_t)cur.idx, hi = (uint32_t)(cur.idx >> 32);
                // Row of X in the contraction order: 16-byte chunk c holds
                // (x, y) of modes 4c+1..4c+4, interleaved; chunk c is made from
                // Philox blocks 2c and 2c+1 and stored at once (hi and lo).
                unsigned char *ga_hi = gbase + 2 * btile + (uint32_t)b * 2u * ATILE;
                unsigned char *ga_lo = ga_hi + ATILE;
                float nrm2 = 0.f, Sraw = 0.f, zz = 0.f, esum = 0.f;
                uint32_t wmin = 0xFFFFFFFFu;
    #pragma unroll 4
                for (int cch = 0; cch < KMAX / 4; ++cch) {
                    float v[8];
    #pragma unroll
                    for (int jj = 0; jj < 2; ++jj) {
                        const int j = 2 * cch + jj;
                        const uint4 w = philox4x32_10(make_uint4((uint32_t)j, lo, hi, sc.pid), k0, k1);
    #pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int m = 2 * j + h;
                            const float s = UNIF ? s_act[m] : s_sig[m];
                            float rho, xm, ym, rr;
                            box_muller_f32<false>(h ? w.z : w.x, h ? w.w : w.y, s, rho, xm, ym, rr);
                            wmin = min(wmin, h ? w.z : w.x);
                            esum = fmaf(s, rr, esum);
                            v[4 * jj + 2 * h] = xm;
                            v[4 * jj + 2 * h + 1] = ym;
                            const float sk = (s * s) * rho;
                            nrm2 += sk;
                            Sraw = fmaf((float)((m + 1) * (m + 1)), sk, Sraw);
                            zz += s > 0.f ? rho : 0.f;  // modes above K have sigma = 0
                        }
                    }
                    uint4 hv, lv;
                    split8(v, hv, lv);
                    const uint32_t off = sw128_offset((uint32_t)row, (uint32_t)cch * 8u, 128u);
                    *reinterpret_cast<uint4 *>(ga_hi + off) = hv;
                    *reinterpret_cast<uint4 *>(ga_lo + off) = lv;
                }
                cur.nrm2 = nrm2;
                cur.Sraw = Sraw;
                cur.zz = zz;
                cur.esum = esum;
                cur.tail = wmin < kTailBucket;
                fence_async_smem();
                __syncthreads();
                if (!s_abort) {
                    if (tid == 0) {
                        tc_fence_after();
                        const uint32_t ah = a0 + (uint32_t)b * 2u * ATILE, al = ah + ATILE;
                        const uint32_t dt = tmem0 + (uint32_t)b * tcols;
    #pragma unroll
                        for (int ks = 0; ks < KA / 16; ++ks) {
                            const uint32_t koff = (uint32_t)((ks & 3) * 32);  // 16 BF16 = 32 bytes per step
                            const uint32_t aat = (uint32_t)(ks >> 2) * 128u * 128u;
                            const uint32_t bat = (uint32_t)(ks >> 2) * (uint32_t)gridN * 128u;
                            const uint64_t dah = sw128_desc(ah + aat + koff), dal = sw128_desc(al + aat + koff);
                            const uint64_t dbh = sw128_desc(b_hi + bat + koff), dbl = sw128_desc(b_lo + bat + koff);
                            umma_bf16(dt, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                            umma_bf16(dt, dah, dbl, idesc, 1u);
                            umma_bf16(dt, dal, dbh, idesc, 1u);
                        }
                        umma_commit(smem_u32(&s_mbar[b]));
                    }
                    waits_pending[b] = true;
                }
            }
            if (NBUF == 2) {
                if (have_prev) consume(prev, b ^ 1);
                prev = cur;
                have_prev = produce;
                b ^= 1;
            } else {
                consume(cur, b);
            }
        }

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
        for (int e = tid; e < KMAX; e += NT) {
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
    // a commit that timed out may still land: wait for it (bounded) before
    // the accumulator columns are released
#pragma unroll
    for (int bb = 0; bb < NBUF; ++bb)
        if (waits_pending[bb]) (void)mbar_wait_bounded(smem_u32(&s_mbar[bb]), phase[bb]);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) tmem_dealloc(s_tmem, tcols * NBUF);
}

template <int KMAX, int NBUF>
void fill_grid_kernels(GridKernels *t) {
    t->main[0] = (const void *)k_sample_grid<KMAX, false, NBUF>;
    t->main[1] = (const void *)k_sample_grid<KMAX, true, NBUF>;
    t->nwg = NBUF;
    t->kmax = KMAX;
    t->ka = GridShape<KMAX>::KA;
}

}  // namespace tkdv

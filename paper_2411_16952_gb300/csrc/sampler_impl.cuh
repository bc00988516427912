// sampler_impl.cuh - device code of the rejection sampler (Sec. IV.B of
// Moore & Foerster, arXiv 2411.16952): one proposal per thread, everything in
// registers, a persistent CTA loop over chunks of proposal indices.
//
// Per proposal (FP32 fast path):
//   1. Philox4x32-10 words for proposal idx (stream layout in include/tkdv.h);
//   2. Box-Muller pairs -> the 2K standard normals of Eq. (14);
//   3. scale by sigma_k (Eqs. 24-26); |x|^2, S|x|^2 and Q|x|^2 accumulate as
//      the normals are made, so the projection xhat = x/|x| (Sec. IV.B) is
//      applied as scalar factors, never to the 2K components;
//   4. H3 by the double sum of Eq. (42) with the k <-> n-k symmetry folded,
//      two products per packed FP32 instruction;
//   5. log f/(M g) = -beta' S/K^2 + beta' r/(E0 K^2) H3 + K ln Q - log M
//      (Eqs. 40 and 43);
//   6. accept iff ln U < log f/(M g).  The FP32 result decides only when the
//      two sides differ by more than a rounding-error bound ("guard"); inside
//      the guard band the proposal is queued and decided in FP64 by
//      k_refine (same draw, same formulas).  So every decision equals the
//      one an exact evaluation takes, up to FP64 rounding.
//   7. warp-ballot compaction of accepted records into a ring, and streaming
//      statistics of u(0) (Sec. V) in shared memory, flushed per chunk with
//      integer atomics.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "tkdv_internal.h"

namespace tkdv {

// ---- Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) ------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same block with the round keys given (RoundKeys: round r uses
// rk[2r], rk[2r+1]); rk points at the run's kernel arguments, so every key is
// a constant operand of its round.  Each round's two products are formed as
// full 64-bit products (one wide multiply each, high and low words together).
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t *rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53ull;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57ull;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1],
                       (uint32_t)p0);
    }
    return c;
}
// The blocks (j, lo, hi, pid), j = 0, 1, ..., of one proposal from the round
// keys.  (Making the two products that do not depend on j, M1 hi in round 1
// and M0 (hi(M1 hi) ^ lo ^ rk[0]) in round 2, once per proposal measured
// no faster: 10.91e9 against 10.98e9 proposals/s at K = 32.)
struct PhiloxRow {
    const uint32_t *rk;
    uint32_t lo, hi, pid;
    __device__ __forceinline__ PhiloxRow(uint32_t lo_, uint32_t hi_, uint32_t pid_, const uint32_t *rk_)
        : rk(rk_), lo(lo_), hi(hi_), pid(pid_) {}
    __device__ __forceinline__ uint4 block(uint32_t j) const { return philox4x32_10_rk(make_uint4(j, lo, hi, pid), rk); }
};

// one_m(w): the float 1 + (w >> 9) 2^-23, i.e. the bits 0x3f800000 | (w >> 9),
// by one funnel shift of (127 : w) right by 9.
__device__ __forceinline__ float one_m(uint32_t w) { return __uint_as_float(__funnelshift_r(w, 0x7Fu, 9)); }
// (2 floor(w/512) + 1) 2^-24, exact in FP32: the float 1 + m 2^-23 with
// m = w >> 9 is built from its bits, and subtracting 1 - 2^-24 (a float) is
// exact (Sterbenz), leaving (2m + 1) 2^-24.
__device__ __forceinline__ float u01f(uint32_t w) { return one_m(w) - 0x1.fffffep-1f; }
__device__ __forceinline__ double u01d(uint32_t w) {
    return (double)((w >> 8) | 1u) * 0x1p-24;
}

// The map above puts every u < 2^-23 at 2^-24.  That would cap the
// Box-Muller radius (rho <= -2 ln 2^-24 = 33.3) and the accept test
// (ln U >= -16.6, so a draw with Delta below that could never be accepted,
// although the rule accepts it with probability e^Delta).  A word in the
// lowest bucket (w < kTailBucket) is refined by word 0 of the Philox blocks
// with counter (kTailCtr + L 2^24 + g, idx_lo, idx_hi, point_id), L = 1, 2,
// where g = 4 * block + word is the position of the refined word in the
// proposal's stream: U = 2^-23 u(w_1) if w_1 is above the lowest bucket, else
// 2^-46 u(w_2).  U is then uniform with 23 bits of relative resolution down to
// 2^-70.  The FP32 fast path only detects such words (1 in 2^23) and sends the
// proposal to the FP64 pass, which applies the refinement.
constexpr uint32_t kTailBucket = 512u;
constexpr uint32_t kTailCtr = 0x80000000u;

static __device__ __noinline__ double u01d_tail(uint32_t g, uint32_t lo, uint32_t hi, uint32_t pid, uint32_t k0,
                                                uint32_t k1) {
    const uint32_t w1 = philox4x32_10(make_uint4(kTailCtr + (1u << 24) + g, lo, hi, pid), k0, k1).x;
    if (w1 >= kTailBucket) return 0x1p-23 * u01d(w1);
    const uint32_t w2 = philox4x32_10(make_uint4(kTailCtr + (2u << 24) + g, lo, hi, pid), k0, k1).x;
    return 0x1p-46 * u01d(w2);
}

// The uniform of word w at stream position g, its lowest bucket refined.
__device__ __forceinline__ double u01d_ext(uint32_t w, uint32_t g, uint32_t lo, uint32_t hi, uint32_t pid,
                                           uint32_t k0, uint32_t k1) {
    return w >= kTailBucket ? u01d(w) : u01d_tail(g, lo, hi, pid, k0, k1);
}

// 2 pi (u - 1/2) for u = u01f(w), rounded once: (1 + m 2^-23) - 3/2 is exact,
// and 2 pi (u - 1/2) = 2 pi ((1 + m 2^-23) - 3/2) + 2 pi 2^-24 takes one FMA.
__device__ __forceinline__ float angle_f(uint32_t w) {
    constexpr float k2Pi = 6.28318530717958647692f;
    return fmaf(k2Pi, one_m(w) - 1.5f, k2Pi * 0x1p-24f);
}

// The hardware approximations of PTX (lg2, rsqrt, sin, cos .approx) in their
// flush-to-zero forms.  Every argument the sampler gives them (u in
// [2^-24, 1), rho >= 2^-25, |x|^2 > 0, angles of magnitude >= 2 pi 2^-24) and
// every result is a normal float, where the flushing forms return the same
// documented approximation without handling for subnormal operands.
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 1/x correctly rounded (the value of 1.f / x) for normal x and 1/x: the
// flushing form of the rounded reciprocal, without the subnormal path of the
// division.
__device__ __forceinline__ float rcp_rn(float x) {
    float y;
    asm("rcp.rn.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void sincos_approx(float a, float &sn, float &cs) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(sn) : "f"(a));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(cs) : "f"(a));
}

// Squared Box-Muller radius rho = -2 ln u for u = u01f(w), FP32.
// rho_fast (the decision path) takes the hardware base-2 logarithm, whose
// documented error is at most 2 ulp below 1/2 and 2^-22 absolute on [1/2, 2):
// |rho_fast - rho| <= kRhoAbsErr + kRhoRelErr rho (tkdv_check_radius_error
// measures it over all 2^23 values); the decision guard takes the absolute
// part per draw from sum_m sigma_m / sqrt(rho_m).  The floor keeps rho
// positive where that error could cross zero.
__device__ __forceinline__ float rho_fast(uint32_t w) {
    return fmaxf(lg2_approx(u01f(w)) * -1.38629436111989061883f, 0x1p-25f);
}
// rho_acc (the outputs of accepted draws) is rho_fast below u = 1 - 2^-9
// (there rho >= 2^-8 and the absolute error is a small relative one) and
// above it the series -2 ln(1 - t) = 2t (1 + t/2 + t^2/3), t = 1 - u = u01f(~w)
// exact (the map is symmetric), truncated below 2e-9 relative.
__device__ __forceinline__ float rho_acc(uint32_t w) {
    const float t = u01f(~w);
    const float ser = (2.f * t) * fmaf(t, fmaf(t, 1.f / 3.f, 0.5f), 1.f);
    return w >= 0xFF800000u ? ser : rho_fast(w);
}
// Outputs: an error e in rho moves the projected component of mode m by at
// most sigma_m e / (2 sqrt(rho_m) |x|); with rho_fast's 3.3e-7 above the
// series range that stays below 1e-6 while max_m sigma_m / sqrt(rho_m) / |x|
// <= 6.  An accepted draw above it (about 1 % of them at K = 32) takes its
// outputs from rho_acc instead.
constexpr float kOutputRr = 6.f;

// rho_log: the radius of the warp form (65..128 modes), the full-precision
// logarithm (at most 1 ulp): |rho_log - rho| <= kRhoLogRelErr rho, no absolute
// part (tkdv_check_radius_error_log measures it over all 2^23 values).  Its
// outputs need no second pass, and its decision guard has no per-draw radius
// terms.
__device__ __forceinline__ float rho_log(uint32_t w) { return -2.f * logf(u01f(w)); }

// Box-Muller pair in FP32, scaled by s: rho = -2 ln u1 (the squared radius),
// and (x, y) = s sqrt(rho) (cos 2 pi u2, sin 2 pi u2).  The angle is reduced
// exactly to 2 pi (u2 - 1/2) in (-pi, pi), where the hardware sine/cosine have
// an absolute error below 2^-21.4, and cos(t - pi) = -cos t, sin(t - pi) =
// -sin t restore the signs; s sqrt(rho) = (s rho) rsqrt(rho).  The FP32
// decision guard covers these errors (draws near the threshold are redone in
// FP64).  rr returns 1/sqrt(rho).
template <bool ACC>
__device__ __forceinline__ void box_muller_f32(uint32_t w1, uint32_t w2, float s, float &rho, float &x, float &y,
                                               float &rr) {
    rho = ACC ? rho_acc(w1) : rho_fast(w1);
    rr = rsqrt_approx(rho);
    const float a = (-s * rho) * rr;
    float sn, cs;
    sincos_approx(angle_f(w2), sn, cs);
    x = a * cs;
    y = a * sn;
}

// Order-preserving map float -> uint32 (for atomicMax on signed floats).
__device__ __forceinline__ uint32_t fkey(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Scalar constants of the current point, held in registers.
struct Scal {
    float cS, cH, cQ, logM, u0s, h3s, E0, ga, gr, gh, ge, gq, ha, hb, ea, lnc;
    uint32_t pid;
    int K;
};

__device__ __forceinline__ Scal load_scal(const PointConst *P) {
    Scal s;
    s.cS = __ldg(&P->cS);
    s.cH = __ldg(&P->cH);
    s.cQ = __ldg(&P->cQ);
    s.logM = __ldg(&P->logM_f);
    s.u0s = __ldg(&P->u0s);
    s.h3s = __ldg(&P->h3s);
    s.E0 = __ldg(&P->E0);
    s.ga = __ldg(&P->guard_abs);
    s.gr = __ldg(&P->guard_rel);
    s.gh = __ldg(&P->guard_h);
    s.ge = __ldg(&P->guard_e);
    s.gq = __ldg(&P->guard_q);
    s.lnc = __ldg(&P->sir_lnc);
    s.ha = __ldg(&P->hist_a);
    s.hb = __ldg(&P->hist_b);
    s.ea = __ldg(&P->exc_a);
    s.pid = __ldg(&P->point_id);
    s.K = __ldg(&P->K);
    return s;
}

// State of one proposal on the fast path: x, y are the scaled (unprojected)
// cosine and sine halves of mode m = 0..KMAX-1.
template <int KMAX>
struct Draw {
    float x[KMAX], y[KMAX];
    float nrm2;     // |x|^2
    float Sraw;     // sum k^2 (x_k^2 + y_k^2)  = S |x|^2
    float zz;       // sum over active modes of the normals' squares = Q |x|^2
    float u0raw;    // sum_k x_k                = u(0) |x| / u0s
    uint32_t wmin;  // smallest radius word: below kTailBucket the draw needs the FP64 pass
    float esum;     // sum_m sigma_m / sqrt(rho_m): scales the radius-error guard
    float rrmax;    // largest sigma_m/sqrt(rho_m): above kOutputRr |x| outputs need rho_acc
};

// The blocks of one proposal: from the key pair (key schedule computed per
// block), or PhiloxRow from the run's round keys.
struct PairRow {
    uint32_t lo, hi, pid, k0, k1;
    __device__ __forceinline__ uint4 block(uint32_t j) const { return philox4x32_10(make_uint4(j, lo, hi, pid), k0, k1); }
};

// Per-mode constants of a draw, (s, s^2, (m+1)^2 s^2, act) with s = sigma_m
// (the act flag for the uniform proposal), so that each accumulation of a
// mode is one FMA with the squared radius.  ModeSigAct forms them from a
// point's sigma and act arrays; ModeTab reads the same values from a table
// (one 16-byte load per mode).
template <bool UNIF>
__device__ __forceinline__ float4 mode_consts(float sig, float act, int m) {
    const float s = UNIF ? act : sig;
    const float s2 = s * s;
    return make_float4(s, s2, (float)((m + 1) * (m + 1)) * s2, act);
}
template <bool UNIF>
struct ModeSigAct {
    const float *sig, *act;
    __device__ __forceinline__ float4 operator()(int m) const { return mode_consts<UNIF>(sig[m], act[m], m); }
};
struct ModeTab {
    const float4 *md;
    __device__ __forceinline__ float4 operator()(int m) const { return md[m]; }
};

// Steps 1-3 for modes 0..KMAX-1.  Modes beyond K have sigma = act = 0.
template <int KMAX, bool UNIF, bool ACC = false, typename Row = PairRow, typename Modes = ModeSigAct<UNIF>>
__device__ __forceinline__ void draw_fast_k(Draw<KMAX> &d, const Modes &modes, const Row &row);

template <int KMAX, bool UNIF, bool ACC = false>
__device__ __forceinline__ void draw_fast(Draw<KMAX> &d, const float *sig, const float *act,
                                          uint32_t idx_lo, uint32_t idx_hi, uint32_t pid,
                                          uint32_t k0, uint32_t k1) {
    draw_fast_k<KMAX, UNIF, ACC>(d, ModeSigAct<UNIF>{sig, act}, PairRow{idx_lo, idx_hi, pid, k0, k1});
}

template <int KMAX, bool UNIF, bool ACC, typename Row, typename Modes>
__device__ __forceinline__ void draw_fast_k(Draw<KMAX> &d, const Modes &modes, const Row &row) {
    d.nrm2 = 0.f;
    d.Sraw = 0.f;
    d.zz = 0.f;
    d.u0raw = 0.f;
    d.wmin = 0xFFFFFFFFu;
    d.esum = 0.f;
    d.rrmax = 0.f;
#pragma unroll
    for (int j = 0; j < (KMAX + 1) / 2; ++j) {
        const uint4 w = row.block((uint32_t)j);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * j + h;
            if (m < KMAX) {
                const float4 c = modes(m);
                float rho, xm, ym, rr;
                box_muller_f32<ACC>(h ? w.z : w.x, h ? w.w : w.y, c.x, rho, xm, ym, rr);
                d.wmin = min(d.wmin, h ? w.z : w.x);
                const float srr = c.x * rr;
                d.esum += srr;
                d.rrmax = fmaxf(d.rrmax, srr);
                d.x[m] = xm;
                d.y[m] = ym;
                d.nrm2 = fmaf(c.y, rho, d.nrm2);
                d.Sraw = fmaf(c.z, rho, d.Sraw);
                d.zz = fmaf(c.w, rho, d.zz);  // modes above K have act = 0
                d.u0raw += xm;
            }
        }
    }
}

// ---- packed FP32 pairs (sm_100+ f32x2 instructions: one issue, two lanes) ----
typedef unsigned long long f32x2_t;
__device__ __forceinline__ f32x2_t pk2(float lo, float hi) {
    f32x2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f32x2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2_t fma2(f32x2_t a, f32x2_t b, f32x2_t c) {
    f32x2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2_t mul2(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t add2(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Step 4: T = sum_{n=2}^{KMAX} x_n A_n + y_n B_n, with
//   A_n = sum_{k=1}^{n-1} x_k x_{n-k} - y_k y_{n-k},
//   B_n = sum_{k=1}^{n-1} x_k y_{n-k} + y_k x_{n-k},
// i.e. Re(conj(v_n) sum v_k v_{n-k}) for v = x - i y (Eq. 42 up to 2 pi c^3).
// Packed pairs: with V_m = (x_m, y_m) and S_m = (y_m, x_m),
//   V_k . V_m (elementwise) = (x_k x_m, y_k y_m)  -> A-part = lo - hi,
//   V_k . S_m               = (x_k y_m, y_k x_m)  -> B-part = lo + hi,
// so each symmetric pair (k, n-k) costs two packed FMAs.  The x- and
// y-products are summed apart and subtracted at the end; every term passes
// through no more roundings than in a scalar sum over the same pairs, so the
// rounding-error bound behind the accept guard band holds.
template <int KMAX>
__device__ __forceinline__ float triad2(const float *x, const float *y) {
    f32x2_t V[KMAX], S[KMAX];
#pragma unroll
    for (int m = 0; m < KMAX; ++m) {
        V[m] = pk2(x[m], y[m]);
        S[m] = pk2(y[m], x[m]);
    }
    const f32x2_t two = pk2(2.f, 2.f);
    float T = 0.f;
#pragma unroll
    for (int n = 2; n <= KMAX; ++n) {
        f32x2_t P1 = 0ull, P2 = 0ull;  // 0ull is the pair (+0, +0)
#pragma unroll
        for (int k = 1; 2 * k < n; ++k) {
            P1 = fma2(V[k - 1], V[n - k - 1], P1);
            P2 = fma2(V[k - 1], S[n - k - 1], P2);
        }
        if ((n & 1) == 0) {
            const int h = n / 2;
            P1 = fma2(P1, two, mul2(V[h - 1], V[h - 1]));
            P2 = fma2(P2, two, mul2(V[h - 1], S[h - 1]));
        } else {
            P1 = mul2(P1, two);
            P2 = mul2(P2, two);
        }
        float a0, a1, b0, b1;
        upk2(P1, a0, a1);
        upk2(P2, b0, b1);
        T = fmaf(x[n - 1], a0 - a1, T);
        T = fmaf(y[n - 1], b0 + b1, T);
    }
    return T;
}

struct Fast {
    float delta, lnU, d, guard, S, T, inv;
};

// Steps 4-6 on the fast path.
template <int KMAX, bool UNIF>
__device__ __forceinline__ Fast eval_fast(const Draw<KMAX> &dr, const Scal &c, uint32_t wacc) {
    Fast f;
    const float inv2 = rcp_rn(dr.nrm2);
    f.inv = rsqrt_approx(dr.nrm2);
    f.S = dr.Sraw * inv2;
    f.T = triad2<KMAX>(dr.x, dr.y) * (inv2 * f.inv);
    const float tS = c.cS * f.S;
    const float tH = c.cH * f.T;
    const float tQ = UNIF ? 0.f : c.cQ * logf(dr.zz * inv2);
    f.delta = ((tS + tH) + tQ) - c.logM;
    f.lnU = -0.5f * rho_fast(wacc);
    f.d = f.lnU - f.delta;
    f.guard = fmaf(c.ge * dr.esum, f.inv,
                   fmaf(c.gq, inv2, c.ga + c.gr * (fabsf(tS) + fabsf(tQ) + fabsf(tH) + fabsf(f.lnU) + fabsf(c.logM)) + c.gh));
    return f;
}

__device__ __forceinline__ uint32_t accept_word(uint32_t idx_lo, uint32_t idx_hi, uint32_t pid,
                                                int K, uint32_t k0, uint32_t k1) {
    return philox4x32_10(make_uint4((uint32_t)((K + 1) / 2), idx_lo, idx_hi, pid), k0, k1).x;
}

__device__ __forceinline__ int hist_bin(float u0, float a, float b) {
    int v = __float2int_rd(fmaf(u0, a, b));
    return min(max(v, 0), kHistBins - 1);
}
__device__ __forceinline__ int exc_bin(float u0, float a) {
    if (!(u0 > 0.f)) return 0;
    int v = __float2int_ru(u0 * a);
    return min(v, kExcBins - 1);
}

// ---- FP64 evaluation of one proposal (guard band, replay) -----------------
struct Out64 {
    double delta, lnU, u, S, T;
    float H2, H3, u0;
    int accept, near;
};

// The same draw and the same formulas as the fast path, in FP64.  xh (may be
// null) receives the projected state [cos | sin] as floats.
template <int KMAX, bool UNIF>
__device__ __noinline__ void eval64(const PointConst *P, unsigned long long idx, uint32_t k0,
                                    uint32_t k1, Out64 *o, float *xh) {
    const int K = P->K;
    const uint32_t lo = (uint32_t)idx, hi = (uint32_t)(idx >> 32), pid = P->point_id;
    double x[KMAX], y[KMAX];
    double nrm2 = 0.0, Sraw = 0.0, zz = 0.0, u0raw = 0.0;
    for (int m = 0; m < KMAX; ++m) {
        x[m] = 0.0;
        y[m] = 0.0;
    }
    for (int m = 0; m < K; ++m) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(m / 2), lo, hi, pid), k0, k1);
        const int h = m & 1;
        const double u1 = u01d_ext(h ? w.z : w.x, 2u * (uint32_t)m, lo, hi, pid, k0, k1);
        const double u2 = u01d(h ? w.w : w.y);
        const double rho = -2.0 * log(u1);
        const double rad = sqrt(rho);
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        const double s = UNIF ? 1.0 : P->sigma_d[m];
        x[m] = s * rad * cs;
        y[m] = s * rad * sn;
        const double sk = x[m] * x[m] + y[m] * y[m];
        nrm2 += sk;
        Sraw += (double)((m + 1) * (m + 1)) * sk;
        zz += rho;
        u0raw += x[m];
    }
    double T = 0.0;
    for (int n = 2; n <= K; ++n) {
        double A = 0.0, Bv = 0.0;
        for (int k = 1; k <= n - 1; ++k) {
            A += x[k - 1] * x[n - k - 1] - y[k - 1] * y[n - k - 1];
            Bv += x[k - 1] * y[n - k - 1] + y[k - 1] * x[n - k - 1];
        }
        T += x[n - 1] * A + y[n - 1] * Bv;
    }
    const double inv = 1.0 / sqrt(nrm2);
    const double inv2 = inv * inv;
    o->S = Sraw * inv2;
    o->T = T * inv2 * inv;
    double delta = P->cS_d * o->S + P->cH_d * o->T;
    if (!UNIF) delta += P->cQ_d * log(zz * inv2);
    delta -= P->logM;
    const uint32_t wa = accept_word(lo, hi, pid, K, k0, k1);
    o->delta = delta;
    o->u = u01d_ext(wa, 4u * (uint32_t)((K + 1) / 2), lo, hi, pid, k0, k1);
    o->lnU = log(o->u);
    o->accept = o->lnU < delta;
    o->near = fabs(o->lnU - delta) < 1e-6;
    o->H2 = (float)((double)P->E0 * o->S);
    o->H3 = (float)((double)P->h3s * o->T);
    o->u0 = (float)((double)P->u0s * u0raw * inv);
    if (xh) {
        for (int m = 0; m < K; ++m) {
            xh[m] = (float)(x[m] * inv);
            xh[K + m] = (float)(y[m] * inv);
        }
    }
}

// Write the 32-byte header of one accepted record (the projected state follows it).
__device__ __forceinline__ void write_header(unsigned char *rec, unsigned long long idx, uint32_t point,
                                             uint32_t flags, float H2, float H3, float u0, float delta) {
    *reinterpret_cast<unsigned long long *>(rec) = idx;
    uint32_t *h = reinterpret_cast<uint32_t *>(rec + 8);
    h[0] = point;
    h[1] = flags;
    float *f = reinterpret_cast<float *>(rec + 16);
    f[0] = H2;
    f[1] = H3;
    f[2] = u0;
    f[3] = delta;
}

// Write one accepted record.
template <int KMAX>
__device__ __forceinline__ void write_record(unsigned char *rec, unsigned long long idx, uint32_t point,
                                             uint32_t flags, float H2, float H3, float u0, float delta,
                                             const float *x, const float *y, float inv, int K) {
    *reinterpret_cast<unsigned long long *>(rec) = idx;
    uint32_t *h = reinterpret_cast<uint32_t *>(rec + 8);
    h[0] = point;
    h[1] = flags;
    float *f = reinterpret_cast<float *>(rec + 16);
    f[0] = H2;
    f[1] = H3;
    f[2] = u0;
    f[3] = delta;
    float *xh = f + 4;
#pragma unroll
    for (int m = 0; m < KMAX; ++m) {
        if (m < K) {
            xh[m] = x[m] * inv;
            xh[K + m] = y[m] * inv;
        }
    }
}

// Statistics of one accepted draw into the CTA's shared-memory partials.  Out
// of line: accepted draws are rare, and keeping this code out of the hot loop
// keeps that loop's instruction-cache footprint small.
static __device__ __noinline__ void tally_accepted(float u0, float ha, float hb, float ea, uint32_t *s_hist,
                                            uint32_t *s_exc, unsigned long long *s_q) {
    atomicAdd(&s_hist[hist_bin(u0, ha, hb)], 1u);
    atomicAdd(&s_exc[exc_bin(u0, ea)], 1u);
    const float u2 = u0 * u0;
    atomicAdd(&s_q[0], (unsigned long long)__float2ll_rn(u0 * kQ1));
    atomicAdd(&s_q[1], (unsigned long long)__float2ll_rn(u2 * kQ2));
    atomicAdd(&s_q[2], (unsigned long long)__float2ll_rn(u2 * u0 * kQ3));
    atomicAdd(&s_q[3], (unsigned long long)__float2ll_rn(u2 * u2 * kQ4));
}

// Power spectrum of an accepted draw (mean of s_k = xh_k^2 + xh_{K+k}^2 over
// the accepted fields, Sec. V.A) into shared fixed-point sums.
template <int KMAX>
__device__ __forceinline__ void tally_spectrum(unsigned long long *s_spec, const float *x, const float *y, float inv2,
                                               int K) {
    const float sc = inv2 * kSpecScale;
#pragma unroll
    for (int m = 0; m < KMAX; ++m)
        if (m < K) atomicAdd(&s_spec[m], (unsigned long long)__float2ull_rn(fmaf(x[m], x[m], y[m] * y[m]) * sc));
}

// Outputs of one accepted draw made again with rho_acc: used by the grid form,
// which keeps no per-mode state, and by the triad form for the few accepted
// draws holding a radius of the series range.  The draw is evaluated in FP32
// (T by the double sum), its u(0) statistics and spectrum are tallied, and
// its record is written when rec is not null (ring full).  Out of line:
// accepted draws are rare, and the hot loops keep neither this code nor its
// registers.
template <int KMAX, bool UNIF>
__device__ __noinline__ void emit_accepted(const PointConst *P, unsigned long long idx, uint32_t point, uint32_t k0,
                                           uint32_t k1, const float *sig, const float *act, uint32_t *s_hist,
                                           uint32_t *s_exc, unsigned long long *s_q, unsigned long long *s_spec,
                                           unsigned char *rec) {
    const Scal sc = load_scal(P);
    Draw<KMAX> dr;
    draw_fast<KMAX, UNIF, true>(dr, sig, act, (uint32_t)idx, (uint32_t)(idx >> 32), sc.pid, k0, k1);
    const float inv2 = rcp_rn(dr.nrm2);
    const float inv = rsqrt_approx(dr.nrm2);
    const float S = dr.Sraw * inv2;
    const float T = triad2<KMAX>(dr.x, dr.y) * (inv2 * inv);
    const float tQ = UNIF ? 0.f : sc.cQ * logf(dr.zz * inv2);
    const float delta = ((sc.cS * S + sc.cH * T) + tQ) - sc.logM;
    const float u0 = sc.u0s * dr.u0raw * inv;
    tally_accepted(u0, sc.ha, sc.hb, sc.ea, s_hist, s_exc, s_q);
    tally_spectrum<KMAX>(s_spec, dr.x, dr.y, inv2, sc.K);
    if (rec) write_record<KMAX>(rec, idx, point, 0u, sc.E0 * S, sc.h3s * T, u0, delta, dr.x, dr.y, inv, sc.K);
}

// Outputs of one accepted draw made again with rho_acc, in two passes so that
// its 2K components are never all held: pass 1 sums |x|^2, S|x|^2 and
// sum_k x_k (u(0) |x| / u0s) in mode order, pass 2 draws the modes again and
// writes the projected state into the record (xh may be null: ring full) and
// the spectrum terms.  The arithmetic and its order are those of draw_fast
// and write_record / tally_spectrum, so the values are the same.
struct DrawSums {
    float nrm2, Sraw, u0raw;
};
template <int KMAX, bool UNIF>
__device__ __forceinline__ DrawSums acc_draw_sums(const float *sig, const float *act, uint32_t lo, uint32_t hi,
                                                  uint32_t pid, uint32_t k0, uint32_t k1) {
    DrawSums d{0.f, 0.f, 0.f};
#pragma unroll 1
    for (int j = 0; j < (KMAX + 1) / 2; ++j) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)j, lo, hi, pid), k0, k1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * j + h;
            if (m < KMAX) {
                const float4 c = mode_consts<UNIF>(sig[m], act[m], m);
                float rho, xm, ym, rr;
                box_muller_f32<true>(h ? w.z : w.x, h ? w.w : w.y, c.x, rho, xm, ym, rr);
                d.nrm2 = fmaf(c.y, rho, d.nrm2);
                d.Sraw = fmaf(c.z, rho, d.Sraw);
                d.u0raw += xm;
            }
        }
    }
    return d;
}
template <int KMAX, bool UNIF>
__device__ __forceinline__ void acc_draw_emit(const float *sig, const float *act, uint32_t lo, uint32_t hi,
                                              uint32_t pid, uint32_t k0, uint32_t k1, float inv, float inv2, int K,
                                              float *xh, unsigned long long *s_spec, int rot = 0) {
    // rot: the block this lane starts at, so that the lanes of a warp tally
    // different modes at a time (the integer sums do not depend on the order)
    constexpr int NB = (KMAX + 1) / 2;
    const float sc = inv2 * kSpecScale;
#pragma unroll 1
    for (int jr = 0; jr < NB; ++jr) {
        const int j = jr + rot < NB ? jr + rot : jr + rot - NB;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)j, lo, hi, pid), k0, k1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * j + h;
            if (m < K) {
                const float s = UNIF ? act[m] : sig[m];
                float rho, xm, ym, rr;
                box_muller_f32<true>(h ? w.z : w.x, h ? w.w : w.y, s, rho, xm, ym, rr);
                atomicAdd(&s_spec[m], (unsigned long long)__float2ull_rn(fmaf(xm, xm, ym * ym) * sc));
                if (xh) {
                    xh[m] = xm * inv;
                    xh[K + m] = ym * inv;
                }
            }
        }
    }
}

// ---- the persistent sampler ----------------------------------------------
// Floats between two threads' slabs of the accept hand-off (2 KMAX + 4: the
// 16-byte pad moves consecutive lanes' vector stores to different banks).
template <int KMAX>
__host__ __device__ constexpr int xfer_stride() { return 2 * KMAX + 4; }

// XFER: accepted draws hand their state to the warp through shared memory
// (dynamic, xfer_stride floats per thread); else each accepted draw's lane
// tallies its spectrum and writes its record itself.  The first pays off
// once a warp iteration often holds an accepted draw, the second can spill
// less under a tight register budget; the autotune times both.
template <int KMAX, bool UNIF, int NT, int MINB, bool SIR = false, bool XFER = true>
__global__ void __launch_bounds__(NT, MINB)
    k_sample_triad(const __grid_constant__ DevBufs B, const __grid_constant__ RunArgs A, uint32_t k0, uint32_t k1) {
    __shared__ uint32_t s_hist[kHistBins];
    __shared__ uint32_t s_exc[kExcBins];
    __shared__ unsigned long long s_q[4];
    __shared__ unsigned long long s_spec[KMAX];
    __shared__ double s_sir[SIR ? 7 : 1];
    __shared__ uint32_t s_cnt[4];  // accepted, envelope violations, dropped, fallbacks
    __shared__ uint32_t s_maxd;
    __shared__ uint32_t s_chunk;
    __shared__ float s_sig[KMAX], s_act[KMAX];
    __shared__ float4 s_md[KMAX];
    // dynamic: per thread, its accepted draw's scaled state (x | y), padded
    // (kXferStride floats apart, so that the lanes' vector stores spread over
    // the banks); absent in the SIR form
    extern __shared__ __align__(16) float s_xfer[];

    const int tid = threadIdx.x, lane = tid & 31;
    for (int e = tid; e < kHistBins; e += NT) s_hist[e] = 0;
    for (int e = tid; e < KMAX; e += NT) s_spec[e] = 0ull;
    if (SIR && tid < 7) s_sir[tid] = 0.0;
    if (tid < kExcBins) s_exc[tid] = 0;
    if (tid < 4) {
        s_q[tid] = 0ull;
        s_cnt[tid] = 0;
    }
    if (tid == 0) s_maxd = 0;
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
        if (tid < KMAX) {
            const float sg = __ldg(&P->sigma[tid]), ac = __ldg(&P->act[tid]);
            s_sig[tid] = sg;
            s_act[tid] = ac;
            s_md[tid] = mode_consts<UNIF>(sg, ac, tid);
        }
        const Scal sc = load_scal(P);
        __syncthreads();

        float maxd = -INFINITY;
        float a_sir[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // SIR: w, w^2, w S, w u0^p
        for (uint32_t i0 = 0; i0 < n_here; i0 += NT) {
            const uint32_t i = i0 + (uint32_t)tid;
            const bool valid = i < n_here;
            const unsigned long long idx = base + i;
            const uint32_t lo = (uint32_t)idx, hi = (uint32_t)(idx >> 32);
            Draw<KMAX> dr;
            const PhiloxRow prow(lo, hi, sc.pid, A.rk.k);
            // the per-mode constants from the table, or formed from sigma and
            // act where the table's loads spill under the hand-off variant's
            // register budget (the same values either way)
            if constexpr (XFER)
                draw_fast_k<KMAX, UNIF>(dr, ModeSigAct<UNIF>{s_sig, s_act}, prow);
            else
                draw_fast_k<KMAX, UNIF>(dr, ModeTab{s_md}, prow);
            const uint32_t wa = prow.block((uint32_t)((sc.K + 1) / 2)).x;
            const Fast f = eval_fast<KMAX, UNIF>(dr, sc, wa);
            // a radius or accept word in the lowest bucket: FP64 pass (refined tail)
            const bool tail = min(dr.wmin, wa) < kTailBucket;
            bool defer;
            if (SIR) {
                // at least one copy needs U < P(N >= 1) = 1 - exp(-lambda),
                // lambda = c exp(delta); every proposal that may get one goes
                // to the FP64 pass, which draws its copy number exactly
                const float lnT1 = logf(-expm1f(-expf(f.delta + sc.lnc)));
                defer = valid && (f.lnU - lnT1 < f.guard + sc.gr * fabsf(lnT1) + 1e-6f || tail);
                if (valid) {
                    const float w = expf(f.delta);
                    const float u0 = sc.u0s * dr.u0raw * f.inv;
                    a_sir[0] += w;
                    a_sir[1] = fmaf(w, w, a_sir[1]);
                    a_sir[2] = fmaf(w, f.S, a_sir[2]);
                    float pw = w * u0;
                    a_sir[3] += pw;
                    pw *= u0;
                    a_sir[4] += pw;
                    pw *= u0;
                    a_sir[5] += pw;
                    pw *= u0;
                    a_sir[6] += pw;
                }
            } else {
                defer = valid && (fabsf(f.d) < f.guard || tail);
            }
            if (valid && !tail) maxd = fmaxf(maxd, f.delta);

            // guard band -> FP64 queue
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
                    } else {  // queue full: decide in FP32 and flag the run
                        atomicOr(B.status, kStatusRefineOverflow);
                        atomicAdd(&s_cnt[3], 1u);
                        defer = false;
                    }
                }
            }
            const bool acc = !SIR && valid && !defer && f.d < 0.f;
            if (!SIR && valid && !defer && f.delta > 0.f) atomicAdd(&s_cnt[1], 1u);

            if constexpr (XFER) {
                const unsigned ma = __ballot_sync(0xffffffffu, acc);
                if (ma) {
                    const int leader = __ffs(ma) - 1;
                    unsigned long long slot0 = 0;
                    if (lane == leader) {
                        slot0 = atomicAdd(B.ring_count, (unsigned long long)__popc(ma));
                        atomicAdd(&s_cnt[0], (uint32_t)__popc(ma));
                    }
                    slot0 = __shfl_sync(0xffffffffu, slot0, leader);
                    unsigned char *rec = nullptr;
                    bool redo = false;
                    if (acc) {
                        const unsigned long long slot = slot0 + __popc(ma & ((1u << lane) - 1u));
                        if (slot < B.ring_cap)
                            rec = B.ring + slot * B.rec_bytes;
                        else
                            atomicAdd(&s_cnt[2], 1u);
                        redo = dr.rrmax * f.inv > kOutputRr;
                        if (redo) {
                            // a radius of the series range: outputs from rho_acc
                            emit_accepted<KMAX, UNIF>(P, idx, (uint32_t)p, k0, k1, s_sig, s_act, s_hist, s_exc, s_q,
                                                      s_spec, rec);
                        } else {
                            const float u0 = sc.u0s * dr.u0raw * f.inv;
                            tally_accepted(u0, sc.ha, sc.hb, sc.ea, s_hist, s_exc, s_q);
                            if (rec) write_header(rec, idx, (uint32_t)p, 0u, sc.E0 * f.S, sc.h3s * f.T, u0, f.delta);
                        }
                    }
                    // Spectrum and projected state of the other accepted draws: each
                    // hands its (x | y) to its warp through shared memory (one
                    // straight run of vector stores), then the warp takes the draws
                    // one at a time, lane m mode m.  So the hot loop carries no
                    // unrolled per-mode tally or record stores (which, executed in a
                    // quarter of the iterations at 1 % acceptance, cost the loop its
                    // instruction cache), the atomics do not contend and the record
                    // writes are coalesced.
                    const bool coop = acc && !redo;
                    if (coop) {
                        float *xo = s_xfer + (size_t)tid * xfer_stride<KMAX>();
#pragma unroll
                        for (int m = 0; m < KMAX; m += 4) {
                            *reinterpret_cast<float4 *>(xo + m) = make_float4(dr.x[m], dr.x[m + 1], dr.x[m + 2], dr.x[m + 3]);
                            *reinterpret_cast<float4 *>(xo + KMAX + m) =
                                make_float4(dr.y[m], dr.y[m + 1], dr.y[m + 2], dr.y[m + 3]);
                        }
                    }
                    unsigned mq = __ballot_sync(0xffffffffu, coop);
                    __syncwarp();
                    while (mq) {
                        const int L = __ffs(mq) - 1;
                        mq &= mq - 1;
                        const float *xf = s_xfer + (size_t)((tid & ~31) + L) * xfer_stride<KMAX>();
                        const float inv = __shfl_sync(0xffffffffu, f.inv, L);
                        float *xh = reinterpret_cast<float *>(
                            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(rec), L));
                        const float sc2 = (inv * inv) * kSpecScale;
#pragma unroll
                        for (int m0 = 0; m0 < KMAX; m0 += 32) {
                            const int m = m0 + lane;
                            if (m < sc.K) {
                                const float x = xf[m], y = xf[KMAX + m];
                                atomicAdd(&s_spec[m], (unsigned long long)__float2ull_rn(fmaf(x, x, y * y) * sc2));
                                if (xh) {
                                    xh[8 + m] = x * inv;
                                    xh[8 + sc.K + m] = y * inv;
                                }
                            }
                        }
                    }
                    __syncwarp();  // the slabs are rewritten in the next iteration
                }
            } else {
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
                        if (dr.rrmax * f.inv > kOutputRr) {
                            // a radius of the series range: outputs from rho_acc
                            emit_accepted<KMAX, UNIF>(P, idx, (uint32_t)p, k0, k1, s_sig, s_act, s_hist, s_exc, s_q,
                                                      s_spec, rec);
                        } else {
                            const float u0 = sc.u0s * dr.u0raw * f.inv;
                            tally_accepted(u0, sc.ha, sc.hb, sc.ea, s_hist, s_exc, s_q);
                            tally_spectrum<KMAX>(s_spec, dr.x, dr.y, f.inv * f.inv, sc.K);
                            if (rec)
                                write_record<KMAX>(rec, idx, (uint32_t)p, 0u, sc.E0 * f.S, sc.h3s * f.T, u0, f.delta,
                                                   dr.x, dr.y, f.inv, sc.K);
                        }
                    }
                }
            }
        }

        // chunk done: flush this CTA's partials into the point's StatBlock
        uint32_t key = fkey(maxd);
        key = __reduce_max_sync(0xffffffffu, key);
        if (lane == 0 && maxd > -INFINITY) atomicMax(&s_maxd, key);
        if (SIR) {
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                float v = a_sir[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) atomicAdd(&s_sir[q], (double)v);
            }
        }
        __syncthreads();
        StatBlock *st = B.stats + p;
        if (SIR && tid < 7) {
            atomicAdd(&st->sir[tid], s_sir[tid]);
            s_sir[tid] = 0.0;
        }
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
}

// ---- SIR copy numbers in FP64 ---------------------------------------------
// P(N >= k) for N ~ Poisson(lambda), k >= 1: for lambda <= k + 1 the series
// lambda^k e^-lambda / k! * sum_i lambda^i k! / (k + i)! (all terms positive),
// otherwise 1 - e^-lambda sum_{j<k} lambda^j / j!.
static __device__ double poisson_tail_d(double lambda, int k) {
    if (!(lambda > 0.0)) return 0.0;
    if (lambda <= k + 1.0) {
        const double lead = exp(k * log(lambda) - lambda - lgamma(k + 1.0));
        double term = 1.0, sum = 1.0;
        for (int i = 1; i < 256; ++i) {
            term *= lambda / (double)(k + i);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        return lead * sum;
    }
    double p = exp(-lambda), s = p;
    for (int j = 1; j < k; ++j) {
        p *= lambda / (double)j;
        s += p;
    }
    return 1.0 - s;
}
constexpr int kMaxCopies = (1 << 24) - 1;  // copies fit the record's 24-bit field

// ---- FP64 decision of the guard-band proposals ---------------------------
template <int KMAX, bool UNIF>
__global__ void __launch_bounds__(128) k_refine(DevBufs B, uint32_t k0, uint32_t k1) {
    const uint32_t n = min(*(volatile uint32_t *)&B.counters[1], B.refine_cap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const RefineItem it = B.refine[i];
        const PointConst *P = B.pts + it.point;
        StatBlock *st = B.stats + it.point;
        Out64 o;
        float xh[2 * KMAX];
        eval64<KMAX, UNIF>(P, it.idx, k0, k1, &o, xh);
        atomicAdd(&st->n_refined, 1ull);
        atomicMax(&st->maxd_key, (unsigned long long)fkey((float)o.delta));
        unsigned long long copies = 1;
        if (B.sir) {
            // SIR: n = #{k >= 1 : U < P(N >= k)}, N ~ Poisson(c exp(delta))
            const double lam = P->sir_c * exp(o.delta);
            int n = 0;
            double tk = poisson_tail_d(lam, 1);
            while (n < kMaxCopies && o.u < tk) {
                ++n;
                tk = poisson_tail_d(lam, n + 1);
            }
            // near: U within 1e-6 (in log) of the tail value that decided n
            const double tn = n > 0 ? poisson_tail_d(lam, n) : 1.0;
            const bool near = fabs(o.lnU - log(tk)) < 1e-6 || (n > 0 && fabs(o.lnU - log(tn)) < 1e-6);
            o.near = near;
            if (near) atomicAdd(&st->n_near, 1ull);
            if (n == 0) continue;
            atomicAdd(&st->n_kept, 1ull);
            copies = (unsigned long long)n;
        } else {
            if (o.near) atomicAdd(&st->n_near, 1ull);
            if (o.delta > 0.0) atomicAdd(&st->n_viol, 1ull);
            if (!o.accept) continue;
        }
        atomicAdd(&st->n_acc, copies);
        const float u0 = o.u0;
        atomicAdd(&st->hist[hist_bin(u0, __ldg(&P->hist_a), __ldg(&P->hist_b))], copies);
        atomicAdd(&st->exc[exc_bin(u0, __ldg(&P->exc_a))], copies);
        const float u2 = u0 * u0;
        atomicAdd(&st->q[0], copies * (unsigned long long)__float2ll_rn(u0 * kQ1));
        atomicAdd(&st->q[1], copies * (unsigned long long)__float2ll_rn(u2 * kQ2));
        atomicAdd(&st->q[2], copies * (unsigned long long)__float2ll_rn(u2 * u0 * kQ3));
        atomicAdd(&st->q[3], copies * (unsigned long long)__float2ll_rn(u2 * u2 * kQ4));
        for (int m = 0; m < P->K; ++m)
            atomicAdd(&st->spec[m], copies * (unsigned long long)__float2ull_rn(
                                                 fmaf(xh[m], xh[m], xh[P->K + m] * xh[P->K + m]) * kSpecScale));
        const unsigned long long slot = atomicAdd(B.ring_count, 1ull);
        if (slot < B.ring_cap) {
            const int K = P->K;
            unsigned char *rec = B.ring + slot * B.rec_bytes;
            *reinterpret_cast<unsigned long long *>(rec) = it.idx;
            uint32_t *h = reinterpret_cast<uint32_t *>(rec + 8);
            h[0] = it.point;
            h[1] = 1u | (o.near ? 2u : 0u) | (B.sir ? (uint32_t)copies << 8 : 0u);
            float *f = reinterpret_cast<float *>(rec + 16);
            f[0] = o.H2;
            f[1] = o.H3;
            f[2] = o.u0;
            f[3] = (float)o.delta;
            for (int m = 0; m < 2 * K; ++m) f[4 + m] = xh[m];
        } else {
            atomicAdd(&st->n_dropped, 1ull);
        }
    }
}

// ---- replay: per-proposal outputs of listed indices -----------------------
// out row: [delta, lnU, accept, flags, H2, H3, u0, S, xhat(2K)]
template <int KMAX, bool UNIF>
__global__ void __launch_bounds__(128) k_replay(const PointConst *P, const unsigned long long *idx,
                                               unsigned long long n, uint32_t k0, uint32_t k1,
                                               double *out) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Scal sc = load_scal(P);
    const int K = sc.K;
    const unsigned long long id = idx[i];
    const uint32_t lo = (uint32_t)id, hi = (uint32_t)(id >> 32);
    Draw<KMAX> dr;
    draw_fast<KMAX, UNIF>(dr, P->sigma, P->act, lo, hi, sc.pid, k0, k1);
    const uint32_t wa = accept_word(lo, hi, sc.pid, K, k0, k1);
    const Fast f = eval_fast<KMAX, UNIF>(dr, sc, wa);
    double *row = out + i * (unsigned long long)(8 + 2 * K);
    if (fabsf(f.d) < f.guard || min(dr.wmin, wa) < kTailBucket) {
        Out64 o;
        float xh[2 * KMAX];
        eval64<KMAX, UNIF>(P, id, k0, k1, &o, xh);
        row[0] = o.delta;
        row[1] = o.lnU;
        row[2] = o.accept;
        row[3] = 1.0 + (o.near ? 2.0 : 0.0);
        row[4] = o.H2;
        row[5] = o.H3;
        row[6] = o.u0;
        row[7] = o.S;
        for (int m = 0; m < 2 * K; ++m) row[8 + m] = xh[m];
        return;
    }
    row[2] = f.d < 0.f ? 1.0 : 0.0;
    row[3] = 0.0;
    if (dr.rrmax * f.inv > kOutputRr) {
        // a radius of the series range: the values are those of rho_acc, as
        // the sampler's outputs of an accepted draw would be
        draw_fast<KMAX, UNIF, true>(dr, P->sigma, P->act, lo, hi, sc.pid, k0, k1);
    }
    const float inv2 = rcp_rn(dr.nrm2);
    const float inv = rsqrt_approx(dr.nrm2);
    const float S = dr.Sraw * inv2;
    const float T = triad2<KMAX>(dr.x, dr.y) * (inv2 * inv);
    const float tQ = UNIF ? 0.f : sc.cQ * logf(dr.zz * inv2);
    row[0] = ((sc.cS * S + sc.cH * T) + tQ) - sc.logM;
    row[1] = f.lnU;
    row[4] = sc.E0 * S;
    row[5] = sc.h3s * T;
    row[6] = sc.u0s * dr.u0raw * inv;
    row[7] = S;
#pragma unroll
    for (int m = 0; m < KMAX; ++m) {
        if (m < K) {
            row[8 + m] = dr.x[m] * inv;
            row[8 + K + m] = dr.y[m] * inv;
        }
    }
}

// Kernel table of one KMAX, in two halves that separate translation units
// can instantiate (the 64-mode kernels take long to compile): the launch
// variants with the accept hand-off, the SIR form, the FP64 pass and replay;
// and the variants with the per-lane accept path.
template <int KMAX>
void fill_triad_kernels_lane(TriadKernels *t) {
    t->main[0][3] = (const void *)k_sample_triad<KMAX, false, 128, 1, false, false>;
    t->main[0][4] = (const void *)k_sample_triad<KMAX, false, 256, 1, false, false>;
    t->main[0][5] = (const void *)k_sample_triad<KMAX, false, 256, 2, false, false>;
    t->main[1][3] = (const void *)k_sample_triad<KMAX, true, 128, 1, false, false>;
    t->main[1][4] = (const void *)k_sample_triad<KMAX, true, 256, 1, false, false>;
    t->main[1][5] = (const void *)k_sample_triad<KMAX, true, 256, 2, false, false>;
}

template <int KMAX>
void fill_triad_kernels_xfer(TriadKernels *t) {
    t->main[0][0] = (const void *)k_sample_triad<KMAX, false, 128, 1>;
    t->main[0][1] = (const void *)k_sample_triad<KMAX, false, 256, 1>;
    t->main[0][2] = (const void *)k_sample_triad<KMAX, false, 256, 2>;
    t->main[1][0] = (const void *)k_sample_triad<KMAX, true, 128, 1>;
    t->main[1][1] = (const void *)k_sample_triad<KMAX, true, 256, 1>;
    t->main[1][2] = (const void *)k_sample_triad<KMAX, true, 256, 2>;
    t->n_variants = 6;
    t->sir[0] = (const void *)k_sample_triad<KMAX, false, 256, 1, true, false>;
    t->sir[1] = (const void *)k_sample_triad<KMAX, true, 256, 1, true, false>;
    t->refine[0] = (const void *)k_refine<KMAX, false>;
    t->refine[1] = (const void *)k_refine<KMAX, true>;
    t->replay[0] = (const void *)k_replay<KMAX, false>;
    t->replay[1] = (const void *)k_replay<KMAX, true>;
    t->replay_per_block = 128;
    t->xfer_bytes_per_thread = (int)(xfer_stride<KMAX>() * sizeof(float));
}

template <int KMAX>
void fill_triad_kernels(TriadKernels *t) {
    fill_triad_kernels_xfer<KMAX>(t);
    fill_triad_kernels_lane<KMAX>(t);
}

}  // namespace tkdv

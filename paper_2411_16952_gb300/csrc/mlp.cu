// mlp.cu - the learned proposal: a 4 -> 64 -> 64 -> 64 MLP that maps a
// parameter point (K, E0, beta', C3/C2) to per-mode log-variance corrections
// c_k of the paper's proposal, sigma_k'^2 = sigma_k^2 e^{c_k}.
//
// The proposal stays a projected centred Gaussian, so its density against the
// uniform measure keeps the closed form of Eqs. (33)-(38):
//   g(xh) = prod_k w'_k Q^-K,  w'_k = 1/sigma_k'^2,  Q = sum_k w'_k s_k,
// and the accept test of Eq. (40) stays exact with K ln Q and a recomputed
// envelope M.  Training minimises, per point and over accepted samples i
// (draws from f), the tempered negative log-likelihood
//   J_tau = tau log mean_i exp((z_i + ell_i)/tau),  ell_i = K ln Q_i - sum ln w'_k,
// with z_i = -beta H_i (tau = inf: the plain mean, i.e. KL(f || g) + const);
// small tau weights the draws with the largest f/g, which set the acceptance.
//
// Parameters are held as FP32 masters (Adam) and used as BF16 copies in every
// forward and backward pass; all sums accumulate in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/tkdv.h"
#include "tkdv_internal.h"

namespace tkdv {
namespace mlpk {

constexpr int H = 64, KO = 64, NIN = 4;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * NIN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + KO * H, NPARAM = OFF_B3 + KO;
static_assert(NPARAM == TKDV_MLP_NPARAM, "parameter count");

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, int i) { return __bfloat162float(w[i]); }

// Forward pass of P points, one CTA of 64 threads per point.
__global__ void __launch_bounds__(64) k_forward(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ feats,
                                                float *h1, float *h2, float *out) {
    const int p = blockIdx.x, j = threadIdx.x;
    __shared__ float sf[NIN], s1[H], s2[H];
    if (j < NIN) sf[j] = feats[p * NIN + j];
    __syncthreads();
    float a = bf(w, OFF_B1 + j);
#pragma unroll
    for (int i = 0; i < NIN; ++i) a = fmaf(bf(w, OFF_W1 + j * NIN + i), sf[i], a);
    const float t1 = tanhf(a);
    s1[j] = t1;
    h1[p * H + j] = t1;
    __syncthreads();
    a = bf(w, OFF_B2 + j);
    for (int i = 0; i < H; ++i) a = fmaf(bf(w, OFF_W2 + j * H + i), s1[i], a);
    const float t2 = tanhf(a);
    s2[j] = t2;
    h2[p * H + j] = t2;
    __syncthreads();
    a = bf(w, OFF_B3 + j);
    for (int i = 0; i < H; ++i) a = fmaf(bf(w, OFF_W3 + j * H + i), s2[i], a);
    out[p * KO + j] = a;
}

// Per point: gauge-fixed c (mean zero over k < K), w'_k = w_k e^{-c_k},
// and the constant sum_k ln w'_k.  One CTA of 64 threads per point.
__global__ void __launch_bounds__(64) k_prepare(const float *__restrict__ out, const int *__restrict__ Ks,
                                                const float *__restrict__ wpaper, float *wprime, float *sumlogw) {
    const int p = blockIdx.x, k = threadIdx.x, K = Ks[p];
    __shared__ float red[64];
    const float o = k < K ? out[p * KO + k] : 0.f;
    red[k] = o;
    __syncthreads();
    for (int s = 32; s > 0; s >>= 1) {
        if (k < s) red[k] += red[k + s];
        __syncthreads();
    }
    const float mean = red[0] / (float)K;
    __syncthreads();
    const float c = o - mean;
    const float wv = k < K ? wpaper[p * KO + k] * expf(-c) : 0.f;
    wprime[p * KO + k] = wv;
    red[k] = k < K ? logf(wv) : 0.f;
    __syncthreads();
    for (int s = 32; s > 0; s >>= 1) {
        if (k < s) red[k] += red[k + s];
        __syncthreads();
    }
    if (k == 0) sumlogw[p] = red[0];
}

// Loss partials: grid (nblk, P), 256 threads; each thread streams its samples
// (rows of `stride` floats: s_1..s_K) and keeps an online log-sum-exp of
// a_i = (z_i + ell_i)/tau with the weighted sums V_k = sum e^{a_i - m} s_ik/Q_i,
// S = sum e^{a_i - m}, L = sum e^{a_i - m} ell_i.  tau <= 0 means tau = inf
// (a_i = 0).  Partials per block: [m, S, L, V_1..V_K] (stride KO + 3).
template <int KMAXL>
__global__ void __launch_bounds__(256) k_loss_partial(const float *__restrict__ s, const float *__restrict__ z,
                                                      const unsigned long long *__restrict__ row0,
                                                      const unsigned long long *__restrict__ nrows,
                                                      const int *__restrict__ Ks, const float *__restrict__ wprime,
                                                      const float *__restrict__ sumlogw, int stride, float tau,
                                                      float *partial) {
    const int p = blockIdx.y, K = Ks[p];
    const unsigned long long n = nrows[p], base = row0[p];
    float w[KMAXL], V[KMAXL];
#pragma unroll
    for (int k = 0; k < KMAXL; ++k) {
        w[k] = k < K ? wprime[p * KO + k] : 0.f;
        V[k] = 0.f;
    }
    const float slw = sumlogw[p];
    float m = -INFINITY, S = 0.f, L = 0.f;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float *row = s + (base + i) * (unsigned long long)stride;
        float sk[KMAXL];
#pragma unroll
        for (int k = 0; k < KMAXL; k += 4) {
            if (k < stride) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(row + k));
                sk[k] = v.x;
                if (k + 1 < KMAXL) sk[k + 1] = v.y;
                if (k + 2 < KMAXL) sk[k + 2] = v.z;
                if (k + 3 < KMAXL) sk[k + 3] = v.w;
            } else {
                sk[k] = 0.f;
                if (k + 1 < KMAXL) sk[k + 1] = 0.f;
                if (k + 2 < KMAXL) sk[k + 2] = 0.f;
                if (k + 3 < KMAXL) sk[k + 3] = 0.f;
            }
        }
        float Q = 0.f;
#pragma unroll
        for (int k = 0; k < KMAXL; ++k) Q = fmaf(w[k], sk[k], Q);
        const float ell = (float)K * logf(Q) - slw;
        const float a = tau > 0.f ? (__ldg(z + base + i) + ell) / tau : 0.f;
        float scale = 1.f, e = 1.f;
        if (a > m) {
            scale = expf(m - a);  // 0 on the first sample
            m = a;
        } else {
            e = expf(a - m);
        }
        S = S * scale + e;
        L = L * scale + e * ell;
        const float eq = e / Q;
#pragma unroll
        for (int k = 0; k < KMAXL; ++k) V[k] = fmaf(eq, sk[k], V[k] * scale);
    }
    // block reduction of (m, S, L, V) by log-sum-exp merging through shared memory
    __shared__ float sm[256];
    __shared__ float sv[256];
    const int t = threadIdx.x;
    sm[t] = m;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
        if (t < s2) sm[t] = fmaxf(sm[t], sm[t + s2]);
        __syncthreads();
    }
    const float M = sm[0];
    __syncthreads();
    const float f = (m == -INFINITY) ? 0.f : expf(m - M);
    float *out = partial + ((size_t)p * gridDim.x + blockIdx.x) * (KO + 3);
    auto block_sum = [&](float v) -> float {
        sv[t] = v;
        __syncthreads();
        for (int s2 = 128; s2 > 0; s2 >>= 1) {
            if (t < s2) sv[t] += sv[t + s2];
            __syncthreads();
        }
        const float r = sv[0];
        __syncthreads();
        return r;
    };
    const float Sb = block_sum(S * f);
    const float Lb = block_sum(L * f);
    if (t == 0) {
        out[0] = M;
        out[1] = Sb;
        out[2] = Lb;
    }
#pragma unroll
    for (int k = 0; k < KMAXL; ++k) {
        const float Vb = block_sum(V[k] * f);
        if (t == 0) out[3 + k] = Vb;
    }
    if (t == 0)
        for (int k = KMAXL; k < KO; ++k) out[3 + k] = 0.f;
}

// Merge the partials of each point: loss J_p and dJ/dc_raw (through the gauge).
__global__ void __launch_bounds__(64) k_loss_merge(const float *__restrict__ partial, int nblk,
                                                   const unsigned long long *__restrict__ nrows,
                                                   const int *__restrict__ Ks, const float *__restrict__ wprime,
                                                   float tau, float *dout, float *loss) {
    const int p = blockIdx.x, k = threadIdx.x, K = Ks[p];
    const float *pp = partial + (size_t)p * nblk * (KO + 3);
    float M = -INFINITY;
    for (int b = 0; b < nblk; ++b) M = fmaxf(M, pp[b * (KO + 3)]);
    float S = 0.f, L = 0.f, V = 0.f;
    for (int b = 0; b < nblk; ++b) {
        const float mb = pp[b * (KO + 3)];
        const float f = (mb == -INFINITY) ? 0.f : expf(mb - M);
        S += f * pp[b * (KO + 3) + 1];
        L += f * pp[b * (KO + 3) + 2];
        if (k < KO) V += f * pp[b * (KO + 3) + 3 + k];
    }
    // dJ/dc_k = 1 - K w'_k V_k / S   (k < K); zero mean over k < K already
    __shared__ float g[64], red[64];
    const float gk = k < K ? 1.f - (float)K * wprime[p * KO + k] * V / S : 0.f;
    g[k] = gk;
    red[k] = gk;
    __syncthreads();
    for (int s2 = 32; s2 > 0; s2 >>= 1) {
        if (k < s2) red[k] += red[k + s2];
        __syncthreads();
    }
    const float mean = red[0] / (float)K;
    dout[p * KO + k] = k < K ? g[k] - mean : 0.f;
    if (k == 0) {
        const double n = (double)nrows[p];
        loss[p] = tau > 0.f ? (float)((double)tau * ((double)M + log((double)S / n))) : L / S;
    }
}

// Backward pass through the MLP for all points; one CTA of 256 threads.
// grad (NPARAM floats) receives the sum over points.
__global__ void __launch_bounds__(256) k_backward(const __nv_bfloat16 *__restrict__ w, const float *__restrict__ feats,
                                                  const float *__restrict__ h1, const float *__restrict__ h2,
                                                  const float *__restrict__ dout, int P, float *da2, float *da1,
                                                  float *grad) {
    const int t = threadIdx.x;
    // da2[p][i] = (sum_j dout[p][j] W3[j][i]) (1 - h2^2)
    for (int e = t; e < P * H; e += blockDim.x) {
        const int p = e / H, i = e % H;
        float a = 0.f;
        for (int j = 0; j < KO; ++j) a = fmaf(dout[p * KO + j], bf(w, OFF_W3 + j * H + i), a);
        const float hv = h2[p * H + i];
        da2[e] = a * (1.f - hv * hv);
    }
    __syncthreads();
    for (int e = t; e < P * H; e += blockDim.x) {
        const int p = e / H, i = e % H;
        float a = 0.f;
        for (int j = 0; j < H; ++j) a = fmaf(da2[p * H + j], bf(w, OFF_W2 + j * H + i), a);
        const float hv = h1[p * H + i];
        da1[e] = a * (1.f - hv * hv);
    }
    __syncthreads();
    for (int e = t; e < KO * H; e += blockDim.x) {  // dW3[j][i] = sum_p dout[p][j] h2[p][i]
        const int j = e / H, i = e % H;
        float a = 0.f;
        for (int p = 0; p < P; ++p) a = fmaf(dout[p * KO + j], h2[p * H + i], a);
        grad[OFF_W3 + e] = a;
    }
    for (int j = t; j < KO; j += blockDim.x) {
        float a = 0.f;
        for (int p = 0; p < P; ++p) a += dout[p * KO + j];
        grad[OFF_B3 + j] = a;
    }
    for (int e = t; e < H * H; e += blockDim.x) {
        const int j = e / H, i = e % H;
        float a = 0.f;
        for (int p = 0; p < P; ++p) a = fmaf(da2[p * H + j], h1[p * H + i], a);
        grad[OFF_W2 + e] = a;
    }
    for (int j = t; j < H; j += blockDim.x) {
        float a = 0.f, b = 0.f;
        for (int p = 0; p < P; ++p) {
            a += da2[p * H + j];
            b += da1[p * H + j];
        }
        grad[OFF_B2 + j] = a;
        grad[OFF_B1 + j] = b;
    }
    for (int e = t; e < H * NIN; e += blockDim.x) {
        const int j = e / NIN, i = e % NIN;
        float a = 0.f;
        for (int p = 0; p < P; ++p) a = fmaf(da1[p * H + j], feats[p * NIN + i], a);
        grad[OFF_W1 + e] = a;
    }
}

// Adam on the FP32 masters; refreshes the BF16 copies.
__global__ void k_adam(float *master, float *m1, float *m2, const float *grad, __nv_bfloat16 *wb, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float g = grad[i];
    const float a = b1 * m1[i] + (1.f - b1) * g;
    const float b = b2 * m2[i] + (1.f - b2) * g * g;
    m1[i] = a;
    m2[i] = b;
    const float v = master[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    master[i] = v;
    wb[i] = __float2bfloat16_rn(v);
}

__global__ void k_to_bf16(const float *master, __nv_bfloat16 *wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NPARAM) wb[i] = __float2bfloat16_rn(master[i]);
}

// Training rows from the sampler's accepted records: s_k = xh_k^2 + xh_{K+k}^2
// and z = -beta H = -beta'/(E0 K^2) (H2 - r H3), scattered per point.
__global__ void k_records_to_rows(const unsigned char *__restrict__ ring, unsigned long long nrec, int rec_bytes,
                                  int K, int stride, const unsigned long long *__restrict__ row0,
                                  const unsigned long long *__restrict__ cap, unsigned long long *fill,
                                  const float *__restrict__ zcoef /* per point: beta'/(E0 K^2), r */, float *s,
                                  float *z) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrec) return;
    const unsigned char *rec = ring + i * (unsigned long long)rec_bytes;
    const uint32_t p = *reinterpret_cast<const uint32_t *>(rec + 8);
    const unsigned long long slot = atomicAdd(&fill[p], 1ull);
    if (slot >= cap[p]) return;
    const float *f = reinterpret_cast<const float *>(rec + 16);
    const float *xh = f + 4;
    float *row = s + (row0[p] + slot) * (unsigned long long)stride;
    for (int k = 0; k < stride; ++k) row[k] = k < K ? xh[k] * xh[k] + xh[K + k] * xh[K + k] : 0.f;
    z[row0[p] + slot] = -zcoef[2 * p] * (f[0] - zcoef[2 * p + 1] * f[1]);
}

}  // namespace mlpk
}  // namespace tkdv

using namespace tkdv;
using namespace tkdv::mlpk;

struct tkdv_mlp {
    float *d_master = nullptr, *d_m1 = nullptr, *d_m2 = nullptr, *d_grad = nullptr;
    __nv_bfloat16 *d_wb = nullptr;
    // training set
    int P = 0, stride = 4, kmax = 4;
    std::vector<int> K;
    float *d_feats = nullptr, *d_wpaper = nullptr, *d_s = nullptr, *d_z = nullptr;
    unsigned long long *d_row0 = nullptr, *d_nrows = nullptr;
    std::vector<unsigned long long> nrows;
    int *d_K = nullptr;
    // work buffers
    float *d_h1 = nullptr, *d_h2 = nullptr, *d_out = nullptr, *d_wprime = nullptr, *d_slw = nullptr,
          *d_partial = nullptr, *d_dout = nullptr, *d_loss = nullptr, *d_da1 = nullptr, *d_da2 = nullptr;
    int nblk = 0;
    int step = 0;
    std::string err;
};

namespace {

int mfail(tkdv_mlp *m, int code, const std::string &msg) {
    if (m) m->err = msg;
    return code;
}

#define MCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return mfail(m, e_ == cudaErrorMemoryAllocation ? TKDV_ERR_OOM : TKDV_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));          \
    } while (0)

void free_set(tkdv_mlp *m) {
    for (void *p : {(void *)m->d_feats, (void *)m->d_wpaper, (void *)m->d_s, (void *)m->d_z, (void *)m->d_row0,
                    (void *)m->d_nrows, (void *)m->d_K, (void *)m->d_h1, (void *)m->d_h2, (void *)m->d_out,
                    (void *)m->d_wprime, (void *)m->d_slw, (void *)m->d_partial, (void *)m->d_dout,
                    (void *)m->d_loss, (void *)m->d_da1, (void *)m->d_da2})
        if (p) cudaFree(p);
    m->d_feats = m->d_wpaper = m->d_s = m->d_z = nullptr;
    m->d_row0 = m->d_nrows = nullptr;
    m->d_K = nullptr;
    m->d_h1 = m->d_h2 = m->d_out = m->d_wprime = m->d_slw = m->d_partial = m->d_dout = m->d_loss = m->d_da1 =
        m->d_da2 = nullptr;
    m->P = 0;
}

// Work buffers for P points.
int alloc_work(tkdv_mlp *m, int P) {
    m->nblk = 64;
    MCK(cudaMalloc(&m->d_h1, sizeof(float) * P * H));
    MCK(cudaMalloc(&m->d_h2, sizeof(float) * P * H));
    MCK(cudaMalloc(&m->d_out, sizeof(float) * P * KO));
    MCK(cudaMalloc(&m->d_wprime, sizeof(float) * P * KO));
    MCK(cudaMalloc(&m->d_slw, sizeof(float) * P));
    MCK(cudaMalloc(&m->d_partial, sizeof(float) * P * m->nblk * (KO + 3)));
    MCK(cudaMalloc(&m->d_dout, sizeof(float) * P * KO));
    MCK(cudaMalloc(&m->d_loss, sizeof(float) * P));
    MCK(cudaMalloc(&m->d_da1, sizeof(float) * P * H));
    MCK(cudaMalloc(&m->d_da2, sizeof(float) * P * H));
    return TKDV_OK;
}

const void *partial_kernel(int kmax) {
    if (kmax <= 16) return (const void *)k_loss_partial<16>;
    if (kmax <= 32) return (const void *)k_loss_partial<32>;
    return (const void *)k_loss_partial<64>;
}

}  // namespace

extern "C" {

int tkdv_mlp_features(int K, double beta_p, double E0, double r, double *out4) {
    if (!out4 || K < 1 || K > 64 || !(E0 > 0)) return TKDV_ERR_INVALID_ARG;
    const double lam = beta_p * r;
    out4[0] = std::log(std::max(beta_p, 1e-3)) / std::log(100.0);
    out4[1] = std::log(E0);
    out4[2] = std::log1p(std::max(lam, 0.0) / 100.0) / std::log(100.0);
    out4[3] = K / 64.0;
    return TKDV_OK;
}

int tkdv_mlp_create(uint64_t seed, tkdv_mlp **out) {
    if (!out) return TKDV_ERR_INVALID_ARG;
    *out = nullptr;
    tkdv_mlp *m = new tkdv_mlp();
    std::vector<float> w(NPARAM, 0.f);
    std::mt19937_64 gen(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int i = 0; i < H * NIN; ++i) w[OFF_W1 + i] = 0.3f * nd(gen);
    for (int i = 0; i < H * H; ++i) w[OFF_W2 + i] = 0.15f * nd(gen);  // W3, biases: zero (c = 0 at start)
    auto bail = [&](int rc) {
        tkdv_mlp_destroy(m);
        return rc;
    };
    int rc;
    if ((rc = cudaMalloc(&m->d_master, 4 * NPARAM)) || (rc = cudaMalloc(&m->d_m1, 4 * NPARAM)) ||
        (rc = cudaMalloc(&m->d_m2, 4 * NPARAM)) || (rc = cudaMalloc(&m->d_grad, 4 * NPARAM)) ||
        (rc = cudaMalloc(&m->d_wb, 2 * NPARAM)))
        return bail(rc == cudaErrorMemoryAllocation ? TKDV_ERR_OOM : TKDV_ERR_CUDA);
    cudaError_t e = cudaMemcpy(m->d_master, w.data(), 4 * NPARAM, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_m1, 0, 4 * NPARAM);
    if (e == cudaSuccess) e = cudaMemset(m->d_m2, 0, 4 * NPARAM);
    if (e == cudaSuccess) {
        k_to_bf16<<<(NPARAM + 255) / 256, 256>>>(m->d_master, m->d_wb);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) return bail(TKDV_ERR_CUDA);
    *out = m;
    return TKDV_OK;
}

void tkdv_mlp_destroy(tkdv_mlp *m) {
    if (!m) return;
    free_set(m);
    for (void *p : {(void *)m->d_master, (void *)m->d_m1, (void *)m->d_m2, (void *)m->d_grad, (void *)m->d_wb})
        if (p) cudaFree(p);
    delete m;
}

const char *tkdv_mlp_last_error(const tkdv_mlp *m) { return m ? m->err.c_str() : ""; }

int tkdv_mlp_get_params(tkdv_mlp *m, float *master, float *bf16_values) {
    if (!m) return TKDV_ERR_INVALID_ARG;
    if (master) MCK(cudaMemcpy(master, m->d_master, 4 * NPARAM, cudaMemcpyDeviceToHost));
    if (bf16_values) {
        std::vector<uint16_t> b(NPARAM);
        MCK(cudaMemcpy(b.data(), m->d_wb, 2 * NPARAM, cudaMemcpyDeviceToHost));
        for (int i = 0; i < NPARAM; ++i) {
            const uint32_t u = (uint32_t)b[i] << 16;
            std::memcpy(&bf16_values[i], &u, 4);
        }
    }
    return TKDV_OK;
}

int tkdv_mlp_set_params(tkdv_mlp *m, const float *master) {
    if (!m || !master) return TKDV_ERR_INVALID_ARG;
    MCK(cudaMemcpy(m->d_master, master, 4 * NPARAM, cudaMemcpyHostToDevice));
    MCK(cudaMemset(m->d_m1, 0, 4 * NPARAM));
    MCK(cudaMemset(m->d_m2, 0, 4 * NPARAM));
    m->step = 0;
    k_to_bf16<<<(NPARAM + 255) / 256, 256>>>(m->d_master, m->d_wb);
    MCK(cudaDeviceSynchronize());
    return TKDV_OK;
}

int tkdv_mlp_infer(tkdv_mlp *m, int P, const double *feats, const int *K, double *c_out) {
    if (!m || P < 1 || P > TKDV_MAX_POINTS || !feats || !K || !c_out) return TKDV_ERR_INVALID_ARG;
    for (int p = 0; p < P; ++p)
        if (K[p] < 1 || K[p] > 64) return mfail(m, TKDV_ERR_INVALID_ARG, "K must be in 1..64");
    std::vector<float> f(P * NIN);
    for (int i = 0; i < P * NIN; ++i) f[i] = (float)feats[i];
    float *d_f = nullptr, *d_h = nullptr, *d_o = nullptr;
    MCK(cudaMalloc(&d_f, 4 * P * NIN));
    cudaError_t e = cudaMalloc(&d_h, 4 * P * H * 2);
    if (e == cudaSuccess) e = cudaMalloc(&d_o, 4 * P * KO);
    if (e == cudaSuccess) e = cudaMemcpy(d_f, f.data(), 4 * P * NIN, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_forward<<<P, 64>>>(m->d_wb, d_f, d_h, d_h + P * H, d_o);
        e = cudaDeviceSynchronize();
    }
    std::vector<float> o(P * KO);
    if (e == cudaSuccess) e = cudaMemcpy(o.data(), d_o, 4 * P * KO, cudaMemcpyDeviceToHost);
    cudaFree(d_f);
    cudaFree(d_h);
    cudaFree(d_o);
    if (e != cudaSuccess) return mfail(m, TKDV_ERR_CUDA, std::string("infer: ") + cudaGetErrorString(e));
    for (int p = 0; p < P; ++p) {
        double mean = 0;
        for (int k = 0; k < K[p]; ++k) mean += o[p * KO + k];
        mean /= K[p];
        for (int k = 0; k < KO; ++k) c_out[p * KO + k] = k < K[p] ? (double)o[p * KO + k] - mean : 0.0;
    }
    return TKDV_OK;
}

int tkdv_mlp_set_data(tkdv_mlp *m, int P, const int *K, const double *feats, const double *w_paper,
                      const uint64_t *counts, const float *s_rows, const float *z) {
    if (!m || P < 1 || P > TKDV_MAX_POINTS || !K || !feats || !w_paper || !counts || !s_rows)
        return TKDV_ERR_INVALID_ARG;
    free_set(m);
    m->P = P;
    m->K.assign(K, K + P);
    m->kmax = 1;
    for (int p = 0; p < P; ++p) {
        if (K[p] < 1 || K[p] > 64) return mfail(m, TKDV_ERR_INVALID_ARG, "K must be in 1..64");
        m->kmax = std::max(m->kmax, K[p]);
    }
    m->stride = (m->kmax + 3) / 4 * 4;
    m->nrows.assign(counts, counts + P);
    std::vector<unsigned long long> row0(P, 0);
    unsigned long long tot = 0;
    for (int p = 0; p < P; ++p) {
        row0[p] = tot;
        tot += counts[p];
        if (counts[p] == 0) return mfail(m, TKDV_ERR_INVALID_ARG, "every point needs samples");
    }
    std::vector<float> f(P * NIN), wp(P * KO, 0.f);
    for (int i = 0; i < P * NIN; ++i) f[i] = (float)feats[i];
    for (int p = 0; p < P; ++p)
        for (int k = 0; k < K[p]; ++k) wp[p * KO + k] = (float)w_paper[p * KO + k];
    std::vector<float> zz(tot, 0.f);
    if (z) std::memcpy(zz.data(), z, 4 * tot);
    MCK(cudaMalloc(&m->d_feats, 4 * P * NIN));
    MCK(cudaMalloc(&m->d_wpaper, 4 * P * KO));
    MCK(cudaMalloc(&m->d_s, 4 * tot * m->stride));
    MCK(cudaMalloc(&m->d_z, 4 * tot));
    MCK(cudaMalloc(&m->d_row0, 8 * P));
    MCK(cudaMalloc(&m->d_nrows, 8 * P));
    MCK(cudaMalloc(&m->d_K, 4 * P));
    MCK(cudaMemcpy(m->d_feats, f.data(), 4 * P * NIN, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->d_wpaper, wp.data(), 4 * P * KO, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->d_s, s_rows, 4 * tot * m->stride, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->d_z, zz.data(), 4 * tot, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->d_row0, row0.data(), 8 * P, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->d_nrows, m->nrows.data(), 8 * P, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->d_K, m->K.data(), 4 * P, cudaMemcpyHostToDevice));
    return alloc_work(m, P);
}

int tkdv_mlp_set_data_records(tkdv_mlp *m, int P, const int *K, const double *feats, const double *w_paper,
                              const double *zcoef, const void *records_dev, uint64_t n_records, int K_records,
                              uint64_t max_per_point) {
    if (!m || P < 1 || P > TKDV_MAX_POINTS || !K || !feats || !w_paper || !zcoef || (!records_dev && n_records) ||
        max_per_point == 0 || K_records < 1 || K_records > 64)
        return TKDV_ERR_INVALID_ARG;
    for (int p = 0; p < P; ++p)
        if (K[p] != K_records) return mfail(m, TKDV_ERR_INVALID_ARG, "all points must have the records' K");
    free_set(m);
    m->P = P;
    m->K.assign(K, K + P);
    m->kmax = K_records;
    m->stride = (K_records + 3) / 4 * 4;
    std::vector<unsigned long long> row0(P), cap(P, max_per_point);
    for (int p = 0; p < P; ++p) row0[p] = (unsigned long long)p * max_per_point;
    const unsigned long long tot = (unsigned long long)P * max_per_point;
    std::vector<float> f(P * NIN), wp(P * KO, 0.f), zc(2 * P);
    for (int i = 0; i < P * NIN; ++i) f[i] = (float)feats[i];
    for (int p = 0; p < P; ++p) {
        for (int k = 0; k < K[p]; ++k) wp[p * KO + k] = (float)w_paper[p * KO + k];
        zc[2 * p] = (float)zcoef[2 * p];
        zc[2 * p + 1] = (float)zcoef[2 * p + 1];
    }
    unsigned long long *d_cap = nullptr, *d_fill = nullptr;
    float *d_zc = nullptr;
    MCK(cudaMalloc(&m->d_feats, 4 * P * NIN));
    MCK(cudaMalloc(&m->d_wpaper, 4 * P * KO));
    MCK(cudaMalloc(&m->d_s, 4 * tot * m->stride));
    MCK(cudaMalloc(&m->d_z, 4 * tot));
    MCK(cudaMalloc(&m->d_row0, 8 * P));
    MCK(cudaMalloc(&m->d_nrows, 8 * P));
    MCK(cudaMalloc(&m->d_K, 4 * P));
    MCK(cudaMalloc(&d_cap, 8 * P));
    MCK(cudaMalloc(&d_fill, 8 * P));
    MCK(cudaMalloc(&d_zc, 4 * 2 * P));
    MCK(cudaMemcpy(m->d_feats, f.data(), 4 * P * NIN, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->d_wpaper, wp.data(), 4 * P * KO, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->d_row0, row0.data(), 8 * P, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(m->d_K, m->K.data(), 4 * P, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(d_cap, cap.data(), 8 * P, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(d_zc, zc.data(), 8 * P, cudaMemcpyHostToDevice));
    MCK(cudaMemset(d_fill, 0, 8 * P));
    if (n_records) {
        const int rb = (int)record_bytes(K_records);
        k_records_to_rows<<<(unsigned)((n_records + 255) / 256), 256>>>((const unsigned char *)records_dev, n_records,
                                                                        rb, K_records, m->stride, m->d_row0, d_cap,
                                                                        d_fill, d_zc, m->d_s, m->d_z);
    }
    std::vector<unsigned long long> fill(P);
    MCK(cudaMemcpy(fill.data(), d_fill, 8 * P, cudaMemcpyDeviceToHost));
    cudaFree(d_cap);
    cudaFree(d_fill);
    cudaFree(d_zc);
    m->nrows.resize(P);
    for (int p = 0; p < P; ++p) {
        m->nrows[p] = std::min<unsigned long long>(fill[p], max_per_point);
        if (m->nrows[p] == 0) return mfail(m, TKDV_ERR_INVALID_ARG, "a point has no accepted records");
    }
    MCK(cudaMemcpy(m->d_nrows, m->nrows.data(), 8 * P, cudaMemcpyHostToDevice));
    return alloc_work(m, P);
}

int tkdv_mlp_rows(tkdv_mlp *m, uint64_t *counts) {
    if (!m || !counts) return TKDV_ERR_INVALID_ARG;
    for (int p = 0; p < m->P; ++p) counts[p] = m->nrows[p];
    return TKDV_OK;
}

int tkdv_mlp_step(tkdv_mlp *m, float lr, float tau, int update, double *loss, float *grad_out) {
    if (!m || m->P < 1) return TKDV_ERR_INVALID_ARG;
    const int P = m->P;
    k_forward<<<P, 64>>>(m->d_wb, m->d_feats, m->d_h1, m->d_h2, m->d_out);
    k_prepare<<<P, 64>>>(m->d_out, m->d_K, m->d_wpaper, m->d_wprime, m->d_slw);
    {
        const void *fn = partial_kernel(m->kmax);
        const float *s = m->d_s, *z = m->d_z, *wpr = m->d_wprime, *slw = m->d_slw;
        const unsigned long long *r0 = m->d_row0, *nr = m->d_nrows;
        const int *Kd = m->d_K;
        int stride = m->stride;
        float t = tau;
        float *part = m->d_partial;
        void *args[] = {&s, &z, &r0, &nr, &Kd, &wpr, &slw, &stride, &t, &part};
        MCK(cudaLaunchKernel(fn, dim3(m->nblk, P), dim3(256), args, 0, 0));
    }
    k_loss_merge<<<P, 64>>>(m->d_partial, m->nblk, m->d_nrows, m->d_K, m->d_wprime, tau, m->d_dout, m->d_loss);
    k_backward<<<1, 256>>>(m->d_wb, m->d_feats, m->d_h1, m->d_h2, m->d_dout, P, m->d_da2, m->d_da1, m->d_grad);
    if (update) {
        m->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
        k_adam<<<(NPARAM + 255) / 256, 256>>>(m->d_master, m->d_m1, m->d_m2, m->d_grad, m->d_wb, lr, b1, b2, 1e-8f,
                                              c1, c2);
    }
    MCK(cudaGetLastError());
    MCK(cudaDeviceSynchronize());
    if (loss) {
        std::vector<float> l(P);
        MCK(cudaMemcpy(l.data(), m->d_loss, 4 * P, cudaMemcpyDeviceToHost));
        double t = 0;
        for (float v : l) t += v;
        *loss = t;
    }
    if (grad_out) MCK(cudaMemcpy(grad_out, m->d_grad, 4 * NPARAM, cudaMemcpyDeviceToHost));
    return TKDV_OK;
}

}  // extern "C"

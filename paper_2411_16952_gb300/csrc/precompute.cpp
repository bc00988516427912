// precompute.cpp - host side of the per-point precompute of the rejection
// algorithm (Sec. IV.B, first step): alpha* (Eq. 29), the proposal variances
// sigma_k^2 (Eq. 25) and the rejection constant M = sup f/g (Eq. 45).
//
// The paper optimises f/g with Nelder-Mead from the Dirichlet kernel
// (Eq. 46).  Here the maximum is found by L-BFGS with the analytic gradient
// of log f/g on the sphere, from the Dirichlet kernel and a set of other
// starts (tapered Dirichlet kernels, single modes, seeded random directions);
// the largest local maximum wins.  A too-small M would bias the sampler
// (f/(Mg) > 1 somewhere), so the search errs on the side of many starts.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "../../include/tkdv.h"

namespace {

// log f/g(xh) = cS S + cH T + cQ ln Q with, for v_k = xh_k - i xh_{K+k},
//   S = sum k^2 s_k, s_k = xh_k^2 + xh_{K+k}^2         (H2 = E0 S, Eq. 20)
//   T = sum_n Re(conj(v_n) sum_{k<n} v_k v_{n-k})      (H3 = 2 pi (E0/2pi)^{3/2} T, Eq. 42)
//   Q = sum_k w_k s_k, w_k = 1/sigma_k^2               (2 a(xh) of Eq. 33)
struct Objective {
    int K = 0;
    double cS = 0, cH = 0, cQ = 0;
    std::vector<double> w;

    // value and gradient (d/dxh, length 2K) at a point of the sphere
    double eval(const double *xh, double *g) const {
        const double *x = xh, *y = xh + K;
        std::vector<double> A(K + 1, 0.0), B(K + 1, 0.0);
        double S = 0, Q = 0, T = 0;
        for (int k = 1; k <= K; ++k) {
            const double s = x[k - 1] * x[k - 1] + y[k - 1] * y[k - 1];
            S += (double)k * k * s;
            Q += w[k - 1] * s;
        }
        for (int n = 2; n <= K; ++n) {
            double a = 0, b = 0;
            for (int k = 1; k < n; ++k) {
                a += x[k - 1] * x[n - k - 1] - y[k - 1] * y[n - k - 1];
                b += x[k - 1] * y[n - k - 1] + y[k - 1] * x[n - k - 1];
            }
            A[n] = a;
            B[n] = b;
            T += x[n - 1] * a + y[n - 1] * b;
        }
        double val = cS * S + cH * T;
        if (cQ != 0) val += cQ * std::log(Q);
        if (g) {
            for (int j = 1; j <= K; ++j) {
                double dx = A[j], dy = B[j];
                for (int n = j + 1; n <= K; ++n) {
                    dx += 2.0 * (x[n - 1] * x[n - j - 1] + y[n - 1] * y[n - j - 1]);
                    dy += 2.0 * (y[n - 1] * x[n - j - 1] - x[n - 1] * y[n - j - 1]);
                }
                double gx = cS * 2.0 * j * j * x[j - 1] + cH * dx;
                double gy = cS * 2.0 * j * j * y[j - 1] + cH * dy;
                if (cQ != 0) {
                    gx += cQ * 2.0 * w[j - 1] * x[j - 1] / Q;
                    gy += cQ * 2.0 * w[j - 1] * y[j - 1] / Q;
                }
                g[j - 1] = gx;
                g[K + j - 1] = gy;
            }
        }
        return val;
    }

    // f(y) = log f/g(y/|y|) and its gradient in y
    double eval_y(const std::vector<double> &yv, std::vector<double> &gy) const {
        const int n = 2 * K;
        double nn = 0;
        for (double v : yv) nn += v * v;
        nn = std::sqrt(nn);
        std::vector<double> xh(n), g(n);
        for (int i = 0; i < n; ++i) xh[i] = yv[i] / nn;
        const double val = eval(xh.data(), g.data());
        double dot = 0;
        for (int i = 0; i < n; ++i) dot += g[i] * xh[i];
        gy.resize(n);
        for (int i = 0; i < n; ++i) gy[i] = (g[i] - dot * xh[i]) / nn;
        return val;
    }
};

// L-BFGS ascent of f(y) from y0; returns the best value found.
double lbfgs_max(const Objective &ob, std::vector<double> y) {
    const int n = 2 * ob.K, m = 12;
    auto normalise = [&](std::vector<double> &v) {
        double s = 0;
        for (double a : v) s += a * a;
        s = std::sqrt(s);
        for (double &a : v) a /= s;
    };
    normalise(y);
    std::vector<double> g, gn, yn(n), d(n);
    double f = ob.eval_y(y, g);
    std::vector<std::vector<double>> S, Yd;
    std::vector<double> rho;
    int stall = 0;
    for (int it = 0; it < 3000; ++it) {
        double gnorm = 0;
        for (double v : g) gnorm += v * v;
        if (std::sqrt(gnorm) < 1e-13) break;
        // two-loop recursion on the ascent direction (minimising -f)
        std::vector<double> q(n);
        for (int i = 0; i < n; ++i) q[i] = g[i];
        std::vector<double> al(S.size());
        for (int k = (int)S.size() - 1; k >= 0; --k) {
            double a = 0;
            for (int i = 0; i < n; ++i) a += S[k][i] * q[i];
            a *= rho[k];
            al[k] = a;
            for (int i = 0; i < n; ++i) q[i] -= a * Yd[k][i];
        }
        double gamma = 1.0;
        if (!S.empty()) {
            double sy = 0, yy = 0;
            for (int i = 0; i < n; ++i) {
                sy += S.back()[i] * Yd.back()[i];
                yy += Yd.back()[i] * Yd.back()[i];
            }
            gamma = sy / yy;
        } else {
            gamma = 0.1 / std::sqrt(gnorm);
        }
        for (int i = 0; i < n; ++i) q[i] *= gamma;
        for (int k = 0; k < (int)S.size(); ++k) {
            double b = 0;
            for (int i = 0; i < n; ++i) b += Yd[k][i] * q[i];
            b *= rho[k];
            for (int i = 0; i < n; ++i) q[i] += S[k][i] * (al[k] - b);
        }
        d = q;
        double slope = 0;
        for (int i = 0; i < n; ++i) slope += d[i] * g[i];
        if (!(slope > 0)) {  // not an ascent direction: restart from the gradient
            S.clear();
            Yd.clear();
            rho.clear();
            for (int i = 0; i < n; ++i) d[i] = g[i] * (0.1 / std::sqrt(gnorm));
            slope = 0;
            for (int i = 0; i < n; ++i) slope += d[i] * g[i];
        }
        double t = 1.0, fn = 0;
        bool ok = false;
        for (int ls = 0; ls < 60; ++ls) {
            for (int i = 0; i < n; ++i) yn[i] = y[i] + t * d[i];
            fn = ob.eval_y(yn, gn);
            if (fn >= f + 1e-4 * t * slope) {
                ok = true;
                break;
            }
            t *= 0.5;
        }
        if (!ok) break;
        std::vector<double> s(n), yd(n);
        double sy = 0;
        for (int i = 0; i < n; ++i) {
            s[i] = yn[i] - y[i];
            yd[i] = -(gn[i] - g[i]);  // gradient of -f
            sy += s[i] * yd[i];
        }
        if (sy > 1e-300) {
            S.push_back(s);
            Yd.push_back(yd);
            rho.push_back(1.0 / sy);
            if ((int)S.size() > m) {
                S.erase(S.begin());
                Yd.erase(Yd.begin());
                rho.erase(rho.begin());
            }
        }
        const double gain = fn - f;
        y = yn;
        g = gn;
        f = fn;
        double ny = 0;
        for (double v : y) ny += v * v;
        if (ny > 4.0) {  // keep |y| near 1 (f is scale invariant)
            const double s0 = std::sqrt(ny);
            for (double &v : y) v /= s0;
            for (double &v : g) v *= s0;
            S.clear();
            Yd.clear();
            rho.clear();
        }
        if (gain <= 1e-16 * (1.0 + std::fabs(f))) {
            if (++stall >= 8) break;
        } else {
            stall = 0;
        }
    }
    return f;
}

}  // namespace

extern "C" int tkdv_alpha_star(int K, double beta_p, double *out) {
    if (K < 1 || K > 1024 || !(beta_p >= 0) || !out) return TKDV_ERR_INVALID_ARG;
    const double K3 = (double)K * K * K;
    auto F = [&](double a, double *dF) {
        double s = 0, s2 = 0;
        for (int k = 1; k <= K; ++k) {
            const double q = 1.0 / (1.0 + a * beta_p * (double)k * k / K3);
            s += q;
            s2 += q * q;
        }
        if (dF) *dF = -s2 / K;
        return 1.0 - a / K * s;
    };
    if (beta_p == 0.0) {
        *out = 1.0;
        return TKDV_OK;
    }
    // F decreases from 1 to 1 - K^2 sum(1/k^2)/beta'; a root exists iff that is < 0
    double bound = 0;
    for (int k = 1; k <= K; ++k) bound += 1.0 / ((double)k * k);
    bound *= (double)K * K;
    if (beta_p >= bound) return TKDV_ERR_NO_ALPHA;
    double lo = 0.0, hi = 1.0;
    while (F(hi, nullptr) > 0) {
        lo = hi;
        hi *= 2.0;
        if (hi > 1e300) return TKDV_ERR_NO_ALPHA;
    }
    double a = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
        double dF;
        const double f = F(a, &dF);
        if (f > 0)
            lo = a;
        else
            hi = a;
        if (f == 0.0 || hi - lo <= 4e-16 * hi) break;
        double an = a - f / dF;  // Newton step, kept inside the bracket
        if (!(an > lo && an < hi)) an = 0.5 * (lo + hi);
        if (an == a) break;
        a = an;
    }
    *out = a;
    return TKDV_OK;
}

extern "C" int tkdv_log_M(int K, double beta_p, double E0, double r, const double *sigma2, double *out) {
    if (K < 1 || K > TKDV_KMAX || !(E0 > 0) || !(beta_p >= 0) || !std::isfinite(r) || !out)
        return TKDV_ERR_INVALID_ARG;
    Objective ob;
    ob.K = K;
    const double K2 = (double)K * K;
    ob.cS = -beta_p / K2;
    const double c = std::sqrt(E0 / (2.0 * M_PI));
    ob.cH = beta_p * r / (E0 * K2) * 2.0 * M_PI * c * c * c;
    ob.w.assign(K, 1.0);
    if (sigma2) {
        ob.cQ = K;
        for (int k = 0; k < K; ++k) {
            if (!(sigma2[k] > 0)) return TKDV_ERR_INVALID_ARG;
            ob.w[k] = 1.0 / sigma2[k];
        }
    }
    const int n = 2 * K;
    std::vector<std::vector<double>> starts;
    std::vector<double> v(n, 0.0);
    for (int k = 0; k < K; ++k) v[k] = 1.0;  // Dirichlet kernel, Eq. (46)
    starts.push_back(v);
    for (double gam : {0.5, 2.0, 8.0, 32.0}) {  // Dirichlet kernels with a Gaussian taper
        std::fill(v.begin(), v.end(), 0.0);
        for (int k = 1; k <= K; ++k) v[k - 1] = std::exp(-gam * (double)k * k / K2);
        starts.push_back(v);
    }
    std::mt19937_64 gen(0x7D0C5EEDull);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (int k = 0; k < K; ++k) {  // single modes, nudged off the stationary point
        for (int i = 0; i < n; ++i) v[i] = 1e-3 * nd(gen);
        v[k] = 1.0;
        starts.push_back(v);
    }
    for (int s = 0; s < 8; ++s) {
        for (int i = 0; i < n; ++i) v[i] = nd(gen);
        starts.push_back(v);
    }
    double best = -INFINITY;
    for (auto &s0 : starts) best = std::max(best, lbfgs_max(ob, s0));
    if (!std::isfinite(best)) return TKDV_ERR_ENVELOPE;
    *out = best;
    return TKDV_OK;
}

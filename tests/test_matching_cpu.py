"""The bisection driver of the downstream beta' (host logic, no GPU).

Closed form used here and in the GPU test: at C3/C2 = 0 the target measure
is f ~ exp(-beta' S / K^2) on the sphere, and under the uniform measure the
pair energies s_k are Dirichlet(1, .., 1), so Z(a) = E[exp(-a S)] with
a = beta'/K^2 is (K-1)! a^-(K-1) sum_k b_k exp(-a k^2), b_k =
1/prod_{j != k}(j^2 - k^2) (Hermite-Genocchi), and the ensemble mean of S is
-d ln Z/da = (K-1)/a + sum_k k^2 b_k e^{-a k^2} / sum_k b_k e^{-a k^2}.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2411_16952_gb300 import matching as MT


def mean_S_closed(K, bp):
    a = bp / K**2
    k = np.arange(1, K + 1, dtype=np.float64)
    b = np.array([1.0 / np.prod([j * j - kk * kk for j in k if j != kk]) for kk in k])
    e = np.exp(-a * k * k) * b
    return (K - 1) / a + float(np.sum(k * k * e) / np.sum(e))


def mean_S_stable(K, bp):
    """The same mean for large K: Z(a) = (K-1)! times the divided difference
    of exp at the nodes -a k^2 (Hermite-Genocchi), taken as the corner entry
    of the exponential of the bidiagonal matrix with those nodes on the
    diagonal and ones above it (Opitz's theorem), which avoids the
    cancellation of the explicit sum; mean S = -d ln Z / da by central
    differences."""
    sl = pytest.importorskip("scipy.linalg")

    def lnZ(a):
        x = -a * np.arange(1, K + 1, dtype=np.float64) ** 2
        return math.log(sl.expm(np.diag(x) + np.diag(np.ones(K - 1), 1))[0, K - 1]) + math.lgamma(K)

    a = bp / K**2
    h = 1e-5 * a
    return -(lnZ(a + h) - lnZ(a - h)) / (2 * h)


def fake_batch(K, noise=0.0, seed=0):
    rng = np.random.default_rng(seed)

    def run(betas, point_id0, n, s):
        out = []
        for b in betas:
            spec = np.zeros(64)
            spec[0] = 1000.0 * (mean_S_closed(K, b) + noise * rng.standard_normal())  # k = 1: sum k^2 s_k
            out.append({"n_accepted": 1000, "spectrum": spec, "skew": 0.0})
        return out
    return run


def test_closed_form_against_oracle_mean_S():
    """The closed form of the r = 0 ensemble mean of S against the oracle's
    accepted samples (paper proposal), and the spectrum sums against the
    per-sample S of the same run."""
    K, bp = 8, 30.0
    pt = O.make_point(K, 1.0, bp, 0.0, O.PAPER)
    pt.logM = O.log_M(pt, 0)
    n = 1 << 18
    total, rec = O.run_accepted(pt, 3, 0, 0, n, cap=n)
    S = rec["S"]
    assert total == len(S)
    want = mean_S_closed(K, bp)
    assert abs(S.mean() - want) < 4 * S.std() / math.sqrt(len(S)), (S.mean(), want)
    st = O.run_stats(pt, 3, 0, 0, n)
    k = np.arange(1, K + 1)
    assert abs(np.dot(k * k, st["spectrum"]) / st["n_acc"] - S.mean()) < 1e-9 * S.mean()


def test_bisection_recovers_beta():
    K, beta_true = 8, 30.0
    target = mean_S_closed(K, beta_true)
    res = MT.bisect_beta(K, 1.0, 0.0, MT.mean_S, target, 10.0, 60.0, n_candidates=16, n_steps=4,
                         run_batch=fake_batch(K))
    assert abs(res["beta"] - beta_true) < 1e-4
    lo, hi = res["bracket"]
    assert lo <= beta_true <= hi and hi - lo < 50.0 * (2.0 / 15) ** 4 * 1.01
    assert len(res["history"]) == 4 and len(res["history"][0][0]) == 16


def test_bisection_with_noise_stays_near_root():
    K, beta_true = 8, 30.0
    target = mean_S_closed(K, beta_true)
    res = MT.bisect_beta(K, 1.0, 0.0, MT.mean_S, target, 10.0, 60.0, n_candidates=16, n_steps=3,
                         run_batch=fake_batch(K, noise=0.01, seed=4))
    # slope of mean S near beta' = 30 is about -0.3 per unit beta'
    assert abs(res["beta"] - beta_true) < 0.2


def test_bisection_rejects_unbracketed_target():
    K = 8
    with pytest.raises(ValueError):
        MT.bisect_beta(K, 1.0, 0.0, MT.mean_S, mean_S_closed(K, 80.0), 10.0, 60.0, run_batch=fake_batch(K))
    with pytest.raises(ValueError):
        MT.bisect_beta(K, 1.0, 0.0, MT.mean_S, 1.0, 60.0, 10.0, run_batch=fake_batch(K))


def test_stable_closed_form_matches_explicit_sum():
    """The matrix-exponential form of the r = 0 mean of S equals the explicit
    divided-difference sum where the latter is still accurate (K <= 16), and
    stays between the extreme values of S at K = 64."""
    for K, bp in [(8, 30.0), (8, 60.0), (16, 20.0), (16, 80.0)]:
        assert abs(mean_S_stable(K, bp) - mean_S_closed(K, bp)) < 1e-9 * mean_S_closed(K, bp)
    K = 64
    vals = [mean_S_stable(K, bp) for bp in (20.0, 40.0, 80.0)]
    assert 1.0 < vals[2] < vals[1] < vals[0] < (K + 1) * (2 * K + 1) / 6.0  # below the uniform mean

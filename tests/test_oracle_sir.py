"""Pins of the oracle's sampling-importance resampling (SIR): weights
exp(log f/(Mg)), Poisson copy numbers by inversion of the accept uniform.

* The inversion n = #{k >= 1 : u < P(N >= k)} is the inverse survival
  function of the Poisson law (scipy's isf).
* beta' = 0, uniform proposal: f = g, every weight is exp(-log M), so the copy
  numbers are iid Poisson(c exp(-log M)) and the weighted mean of S is its
  mean under the uniform measure, sum_k k^2 / K = (K+1)(2K+1)/6.
* C3/C2 = 0: the importance-sampling and the resampled means of S both
  estimate the closed-form ensemble mean (tests/test_matching_cpu.py).
* The total number of copies is Poisson with mean c sum_i exp(Delta_i).
"""
import math

import numpy as np
import pytest

import oracle as O
from test_matching_cpu import mean_S_closed


def test_poisson_inversion_is_the_inverse_survival_function():
    sp = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    for lam in (1e-12, 1e-6, 1e-3, 0.1, 1.0, 3.0, 10.0, 50.0):
        us = np.concatenate([10.0 ** -rng.uniform(0, 14, 200), rng.uniform(0, 1, 200)])
        for u in us:
            want = int(sp.poisson.isf(u, lam))
            got = O.poisson_count(lam, u)
            if got != want:  # only where u sits on a tail value to rounding
                k = max(got, want)
                assert abs(u - sp.poisson.sf(k - 1, lam)) <= 1e-12 * u, (lam, u, got, want)
    for lam in (1e-8, 0.3, 2.0, 30.0):
        for k in (1, 2, 5, 40):
            assert abs(O.poisson_tail(lam, k) - sp.poisson.sf(k - 1, lam)) <= 1e-12 + 1e-10 * sp.poisson.sf(k - 1, lam)


def test_sir_equal_weights_at_beta_zero():
    K, n, c, lm = 8, 1 << 16, 0.5, 0.0
    pt = O.make_point(K, 1.0, 0.0, 0.0, O.UNIFORM, logM=lm)
    st, kept = O.run_sir(pt, 4, 1, 0, n, c, cap=n)
    assert st["n_prop"] == n and abs(st["sum_w"] - n) < 1e-9 * n and abs(st["sum_w2"] - n) < 1e-9 * n
    counts = np.zeros(n)
    counts[(kept["idx"]).astype(np.int64)] = kept["copies"]
    assert abs(counts.mean() - c) < 4 * math.sqrt(c / n)
    assert abs(counts.var() - c) < 4 * math.sqrt(2 * c * c / n + c / n)
    assert st["n_copies"] == counts.sum() and st["n_kept"] == np.count_nonzero(counts)
    mean_S = (K + 1) * (2 * K + 1) / 6.0
    assert abs(st["sum_wS"] / st["sum_w"] - mean_S) < 0.02 * mean_S


def test_sir_means_match_closed_form_at_r0():
    K, bp, n, c = 8, 30.0, 1 << 18, 0.25
    pt = O.make_point(K, 1.0, bp, 0.0, O.PAPER)
    pt.logM = O.log_M(pt, 0)
    st, kept = O.run_sir(pt, 9, 2, 0, n, c, cap=n)
    want = mean_S_closed(K, bp)
    S = np.repeat(kept["S"], kept["copies"])
    sd = S.std()
    ess = st["sum_w"] ** 2 / st["sum_w2"]
    assert abs(st["sum_wS"] / st["sum_w"] - want) < 4 * sd / math.sqrt(ess), (st["sum_wS"] / st["sum_w"], want)
    assert abs(st["sum_nS"] / st["n_copies"] - want) < 4 * sd / math.sqrt(st["n_copies"])
    assert abs(S.mean() - st["sum_nS"] / st["n_copies"]) < 1e-9 * want
    mu = c * st["sum_w"]
    assert abs(st["n_copies"] - mu) < 5 * math.sqrt(mu)
    k = np.arange(1, K + 1)
    assert abs(np.dot(k * k, st["spectrum"]) - st["sum_nS"]) < 1e-9 * st["sum_nS"]

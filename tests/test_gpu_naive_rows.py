"""Naive (uniform-proposal) rows of Table 2.

For mean-zero log-variance changes and for the uniform proposal alike, the
acceptance of a rejection sampler with proposal density g = prod w_k Q^-K
(Eqs. 33-38; w = 1 for the uniform measure) is prod_k w_k Z / M, with
Z = E_mu0[exp(-beta H)] and M the envelope of Eq. (45).  So the improvement
factor of the paper proposal over the uniform one is
exp(sum_k ln w_k + log M_uniform - log M_paper), with no Monte Carlo.

This test measures the uniform proposal's acceptance on the GPU at K = 32
rows where the printed improvement and the identity disagree most, and
checks the measurement against the identity (the printed value is reported
alongside).  Both envelopes come from the library's search.  At these
acceptances a large share of the accepted draws have log f/(Mg) below
ln 2^-24, so the rows also check the refined tail of the uniform map.
"""
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16952_gb300 import _build
    _build.build()
    import paper_2411_16952_gb300 as T
    return T


# The last row is one of the two that Table 2 marks as taking weeks with the
# uniform proposal (uniform acceptance about 7.5e-12: 2^40 proposals, under
# two minutes, give about 8 accepts).
ROWS = [(20.0, 150.0, 28, 26), (40.0, 150.0, 32, 26), (40.0, 225.0, 34, 28), (40.0, 300.0, 36, 30),
        (40.0, 450.0, 40, 34)]
# The other asterisked row (uniform acceptance about 3.5e-13 by the identity:
# 2^44 proposals, about half an hour of one GPU, give about 6 accepts); run
# with TKDV_LONG_TESTS=1.
LONG_ROWS = [(60.0, 300.0, 44, 36)]
long_only = pytest.mark.skipif(not os.environ.get("TKDV_LONG_TESTS"), reason="set TKDV_LONG_TESTS=1")


@pytest.mark.parametrize("bp,r,log2n,log2p", ROWS + [pytest.param(*x, marks=long_only) for x in LONG_ROWS])
def test_uniform_acceptance_matches_identity(T, bp, r, log2n, log2p):
    K, E0 = 32, 1.0
    row = [x for x in GOLD["table2_K32"]["rows"] if x[0] == bp and x[1] == r][0]
    acc_paper_printed, imp_printed = row[3], row[4]
    a = T.tkdv_alpha_star(K, bp)
    k = np.arange(1, K + 1)
    s2 = 1.0 / (1.0 + a * bp * k * k / K**3)
    lm_p = T.tkdv_log_M(K, bp, E0, r, s2)
    lm_u = T.tkdv_log_M(K, bp, E0, r, None)
    improvement = math.exp(np.sum(np.log(1.0 / s2)) + lm_u - lm_p)
    # measured: both proposals on the GPU
    n_u = 1 << log2n
    n_p = 1 << log2p
    Su = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_UNIFORM, point_id=1)], sample_capacity=16)
    Sp = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=2)], sample_capacity=16)
    Su.autotune(1 << 22)
    Su.run(n_u, 3)
    Sp.run(n_p, 3)
    su, sp = Su.stats()[0], Sp.stats()[0]
    Su.close()
    Sp.close()
    assert su["n_envelope_violations"] == 0 and sp["n_envelope_violations"] == 0
    acc_u, acc_p = su["n_accepted"] / n_u, sp["n_accepted"] / n_p
    assert su["n_accepted"] >= (1 if log2n >= 40 else 100)
    pred_u = acc_p / improvement
    se = math.sqrt(pred_u / n_u) + pred_u * math.sqrt((1 - acc_p) / (acc_p * n_p))
    assert abs(acc_u - pred_u) <= 4 * se, (acc_u, pred_u, se)
    print("K=32 beta'=%g C3/C2=%g: uniform acceptance %.3e (%d accepts of 2^%d), paper proposal %.3e; "
          "improvement measured %.3g, identity %.3g, printed %g" % (
              bp, r, acc_u, su["n_accepted"], log2n, acc_p, acc_p / acc_u, improvement, imp_printed))

"""The bisection driver of the downstream beta' on the GPU sampler.

At C3/C2 = 0 the ensemble mean of S = H2/E0 has a closed form
(tests/test_matching_cpu.py::mean_S_closed).  Taking the value at
beta' = 30 as the target, the driver must recover beta' = 30 from 16
candidates per step sampled in one batched launch, reading S from the
per-mode spectrum statistic.
"""
import pytest

from test_matching_cpu import mean_S_closed, mean_S_stable

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16952_gb300 import _build
    _build.build()
    import paper_2411_16952_gb300 as T
    return T


@pytest.mark.parametrize("h3_mode,grid_N", [(0, 0), (1, 32)])
def test_bisection_recovers_closed_form_beta(T, h3_mode, grid_N):
    from paper_2411_16952_gb300 import matching as MT
    K, beta_true = 8, 30.0
    res = MT.bisect_beta(K, 1.0, 0.0, MT.mean_S, mean_S_closed(K, beta_true), 10.0, 60.0, n_candidates=16,
                         n_steps=3, proposals_per_candidate=1 << 22, seed=5, h3_mode=h3_mode, grid_N=grid_N)
    # per candidate ~4e6 accepted fields: mean S to ~2e-3, slope ~ -0.3 per unit beta'
    assert abs(res["beta"] - beta_true) < 0.05, res["beta"]
    print("bisection (h3_mode %d): beta' = %.4f, bracket %s" % (h3_mode, res["beta"], res["bracket"]))


def test_bisection_K64_grid256(T):
    """The 64-mode configuration of the downstream search: K = 64, the grid
    form with N = 256 points, 16 candidates per step in one launch.  The
    target is the closed-form mean of S at beta' = 40 (matrix-exponential
    form, pinned against the explicit sum on the CPU)."""
    from paper_2411_16952_gb300 import matching as MT
    K, beta_true = 64, 40.0
    res = MT.bisect_beta(K, 1.0, 0.0, MT.mean_S, mean_S_stable(K, beta_true), 20.0, 80.0, n_candidates=16,
                         n_steps=3, proposals_per_candidate=1 << 22, seed=9, h3_mode=T.H3_GRID_BF16X3, grid_N=256)
    # mean S falls by about 4.8 per unit beta' here; its sampling error per
    # candidate (about 4e6 accepted fields) is below 0.1
    assert abs(res["beta"] - beta_true) < 0.15, res["beta"]
    print("K = 64, N = 256 bisection: beta' = %.4f, bracket %s" % (res["beta"], res["bracket"]))

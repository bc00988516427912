"""The headline workload at full size, in the launch configuration the
benchmark times: K = 32, eight points (beta' = geomspace(20, 60, 8),
C3/C2 = 9000 / beta', E0 = 1, paper proposal), 2^28 proposals per point in
one autotuned persistent launch, seed 0; the grid form (N = 128) and the
FP32 triad form.  The oracle's envelopes (tests/golden/envelopes.json) are
injected, so both sides decide against the same log M.

* every accepted record is replayed by the oracle: accepted there too (or
  within 1e-6 of the threshold), H, u0 and xhat within the parity
  tolerances;
* on the first 2^22 indices of every point the accepted set equals the
  oracle's, so no acceptance is missing;
* the statistics agree with the records (counts, u0 sums).
"""
import numpy as np
import pytest

import oracle as O
from test_gpu_parity import check_records_against_oracle, compare_accept_sets, envelope

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


@pytest.mark.parametrize("form", ["grid", "triad"])
def test_headline_workload_full_size(T, form):
    from paper_2411_16952_gb300 import workloads
    wl = workloads.extreme_k32(1 << 28)
    K, E0, n, seed, prefix = wl["K"], wl["E0"], wl["n"], 0, 1 << 22
    lms = [envelope(K, E0, b, r, O.PAPER) for b, r in wl["points"]]
    pts = [T.make_point(b, E0, r, T.PROPOSAL_PAPER, point_id=p, logM=lm)
           for p, ((b, r), lm) in enumerate(zip(wl["points"], lms))]
    mode = T.H3_GRID_BF16X3 if form == "grid" else T.H3_TRIAD_F32
    S = T.Sampler(K, pts, h3_mode=mode, grid_N=wl["grid_N"] if form == "grid" else 0, sample_capacity=1 << 21)
    S.autotune(1 << 22)
    S.run(n, seed)
    st = S.stats()
    rec = S.samples(1 << 21)
    S.close()
    total = 0
    for p, ((b, r), lm) in enumerate(zip(wl["points"], lms)):
        s = st[p]
        assert s["n_proposals"] == n and s["n_dropped"] == 0 and s["n_fallback"] == 0
        mine = rec["point"] == p
        idx = rec["idx"][mine]
        assert len(idx) == s["n_accepted"] > 1000
        total += len(idx)
        pt = O.make_point(K, E0, b, r, O.PAPER, logM=lm)
        o = O.replay(pt, seed, p, idx)
        assert np.all(o["accept"] | o["near"]), idx[~(o["accept"] | o["near"])][:8]
        check_records_against_oracle({k: v[mine] for k, v in rec.items()}, o, r, K)
        # the records' u0 sums are the statistics' (fixed-point sums of FP32 values)
        u0 = rec["u0"][mine].astype(np.float64)
        assert abs(s["sum_u0"][0] - u0.sum()) <= 1e-6 * len(u0) + 1e-6 * abs(u0.sum())
        # no acceptance missing on the prefix
        _, opre = O.run_accepted(pt, seed, p, 0, prefix, cap=1 << 16)
        compare_accept_sets(idx[idx < prefix], pt, seed, p, opre["idx"])
    assert len(rec["idx"]) == total
    print("%s form: %d accepted of 8 x 2^28" % (form, total))

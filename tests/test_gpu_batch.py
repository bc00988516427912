"""The 64-point batch (beta' log-uniform on [6, 600], E0 in [0.5, 2], D in
{1, 0.24}, budgets 2^18..2^26, K = 32) in one persistent launch at full size:
every point's accepted records and a sample of every point's proposals are
replayed by the oracle; per-point statistics are consistent with the
records."""
import math

import numpy as np
import pytest

import oracle as O

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


def oracle_envelope(K, E0, bp, r):
    """The paper's envelope search: Nelder-Mead from the Dirichlet kernel (Eq. 46)."""
    pt = O.make_point(K, E0, bp, r, O.PAPER)
    x0 = np.zeros(2 * K)
    x0[:K] = 1 / math.sqrt(K)
    v, _ = O.nelder_mead(pt, x0, 200000)
    return v


@pytest.mark.parametrize("mode", ["triad", "grid"])
def test_batch_of_64_points(T, mode):
    from concurrent.futures import ThreadPoolExecutor
    from paper_2411_16952_gb300 import workloads
    wl = workloads.batch_k32()
    K = wl["K"]
    with ThreadPoolExecutor(8) as ex:
        lms = list(ex.map(lambda p: oracle_envelope(K, wl["E0"][p], wl["beta_p"][p], wl["r"][p]), range(64)))
    pts = [T.make_point(float(wl["beta_p"][p]), float(wl["E0"][p]), float(wl["r"][p]), T.PROPOSAL_PAPER,
                        point_id=p, logM=lms[p]) for p in range(64)]
    h3 = T.H3_GRID_BF16X3 if mode == "grid" else T.H3_TRIAD_F32
    S = T.Sampler(K, pts, h3_mode=h3, grid_N=128 if mode == "grid" else 0, sample_capacity=1 << 24)
    S.autotune(1 << 20)
    S.run_budgets(wl["budgets"], 31)
    st = S.stats()
    rec = S.samples(1 << 24)
    S.close()
    # the ring keeps 2^24 records; any excess is counted per point as dropped
    assert len(rec["idx"]) + sum(s["n_dropped"] for s in st) == sum(s["n_accepted"] for s in st)
    rng = np.random.default_rng(0)
    for p in range(64):
        s = st[p]
        assert s["n_proposals"] == int(wl["budgets"][p])
        mine = rec["point"] == p
        assert mine.sum() + s["n_dropped"] == s["n_accepted"]
        assert int(s["hist"].sum()) == s["n_accepted"]
        pt = O.make_point(K, float(wl["E0"][p]), float(wl["beta_p"][p]), float(wl["r"][p]), O.PAPER, logM=lms[p])
        # accepted records: the oracle accepts them too (or puts them within 1e-6 of the threshold)
        idx = rec["idx"][mine]
        sel = idx[:40]
        if len(sel):
            o = O.replay(pt, 31, p, sel)
            assert np.all(o["accept"] | o["near"]), p
            j = np.nonzero(mine)[0][:40]
            scale = np.abs(o["H2"]) + np.abs(pt.r * o["H3"])
            dH = (rec["H2"][j] - pt.r * rec["H3"][j]) - (o["H2"] - pt.r * o["H3"])
            assert np.all(np.abs(dH) <= 1e-5 * scale), p
        if s["n_dropped"]:
            continue  # records incomplete for this point: the checks below need all of them
        # sampled proposals: accepted by the oracle iff among the records
        probe = rng.integers(0, int(wl["budgets"][p]), 64).astype(np.uint64)
        o = O.replay(pt, 31, p, probe)
        recset = set(idx.tolist())
        for q, i in enumerate(probe):
            if not o["near"][q]:
                assert bool(o["accept"][q]) == (int(i) in recset), (p, int(i))
        # moments consistent with the records' u0
        u0 = rec["u0"][mine].astype(np.float64)
        assert abs(s["sum_u0"][0] - u0.sum()) <= 1e-5 * (1 + np.abs(u0).sum())

"""The multi-rank merge on the library's own output: two disjoint shards of an
index range, sampled by the library on one GPU and merged by dist.combine (the
same reduction merge_stats applies across ranks), equal one run over the whole
range.  Integer statistics, the fixed-point power sums and the spectrum are
exact; the recomputed moments equal the library's; SIR runs carry n_kept and
their importance sums."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16952_gb300 import _build
    _build.build()
    import paper_2411_16952_gb300 as T
    return T


def logM(key):
    return json.load(open(os.path.join(HERE, "golden", "envelopes.json")))["points"][key]["logM"]


INT_KEYS = ("n_proposals", "n_accepted", "n_near_threshold", "n_refined", "n_envelope_violations", "n_dropped",
            "n_fallback", "n_kept")


def run(T, K, points, idx0, count, seed, **kw):
    S = T.Sampler(K, points, sample_capacity=1 << 20, **kw)
    S.run_ranges(idx0, count, seed)
    st = S.stats()
    rec = S.samples(1 << 20)
    S.close()
    return st, rec


@pytest.mark.parametrize("h3_mode", [0, 1])
def test_two_shards_merge_to_one_run(T, h3_mode):
    from paper_2411_16952_gb300 import dist as D
    K, seed, n = 16, 3, 3_000_017
    pts = [T.make_point(20.0, 1.0, 75.0, T.PROPOSAL_PAPER, point_id=0, logM=logM("K16_E1_b20_r75_p1")),
           T.make_point(20.0, 1.0, 75.0, T.PROPOSAL_UNIFORM, point_id=1, logM=logM("K16_E1_b20_r75_p0"))]
    kw = dict(h3_mode=h3_mode, grid_N=64 if h3_mode else 0)
    one, rec1 = run(T, K, pts, [0, 0], [n, n], seed, **kw)
    shards = []
    recs = []
    for r in range(2):
        s0, c = D.shard_range(n, r, 2)
        st, rec = run(T, K, pts, [s0, s0], [c, c], seed, **kw)
        shards.append(st)
        recs.append(rec)
    merged = D.combine(shards)
    for p in range(2):
        for k in INT_KEYS:
            assert merged[p][k] == one[p][k], (p, k)
        assert np.array_equal(merged[p]["hist"], one[p]["hist"])
        assert np.array_equal(merged[p]["exceed"], one[p]["exceed"])
        assert np.array_equal(merged[p]["sum_u0"], one[p]["sum_u0"])
        assert np.array_equal(merged[p]["spectrum"], one[p]["spectrum"])
        assert merged[p]["max_delta"] == one[p]["max_delta"]
        for k in ("mean", "var", "skew", "kurt"):
            assert abs(merged[p][k] - one[p][k]) <= 1e-12 * (1 + abs(one[p][k])), (p, k)
        assert merged[p]["logM"] == one[p]["logM"]
    assert one[0]["n_accepted"] > 1000
    # the shards' records together are the one run's records
    idx = np.concatenate([r["idx"] + (r["point"].astype(np.uint64) << np.uint64(40)) for r in recs])
    idx1 = rec1["idx"] + (rec1["point"].astype(np.uint64) << np.uint64(40))
    assert np.array_equal(np.sort(idx), np.sort(idx1))


def test_sir_shards_merge(T):
    from paper_2411_16952_gb300 import dist as D
    K, seed, n = 16, 5, 2_000_003
    pts = [T.make_point(20.0, 1.0, 75.0, T.PROPOSAL_PAPER, point_id=2, logM=logM("K16_E1_b20_r75_p1"),
                        sir_c=50.0)]
    one, _ = run(T, K, pts, [0], [n], seed, sir=True)
    shards = [run(T, K, pts, [D.shard_range(n, r, 2)[0]], [D.shard_range(n, r, 2)[1]], seed, sir=True)[0]
              for r in range(2)]
    merged = D.combine(shards)
    for k in INT_KEYS:
        assert merged[0][k] == one[0][k], k
    assert merged[0]["n_kept"] > 100
    assert np.array_equal(merged[0]["hist"], one[0]["hist"])
    for k in ("sir_sum_w", "sir_sum_w2", "sir_sum_wS"):
        # FP64 sums of FP32 partial sums: the split moves their last FP32 bits
        assert abs(merged[0][k] - one[0][k]) <= 1e-5 * abs(one[0][k]), k
    assert np.allclose(merged[0]["sir_sum_w_u0"], one[0]["sir_sum_w_u0"], rtol=1e-5, atol=1e-6)

"""The sampler at 65..128 modes (one warp per batch of four proposals) against
the oracle.

K = 128 is the cutoff of the paper's parallel-speedup test (Fig. 7).  The warp
form draws the same stream and takes the same decisions as the one-thread form,
so the one-thread tests carry over.  Accepted sets equal the oracle's, except
draws within 1e-6 of the threshold.  Per-record H, u0 and xhat and the
statistics stay within the same tolerances.  The cases also cover ragged
batches (counts not a multiple of four), K not a multiple of eight and odd K,
launch shapes, split runs, batched points, the allocation-free entry point and
the refined tail of the uniform map.
"""
import math

import numpy as np
import pytest

import oracle as O
from test_gpu_parity import check_records_against_oracle, compare_accept_sets, int_view

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


def tprop(T, prop):
    return T.PROPOSAL_PAPER if prop == O.PAPER else T.PROPOSAL_UNIFORM


def rate_logM(K, E0, bp, r, prop, seed, pid, rate):
    """An envelope accepting about a fraction `rate` of the draws: log of the
    oracle's mean f/g over the first 2048 proposals, minus ln rate.  (At
    K = 128 log f/g is so concentrated that a quantile of it would accept
    almost every draw.)"""
    lf = O.replay(O.make_point(K, E0, bp, r, prop), seed, pid, np.arange(2048, dtype=np.uint64))["logfg"]
    return float(lf.max() + np.log(np.mean(np.exp(lf - lf.max()))) - np.log(rate))


# (K, E0, beta', C3/C2, proposal): beta' C3/C2 = 9000 as in the Table 2 regime
CASES = [(128, 1.0, 60.0, 150.0, O.PAPER), (128, 1.0, 20.0, 450.0, O.UNIFORM), (100, 1.3, 40.0, 225.0, O.PAPER),
         (127, 1.0, 30.0, 300.0, O.PAPER), (65, 0.8, 60.0, 150.0, O.UNIFORM)]


@pytest.mark.parametrize("K,E0,bp,r,prop", CASES)
def test_full_run_matches_oracle(T, K, E0, bp, r, prop):
    """2^17 + 3 proposals from index 7 (a ragged last batch): every proposal of
    the persistent launch is replayed by the oracle."""
    seed, pid, i0, n = 12, 5, 7, (1 << 17) + 3
    lm = rate_logM(K, E0, bp, r, prop, seed, pid, 0.03)
    S = T.Sampler(K, [T.make_point(bp, E0, r, tprop(T, prop), point_id=pid, logM=lm)], sample_capacity=1 << 16)
    S.run_ranges([i0], [n], seed)
    st = S.stats()[0]
    rec = S.samples(1 << 16)
    S.close()
    pt = O.make_point(K, E0, bp, r, prop, logM=lm)
    total, orec = O.run_accepted(pt, seed, pid, i0, n, cap=1 << 16)
    ost = O.run_stats(pt, seed, pid, i0, n)
    assert st["n_proposals"] == n and st["n_dropped"] == 0 and st["n_fallback"] == 0
    assert st["n_accepted"] == len(rec["idx"]) and total > 1000
    excused = compare_accept_sets(rec["idx"], pt, seed, pid, orec["idx"])
    assert abs(st["n_accepted"] - total) <= excused
    assert st["n_near_threshold"] == ost["n_near"]
    common = np.isin(rec["idx"], orec["idx"])
    check_records_against_oracle({k: v[common] for k, v in rec.items()}, orec, r, K)
    if excused == 0:
        for q in range(4):
            assert abs(st["sum_u0"][q] - ost["sum_u0"][q]) <= 2e-6 * (1 + abs(ost["sum_u0"][q])) + 1e-6 * total
        spec_tol = 2e-6 * ost["spectrum"][:K] + total * 2.0**-28 + 1e-9
        assert np.all(np.abs(st["spectrum"][:K] - ost["spectrum"][:K]) <= spec_tol)
        assert np.all(st["spectrum"][K:] == 0)
    print("K=%d prop=%d: accepted %d of %d, refined %d, near %d, excused %d" % (
        K, prop, st["n_accepted"], n, st["n_refined"], st["n_near_threshold"], excused))


def test_launch_shapes_and_split_runs_agree(T):
    """The accepted set and every integer statistic depend only on (parameters,
    seed, index range): 128- or 256-thread CTAs, the CTA count, graph or plain
    launches, and a range cut into runs of 1, 3 and 5 proposals change
    nothing."""
    K, E0, bp, r, seed, pid = 128, 1.0, 60.0, 150.0, 3, 2
    lm = rate_logM(K, E0, bp, r, O.PAPER, seed, pid, 0.05)
    pts = [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=pid, logM=lm)]
    n = 200_003

    def run(ranges, **kw):
        S = T.Sampler(K, pts, sample_capacity=1 << 16, **kw)
        for a, c in ranges:
            S.run_ranges([a], [c], seed)
        st, rec = S.stats()[0], S.samples(1 << 16)
        S.close()
        return st, set(rec["idx"].tolist())

    ref, rref = run([(11, n)])
    for kw in [dict(threads_per_cta=128), dict(ctas_per_sm=1), dict(use_graph=False),
               dict(threads_per_cta=128, ctas_per_sm=1, use_graph=False)]:
        st, ri = run([(11, n)], **kw)
        assert int_view(st) == int_view(ref), kw
        assert ri == rref, kw
    st, ri = run([(11, 1), (12, 3), (15, 5), (20, n - 9)])
    assert int_view(st) == int_view(ref)
    assert ri == rref


def test_batched_points_equal_single_point_runs(T):
    """Three K = 128 points with uneven budgets in one persistent launch give
    the statistics of three separate handles."""
    K = 128
    cfg = [(60.0, 1.0, 150.0, O.PAPER, 0, 70_001), (30.0, 0.7, 300.0, O.PAPER, 1, 150_002),
           (20.0, 1.5, 450.0, O.UNIFORM, 2, 9_999)]
    pts = []
    for bp, E0, r, prop, pid, _ in cfg:
        lm = rate_logM(K, E0, bp, r, prop, 1, pid, 0.05)
        pts.append(T.make_point(bp, E0, r, tprop(T, prop), point_id=pid, logM=lm))
    S = T.Sampler(K, pts, sample_capacity=1 << 16)
    S.run_budgets([c[-1] for c in cfg], 99)
    st = S.stats()
    S.close()
    for p, c in enumerate(cfg):
        S1 = T.Sampler(K, [pts[p]], sample_capacity=1 << 16)
        S1.run_budgets([c[-1]], 99)
        s1 = S1.stats()[0]
        S1.close()
        assert int_view(st[p]) == int_view(s1), p


def test_replay_of_tail_draws_matches_oracle(T):
    """Draws with a radius or accept word in the lowest bucket of the uniform
    map go to the FP64 pass, which refines the word; their values and
    decisions against the oracle."""
    K, seed, pid, E0, bp, r = 128, 5, 9, 1.0, 60.0, 150.0
    idx, tot = O.tail_scan(K, seed, pid, 0, 1 << 21, which=3)
    assert tot >= 5
    pt0 = O.make_point(K, E0, bp, r, O.PAPER)
    lm = float(np.quantile(O.replay(pt0, seed, pid, idx)["logfg"], 0.6))
    S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=pid, logM=lm)], sample_capacity=16)
    g = S.replay(0, idx, seed)
    S.close()
    o = O.replay(O.make_point(K, E0, bp, r, O.PAPER, logM=lm), seed, pid, idx)
    assert np.all(g["flags"] != 0)
    assert np.all(np.abs(g["delta"] - o["delta"]) <= 1e-9 * (1 + np.abs(o["delta"])))
    assert np.all(np.abs(g["lnU"] - o["lnU"]) <= 1e-12 * (1 + np.abs(o["lnU"])))
    assert np.all(np.abs(g["xhat"] - o["xhat"][:, :2 * K]) <= 1e-6)
    assert np.array_equal(g["accept"], o["accept"])


def test_deep_accepts_follow_closed_form(T):
    """Uniform proposal at beta' = 0 with log M = 17: every draw has Delta = -17
    and is accepted with probability e^-17; only accept words in the refined
    lowest bucket can be accepted."""
    K, L, n, seed, pid = 128, 17.0, 1 << 30, 21, 4
    S = T.Sampler(K, [T.make_point(0.0, 1.0, 0.0, T.PROPOSAL_UNIFORM, point_id=pid, logM=L)],
                  sample_capacity=1 << 12)
    S.run_ranges([0], [n], seed)
    st = S.stats()[0]
    rec = S.samples(1 << 12)
    S.close()
    mean = n * math.exp(-L)
    assert st["n_proposals"] == n and abs(st["n_accepted"] - mean) <= 5 * math.sqrt(mean)
    pt = O.make_point(K, 1.0, 0.0, 0.0, O.UNIFORM, logM=L)
    o = O.replay(pt, seed, pid, rec["idx"])
    assert np.all(o["accept"]) and np.all(o["lnU"] < -L)
    # on a prefix the accepted set is exactly the oracle's: the candidates are
    # the indices whose accept word is in the lowest bucket
    m = 1 << 27
    cand, tot = O.tail_scan(K, seed, pid, 0, m, which=2)
    oc = O.replay(pt, seed, pid, cand)
    want = set(int(i) for i in cand[oc["accept"]])
    assert set(int(i) for i in rec["idx"] if int(i) < m) == want
    print("K=128: %d accepts of 2^30 at Delta = -17 (expected %.1f)" % (st["n_accepted"], mean))


def test_static_entry_matches_handle(T):
    """The allocation-free entry point runs the warp form at K = 128 and
    returns what the handle returns."""
    import torch
    K, E0, bp, r, seed = 128, 1.0, 60.0, 150.0, 4
    lm = rate_logM(K, E0, bp, r, O.PAPER, seed, 0, 0.02)
    point = T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=0, logM=lm)
    rb, cap, n = T.tkdv_record_bytes(K), 1 << 14, T.STATIC_MAX_PROPOSALS - 5
    buf = torch.zeros(cap * rb, dtype=torch.uint8, device="cuda")
    st_s, nrec = T.sampler_run_static(K, point, 0, n, seed, buf, cap)
    rec_s = T.decode_records(buf[: nrec * rb].cpu().numpy(), K)
    S = T.Sampler(K, [point], sample_capacity=cap)
    S.run_ranges([0], [n], seed)
    st_h, rec_h = S.stats()[0], S.samples(cap)
    S.close()
    for key in ("n_proposals", "n_accepted", "n_refined", "n_near_threshold", "n_envelope_violations"):
        assert st_s[key] == st_h[key], key
    assert np.array_equal(np.sort(rec_s["idx"]), np.sort(rec_h["idx"]))


def test_library_envelope_has_no_violations(T):
    """The library's own log M at K = 128 (L-BFGS over the 256-dimensional
    sphere) bounds log f/g on 2^24 proposals of the paper proposal."""
    K, E0, bp, r = 128, 1.0, 60.0, 150.0
    S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER)], sample_capacity=1 << 16)
    S.run(1 << 24, 8)
    st = S.stats()[0]
    S.close()
    assert st["n_envelope_violations"] == 0 and st["max_delta"] < 0
    print("K=128 library envelope: log M %.4f, acceptance %.3g, max delta %.3f" % (
        st["logM"], st["n_accepted"] / st["n_proposals"], st["max_delta"]))


def test_learned_corrections_at_K128(T):
    """Per-mode log-variance corrections supplied directly (the learned
    proposal's form; the network itself stops at 64 modes) at K = 128: the
    oracle's diagonal proposal with the same variances gives the same accept
    set, and the library's envelope bounds log f/g on every draw of the run."""
    K, bp, E0, r, seed, pid = 128, 40.0, 1.0, 225.0, 6, 3
    k = np.arange(1, K + 1)
    c = 0.3 * np.cos(math.pi * k / K) - 0.1 * np.sin(3 * math.pi * k / K)
    a = O.alpha_star(K, bp)
    s2 = (1.0 / (1.0 + a * bp * k * k / K**3)) * np.exp(c)
    pt0 = O.make_point(K, E0, bp, r, O.DIAG, sigma2=s2)
    lf = O.replay(pt0, seed, pid, np.arange(2048, dtype=np.uint64))["logfg"]
    lm = float(lf.max() + np.log(np.mean(np.exp(lf - lf.max()))) - np.log(0.03))
    pt = O.make_point(K, E0, bp, r, O.DIAG, sigma2=s2, logM=lm)
    S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_LEARNED, point_id=pid, logM=lm, log_var_correction=c)],
                  sample_capacity=1 << 16)
    _, _, s2_lib = S.point_info(0)
    assert np.allclose(s2_lib, s2, rtol=1e-13)
    n = 1 << 17
    S.run_ranges([0], [n], seed)
    st = S.stats()[0]
    rec = S.samples(1 << 16)
    S.close()
    total, orec = O.run_accepted(pt, seed, pid, 0, n, cap=1 << 16)
    excused = compare_accept_sets(rec["idx"], pt, seed, pid, orec["idx"])
    assert abs(st["n_accepted"] - total) <= excused and total > 1000
    common = np.isin(rec["idx"], orec["idx"])
    check_records_against_oracle({kk: v[common] for kk, v in rec.items()}, orec, r, K)
    S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_LEARNED, point_id=pid, log_var_correction=c)],
                  sample_capacity=16)
    S.run(1 << 22, seed)
    st = S.stats()[0]
    S.close()
    assert st["n_envelope_violations"] == 0 and st["max_delta"] < 0

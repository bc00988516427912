"""Parity of the CUDA sampler (through the C ABI) with the FP64 oracle.

Tolerances (per sample, FP32 fast path):
  * H = H2 - (C3/C2) H3 within 1e-5 (|H2| + |C3/C2 H3|) of the oracle, and
    H2 within 1e-5 relative;
  * log f/(Mg) within 2e-5 (1 + |beta' S/K^2| + |K ln Q| + |log M|) + 2e-5 |c_H| sqrt(K);
  * accept decisions identical, except draws the oracle puts within 1e-6 of
    the threshold (counted and reported);
  * statistics: integer counts identical where the accepted sets are, moment
    sums within FP32 rounding of u0, histogram bins within the draws whose u0
    lies within 1e-5 of a bin edge.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

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


_ENV = None


def envelope(K, E0, bp, r, prop):
    """Oracle log M: from tests/golden/envelopes.json when listed, else computed."""
    global _ENV
    if _ENV is None:
        path = os.path.join(HERE, "golden", "envelopes.json")
        _ENV = json.load(open(path))["points"] if os.path.exists(path) else {}
    key = "K%d_E%.17g_b%.17g_r%.17g_p%d" % (K, E0, bp, r, prop)
    if key in _ENV:
        return _ENV[key]["logM"]
    pt = O.make_point(K, E0, bp, r, prop)
    return O.log_M(pt, 2)


def tprop(T, prop):
    return T.PROPOSAL_PAPER if prop == O.PAPER else T.PROPOSAL_UNIFORM


def check_records_against_oracle(rec, orc, r, K):
    """Per-record H, u0 and xhat of GPU records vs oracle replay of the same indices."""
    o = {int(i): j for j, i in enumerate(orc["idx"])}
    j = np.array([o[int(i)] for i in rec["idx"]])
    H2o, H3o = orc["H2"][j], orc["H3"][j]
    scale = np.abs(H2o) + np.abs(r * H3o)
    Hg = rec["H2"].astype(np.float64) - r * rec["H3"].astype(np.float64)
    Ho = H2o - r * H3o
    assert np.all(np.abs(Hg - Ho) <= 1e-5 * scale), np.max(np.abs(Hg - Ho) / scale)
    assert np.all(np.abs(rec["H2"] - H2o) <= 1e-5 * np.abs(H2o))
    assert np.all(np.abs(rec["u0"] - orc["u0"][j]) <= 1e-5 * (1 + np.abs(orc["u0"][j])))
    assert np.all(np.abs(rec["xhat"] - orc["xhat"][j][:, :2 * K]) <= 2e-6)


def compare_accept_sets(gpu_idx, pt, seed, pid, orc_idx):
    """Accepted index sets must agree except draws the oracle puts within 1e-6
    of the threshold.  Returns the number of such excused draws."""
    g, o = set(int(i) for i in gpu_idx), set(int(i) for i in orc_idx)
    diff = sorted((g - o) | (o - g))
    if not diff:
        return 0
    rep = O.replay(pt, seed, pid, np.array(diff, dtype=np.uint64))
    assert np.all(rep["near"]), [d for d, nr in zip(diff, rep["near"]) if not nr][:10]
    return len(diff)


# ---------------------------------------------------------------- full replay
@pytest.mark.parametrize("prop", [O.PAPER, O.UNIFORM])
def test_small_k16_full_replay(T, prop):
    """K = 16, beta' = 20, C3/C2 = 75, E0 = 1, 2^20 proposals, seed 0: every proposal
    of the persistent launch is replayed by the oracle."""
    K, E0, bp, r, n, seed = 16, 1.0, 20.0, 75.0, 1 << 20, 0
    lm = envelope(K, E0, bp, r, prop)
    S = T.Sampler(K, [T.make_point(bp, E0, r, tprop(T, prop), point_id=0, logM=lm)], sample_capacity=1 << 18)
    S.run_ranges([0], [n], seed)
    st = S.stats()[0]
    rec = S.samples(1 << 18)
    S.close()
    pt = O.make_point(K, E0, bp, r, prop, logM=lm)
    total, orec = O.run_accepted(pt, seed, 0, 0, n, cap=1 << 18)
    ost = O.run_stats(pt, seed, 0, 0, n)
    assert st["n_proposals"] == n and st["n_dropped"] == 0 and st["n_fallback"] == 0
    assert st["n_accepted"] == len(rec["idx"])
    excused = compare_accept_sets(rec["idx"], pt, seed, 0, orec["idx"])
    assert abs(st["n_accepted"] - total) <= excused
    assert st["n_near_threshold"] == ost["n_near"]
    assert st["n_envelope_violations"] == 0 and ost["n_viol"] == 0
    common = np.isin(rec["idx"], orec["idx"])
    sub = {k: v[common] for k, v in rec.items()}
    check_records_against_oracle(sub, orec, r, K)
    # statistics
    if excused == 0:
        for q in range(4):
            assert abs(st["sum_u0"][q] - ost["sum_u0"][q]) <= 2e-6 * (1 + abs(ost["sum_u0"][q])) + 1e-6 * total
        # power spectrum (Sec. V.A): FP32 s_k per accept, each rounded to 2^-28
        spec_tol = 2e-6 * ost["spectrum"] + total * 2.0**-28 + 1e-9
        assert np.all(np.abs(st["spectrum"][:K] - ost["spectrum"]) <= spec_tol)
        edges = np.linspace(st["hist_lo"], st["hist_hi"], 257)
        near_edge = np.sum(np.min(np.abs(orec["u0"][:, None] - edges[None, :]), axis=1) < 1e-5)
        assert int(np.sum(np.abs(st["hist"].astype(np.int64) - ost["hist"].astype(np.int64)))) <= 2 * near_edge
        thr = 0.25 * np.arange(25) * math.sqrt(E0 / math.pi)
        near_thr = np.sum(np.min(np.abs(orec["u0"][:, None] - thr[None, :]), axis=1) < 1e-5)
        assert int(np.sum(np.abs(st["exceed"].astype(np.int64) - ost["exceed"].astype(np.int64)))) <= 25 * near_thr
    print("K16 prop=%d: accepted %d, refined %d, near %d, excused %d" % (
        prop, st["n_accepted"], st["n_refined"], st["n_near_threshold"], excused))


# ------------------------------------------------------------ per-stage replay
REPLAY_CASES = [(1, 0.6, 0.5, 10.0), (2, 1.3, 3.0, 40.0), (3, 1.0, 5.0, 30.0), (5, 0.8, 10.0, 60.0),
                (8, 1.0, 30.0, 50.0), (16, 1.0, 20.0, 75.0), (17, 2.0, 25.0, 40.0), (32, 1.0, 40.0, 225.0),
                (64, 1.0, 40.0, 400.0), (100, 1.0, 40.0, 225.0), (128, 1.0, 60.0, 150.0)]


@pytest.mark.parametrize("K,E0,bp,r", REPLAY_CASES)
@pytest.mark.parametrize("prop", [O.PAPER, O.UNIFORM])
def test_replay_per_stage(T, K, E0, bp, r, prop):
    """Delta, ln U, H2, H3, u0, xhat and accept bit of sampled proposals (indices
    across the 32-bit boundary, point id 7) against the oracle."""
    seed, pid = (1 << 40) + 3, 7
    rng = np.random.default_rng(K * 10 + prop)
    idx = np.concatenate([np.arange(64), rng.integers(0, 1 << 34, 2000), (1 << 32) + np.arange(32)]).astype(np.uint64)
    pt0 = O.make_point(K, E0, bp, r, prop)
    # an envelope that accepts about a third of the draws makes every branch run
    rep0 = O.replay(pt0, seed, pid, idx[:256])
    lm = float(np.quantile(rep0["logfg"], 0.6))
    pt = O.make_point(K, E0, bp, r, prop, logM=lm)
    S = T.Sampler(K, [T.make_point(bp, E0, r, tprop(T, prop), point_id=pid, logM=lm)], sample_capacity=16)
    g = S.replay(0, idx, seed)
    S.close()
    o = O.replay(pt, seed, pid, idx)
    fast = g["flags"] == 0
    cQ = 0.0 if prop == O.UNIFORM else K
    S_o = o["S"]
    Q_term = np.abs(o["logfg"] + bp * S_o / K**2 - bp * r / (E0 * K**2) * o["H3"])
    cH = abs(bp * r / (E0 * K**2) * 2 * math.pi * (E0 / (2 * math.pi)) ** 1.5)
    tol = 2e-5 * (1 + bp * S_o / K**2 + Q_term + abs(lm) + np.abs(o["lnU"])) + 2e-5 * cH * math.sqrt(K) + 2e-5 * cQ
    err = np.abs(g["delta"] - o["delta"])
    assert np.all(err[fast] <= tol[fast]), np.max(err[fast] / tol[fast])
    assert np.all(err[~fast] <= 1e-9 * (1 + np.abs(o["delta"][~fast])))
    assert np.all(np.abs(g["lnU"] - o["lnU"]) <= 2e-6 * (1 + np.abs(o["lnU"])))
    assert np.all(np.abs(g["S"] - o["S"]) <= 1e-5 * o["S"])
    scale = np.abs(o["H2"]) + np.abs(r * o["H3"])
    assert np.all(np.abs((g["H2"] - r * g["H3"]) - (o["H2"] - r * o["H3"])) <= 1e-5 * scale)
    assert np.all(np.abs(g["u0"] - o["u0"]) <= 1e-5 * (1 + np.abs(o["u0"])))
    assert np.all(np.abs(g["xhat"] - o["xhat"][:, :2 * K]) <= 2e-6)
    bad = (g["accept"] != o["accept"]) & ~o["near"]
    assert not np.any(bad), idx[bad][:10]


# ----------------------------------------------------- launch-shape invariance
def run_stats_and_idx(T, K, pts, ranges, seed, **kw):
    S = T.Sampler(K, pts, sample_capacity=1 << 18, **kw)
    for (i0, c) in ranges:
        S.run_ranges(i0, c, seed)
    st = S.stats()
    rec = S.samples(1 << 18)
    S.close()
    return st, rec


def int_view(st):
    return (st["n_proposals"], st["n_accepted"], st["n_refined"], st["n_near_threshold"],
            st["n_envelope_violations"], tuple(st["hist"].tolist()), tuple(st["exceed"].tolist()),
            tuple(np.round(st["sum_u0"] * np.array([2.0**28, 2.0**24, 2.0**20, 2.0**16])).astype(np.int64)))


def test_launch_shape_and_resume_invariance(T):
    """The accepted set and every integer statistic are functions of
    (parameters, seed, index range) only: threads, CTAs, graph or not, and
    splitting a range into several runs change nothing."""
    K, E0, bp, r = 16, 1.0, 20.0, 75.0
    lm = envelope(K, E0, bp, r, O.PAPER)
    pts = [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=3, logM=lm)]
    n = 3_000_001
    ref, rref = run_stats_and_idx(T, K, pts, [([5], [n])], 11)
    variants = [dict(threads_per_cta=128), dict(ctas_per_sm=1), dict(use_graph=False),
                dict(threads_per_cta=128, ctas_per_sm=1, use_graph=False)]
    for kw in variants:
        st, rec = run_stats_and_idx(T, K, pts, [([5], [n])], 11, **kw)
        assert int_view(st[0]) == int_view(ref[0]), kw
        assert set(rec["idx"].tolist()) == set(rref["idx"].tolist())
    st, rec = run_stats_and_idx(T, K, pts, [([5], [1_000_000]), ([1_000_005], [1]), ([1_000_006], [n - 1_000_001])], 11)
    assert int_view(st[0]) == int_view(ref[0])
    assert set(rec["idx"].tolist()) == set(rref["idx"].tolist())


def test_batched_points_equal_single_point_runs(T):
    """Three points with uneven budgets in one persistent launch give the same
    statistics as three separate handles."""
    K = 16
    cfg = [(20.0, 1.0, 75.0, O.PAPER, 0, 300_000), (40.0, 0.7, 30.0, O.PAPER, 1, 1_200_000),
           (20.0, 1.5, 60.0, O.UNIFORM, 2, 50_000)]
    pts = []
    for bp, E0, r, prop, pid, _ in cfg:
        pts.append(T.make_point(bp, E0, r, tprop(T, prop), point_id=pid, logM=envelope(K, E0, bp, r, prop)))
    S = T.Sampler(K, pts, sample_capacity=1 << 16)
    S.run_budgets([c[-1] for c in cfg], 99)
    st = S.stats()
    S.close()
    for p, c in enumerate(cfg):
        s1, _ = run_stats_and_idx(T, K, [pts[p]], [([0], [c[-1]])], 99)
        assert int_view(st[p]) == int_view(s1[0]), p


# ------------------------------------------------------------- edge cases
def test_beta_zero_accepts_everything(T):
    for prop in (T.PROPOSAL_UNIFORM, T.PROPOSAL_PAPER):
        S = T.Sampler(8, [T.make_point(0.0, 1.0, 50.0, prop)], sample_capacity=4)
        S.run(100_000, 1)
        st = S.stats()[0]
        S.close()
        assert st["logM"] == pytest.approx(0.0, abs=1e-12)
        assert st["n_accepted"] == 100_000 and st["n_dropped"] == 100_000 - 4


def test_empty_and_tiny_runs(T):
    S = T.Sampler(4, [T.make_point(3.0, 1.0, 20.0, T.PROPOSAL_PAPER)], sample_capacity=8)
    S.run(0, 1)
    assert S.stats()[0]["n_proposals"] == 0
    S.run(1, 1)
    S.run(7, 1)
    st = S.stats()[0]
    assert st["n_proposals"] == 8
    S.reset()
    assert S.stats()[0]["n_proposals"] == 0
    S.close()


def test_deadline_reports_timeout(T):
    S = T.Sampler(16, [T.make_point(20.0, 1.0, 75.0, T.PROPOSAL_PAPER)])
    S.set_deadline_ns(1)
    S.run(1 << 26, 1)
    with pytest.raises(T.TkdvError) as ei:
        S.sync()
    assert ei.value.code == -5
    st = S.stats()[0]
    assert st["n_proposals"] < 1 << 26
    S.set_deadline_ns(0)
    S.reset()
    S.run(1 << 16, 1)
    S.sync()
    assert S.stats()[0]["n_proposals"] == 1 << 16
    S.close()


def test_envelope_violation_is_counted(T):
    """An envelope below the true maximum shows up as envelope violations."""
    K, E0, bp, r = 8, 1.0, 30.0, 50.0
    lm = envelope(K, E0, bp, r, O.PAPER)
    S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, logM=lm - 3.0)])
    S.run(1 << 20, 5)
    st = S.stats()[0]
    S.close()
    assert st["n_envelope_violations"] > 0 and st["max_delta"] > 0


def test_library_envelope_has_no_violations(T):
    K, E0, bp, r = 16, 1.0, 20.0, 75.0
    S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER)])
    S.run(1 << 22, 8)
    st = S.stats()[0]
    S.close()
    assert abs(st["logM"] - envelope(K, E0, bp, r, O.PAPER)) < 1e-8
    assert st["n_envelope_violations"] == 0 and st["max_delta"] < 0


# ---------------------------------------------- K = 2 acceptance by quadrature
@pytest.mark.parametrize("prop", [O.UNIFORM, O.PAPER])
def test_k2_acceptance_matches_quadrature(T, prop):
    from tests.test_oracle_pins import k2_reduced
    from scipy import integrate, optimize, special
    E0, bp, r = 1.0, 3.0, 40.0
    ell, w, c = k2_reduced(E0, bp, r, prop)
    res = optimize.minimize_scalar(lambda p: -max(ell(p, 0.0), ell(p, math.pi)), bounds=(0, math.pi / 2),
                                   method="bounded", options={"xatol": 1e-12})
    phis = np.linspace(0, math.pi / 2, 4001)
    logM = max(-res.fun, max(max(ell(p, 0.0), ell(p, math.pi)) for p in phis))

    def integrand(phi):
        s1, s2 = math.cos(phi) ** 2, math.sin(phi) ** 2
        amp = bp / (E0 * 4) * r * 2 * math.pi * c**3 * s1 * math.sin(phi)
        return math.sin(2 * phi) * math.exp(-bp / 4 * (s1 + 4 * s2)) * special.i0(amp)

    Z = integrate.quad(integrand, 0, math.pi / 2, epsabs=1e-14, epsrel=1e-12)[0]
    acc = Z * (w[0] * w[1] if prop == O.PAPER else 1.0) * math.exp(-logM)
    n = 1 << 24
    S = T.Sampler(2, [T.make_point(bp, E0, r, tprop(T, prop), logM=logM)], sample_capacity=4)
    S.run(n, 77)
    st = S.stats()[0]
    S.close()
    p = st["n_accepted"] / n
    assert abs(p - acc) < 4 * math.sqrt(acc * (1 - acc) / n), (p, acc)
    assert st["n_envelope_violations"] == 0


def test_raw_records_into_host_buffer(T):
    """sampler_samples into a caller-owned pinned host buffer returns the same
    raw records the decoding call returns."""
    import torch
    K, E0, bp, r = 16, 1.0, 20.0, 75.0
    lm = envelope(K, E0, bp, r, O.PAPER)
    S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, logM=lm)], sample_capacity=1 << 14)
    S.run(1 << 20, 4)
    rb = T.tkdv_record_bytes(K)
    host = torch.empty((1 << 14) * rb, dtype=torch.uint8, pin_memory=True)
    n = S.samples(1 << 14, host_dst=host)
    rec = S.samples(1 << 14)
    with pytest.raises(ValueError):
        S.samples(1 << 14, host_dst=torch.empty(rb, dtype=torch.uint8))
    S.close()
    assert n == len(rec["idx"]) > 0
    raw = T.decode_records(host[: n * rb].numpy(), K)
    for key in ("idx", "point", "flags", "H2", "H3", "u0", "delta", "xhat"):
        assert np.array_equal(raw[key], rec[key]), key


def test_auto_form_takes_the_exact_decisions_of_both_forms(T):
    """TKDV_H3_AUTO: the grid form before autotuning (K <= 64 on this device),
    the faster form after it; every form accepts the same draws.  K = 128 and
    SIR runs take the triad form."""
    K, E0, bp, r, n, seed = 16, 1.0, 20.0, 75.0, 1 << 21, 8
    pts = [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=2, logM=envelope(K, E0, bp, r, O.PAPER))]
    sets, views = {}, {}
    for mode in (T.H3_TRIAD_F32, T.H3_GRID_BF16X3, T.H3_AUTO):
        S = T.Sampler(K, pts, h3_mode=mode, sample_capacity=1 << 16)
        if mode == T.H3_AUTO:
            assert S.h3_form() == T.H3_GRID_BF16X3
            S.autotune(1 << 20)
            assert S.h3_form() in (T.H3_TRIAD_F32, T.H3_GRID_BF16X3)
        S.run_ranges([0], [n], seed)
        st = S.stats()[0]
        sets[mode] = set(S.samples(1 << 16)["idx"].tolist())
        views[mode] = (st["n_proposals"], st["n_accepted"], st["n_envelope_violations"])
        S.close()
    pt = O.make_point(K, E0, bp, r, O.PAPER, logM=pts[0].logM)
    for mode in (T.H3_GRID_BF16X3, T.H3_AUTO):
        diff = sorted(sets[mode] ^ sets[T.H3_TRIAD_F32])
        if diff:
            assert O.replay(pt, seed, 2, np.array(diff, dtype=np.uint64))["near"].all()
    assert views[T.H3_AUTO][0] == n
    S = T.Sampler(128, [T.make_point(60.0, 1.0, 150.0, T.PROPOSAL_PAPER, logM=10.0)], h3_mode=T.H3_AUTO)
    assert S.h3_form() == T.H3_TRIAD_F32
    S.close()
    S = T.Sampler(16, [T.make_point(20.0, 1.0, 75.0, T.PROPOSAL_PAPER, logM=envelope(K, E0, bp, r, O.PAPER))],
                  h3_mode=T.H3_AUTO, sir=True)
    assert S.h3_form() == T.H3_TRIAD_F32
    S.close()


def test_batch_run_equals_a_handle(T):
    """sampler_batch_run (create, run, statistics, destroy in one call) gives
    the statistics of a handle run on the same points, budgets and seed."""
    K = 16
    cfg = [(20.0, 1.0, 75.0, O.PAPER, 0, 300_001), (40.0, 0.7, 30.0, O.PAPER, 1, 100_000)]
    pts = [T.make_point(bp, E0, r, tprop(T, prop), point_id=pid, logM=envelope(K, E0, bp, r, prop))
           for bp, E0, r, prop, pid, _ in cfg]
    budgets = [c[-1] for c in cfg]
    out = T.sampler_batch_run(pts, T.make_options(K, sample_capacity=16), budgets, 5)
    S = T.Sampler(K, pts, sample_capacity=16)
    S.run_budgets(budgets, 5)
    ref = S.stats()
    S.close()
    for p in range(len(cfg)):
        assert int_view(out[p]) == int_view(ref[p]), p
    with pytest.raises(T.TkdvError):
        T.sampler_batch_run(pts, T.make_options(200), budgets, 5)


def test_every_launch_variant_gives_the_same_results(T):
    """Each pinned launch shape (the six triad-form variants, one and the
    most CTAs per SM) gives the same statistics and the same records at an
    acceptance where most warp iterations hold an accepted draw."""
    K, E0, bp, r, n, seed = 16, 1.0, 20.0, 75.0, 1 << 20, 6
    lm = envelope(K, E0, bp, r, O.PAPER) - 2.5  # log M lowered: about 12 % accepted
    pts = [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=4, logM=lm)]
    ref = None
    for variant in range(6):
        for per in (1, 0):
            S = T.Sampler(K, pts, sample_capacity=1 << 18)
            S.set_launch(variant, per)
            S.run_ranges([3], [n], seed)
            st = S.stats()[0]
            rec = S.samples(1 << 18)
            S.close()
            o = np.argsort(rec["idx"])
            view = (int_view(st), tuple(np.round(st["spectrum"][:K] * 2.0**28).astype(np.int64).tolist()))
            if ref is None:
                ref, rref = view, {k: v[o] for k, v in rec.items()}
                assert st["n_accepted"] > 10000
                continue
            assert view == ref, (variant, per)
            for key in ("idx", "H2", "H3", "u0", "xhat"):
                assert np.array_equal(rec[key][o], rref[key]), (variant, per, key)
    S = T.Sampler(K, pts, sample_capacity=16)
    with pytest.raises(T.TkdvError):
        S.set_launch(6, 0)
    with pytest.raises(T.TkdvError):
        S.set_launch(0, 64)
    S.close()

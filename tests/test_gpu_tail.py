"""The refined tail of the uniform map on the GPU, and the FP32 radius bound.

A radius or accept word in the lowest bucket of the uniform map (w < 512) is
refined from further Philox blocks, so U stays uniform down to 2^-70.  The
FP32 fast paths only detect such draws and send them to the FP64 pass.
These tests pin that path against the oracle and against a closed form.

Closed form: for the uniform proposal at beta' = 0 every draw has
log f/g = 0, so with the envelope set to log M = L every draw has
Delta = -L and is accepted with probability e^-L exactly.  For L = 17 only
draws whose accept word is in the lowest bucket (U < 2^-23 < e^-16.64) can
be accepted; without the refinement none would be.
"""
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


@pytest.mark.parametrize("K,grid_N", [(8, 0), (32, 0), (16, 64), (32, 128)])
def test_deep_accepts_follow_closed_form(T, K, grid_N):
    L, n, seed, pid = 17.0, 1 << 31, 21, 4
    mode = T.H3_GRID_BF16X3 if grid_N else T.H3_TRIAD_F32
    S = T.Sampler(K, [T.make_point(0.0, 1.0, 0.0, T.PROPOSAL_UNIFORM, point_id=pid, logM=L)],
                  h3_mode=mode, grid_N=grid_N, sample_capacity=1 << 12)
    S.run_ranges([0], [n], seed)
    st = S.stats()[0]
    rec = S.samples(1 << 12)
    S.close()
    mean = n * math.exp(-L)
    assert st["n_proposals"] == n and st["n_dropped"] == 0
    assert abs(st["n_accepted"] - mean) <= 5 * math.sqrt(mean), (st["n_accepted"], mean)
    assert len(rec["idx"]) == st["n_accepted"]
    # every accepted draw is one the oracle accepts, with ln U below -L
    pt = O.make_point(K, 1.0, 0.0, 0.0, O.UNIFORM, logM=L)
    o = O.replay(pt, seed, pid, rec["idx"])
    assert np.all(o["accept"]) and np.all(o["lnU"] < -L)
    # on a prefix the accepted set is exactly the oracle's: the candidates are
    # the indices whose accept word is in the lowest bucket
    m = 1 << 25
    cand, tot = O.tail_scan(K, seed, pid, 0, m, which=2)
    oc = O.replay(pt, seed, pid, cand)
    want = set(int(i) for i in cand[oc["accept"]])
    got = set(int(i) for i in rec["idx"] if int(i) < m)
    assert got == want
    print("K=%d N=%d: %d accepts of 2^31 at Delta = -17 (expected %.1f); prefix: %d candidates, %d accepted"
          % (K, grid_N, st["n_accepted"], mean, tot, len(want)))


@pytest.mark.parametrize("K,prop", [(8, O.PAPER), (16, O.UNIFORM)])
def test_replay_of_tail_draws_matches_oracle(T, K, prop):
    """Draws with a refined radius or accept word: the device FP64 path
    against the oracle, value by value."""
    seed, pid, E0, bp, r = 5, 9, 1.0, 30.0, 50.0
    idx, tot = O.tail_scan(K, seed, pid, 0, 1 << 25, which=3)
    assert tot >= 5
    pt0 = O.make_point(K, E0, bp, r, prop)
    lm = float(np.quantile(O.replay(pt0, seed, pid, idx)["logfg"], 0.6))
    pt = O.make_point(K, E0, bp, r, prop, logM=lm)
    tp = T.PROPOSAL_PAPER if prop == O.PAPER else T.PROPOSAL_UNIFORM
    S = T.Sampler(K, [T.make_point(bp, E0, r, tp, point_id=pid, logM=lm)], sample_capacity=16)
    g = S.replay(0, idx, seed)
    S.close()
    o = O.replay(pt, seed, pid, idx)
    assert np.all(g["flags"] != 0)  # all decided by the FP64 pass
    assert np.all(np.abs(g["delta"] - o["delta"]) <= 1e-9 * (1 + np.abs(o["delta"])))
    assert np.all(np.abs(g["lnU"] - o["lnU"]) <= 1e-12 * (1 + np.abs(o["lnU"])))
    assert np.all(np.abs(g["xhat"] - o["xhat"][:, :2 * K]) <= 1e-6)
    assert np.array_equal(g["accept"], o["accept"])
    # the refined words reach beyond the old floor of the map
    rho_max = []
    for i in idx:
        z, u = O.stream(K, seed, pid, int(i))
        rho_max.append(max(np.max(z[:K] ** 2 + z[K:] ** 2), -2 * math.log(u)))
    rho_max = np.array(rho_max)
    assert np.all(rho_max >= -2 * math.log(2.0**-23) - 1e-9)
    assert np.any(rho_max > -2 * math.log(2.0**-24) + 1e-6)


def test_fast_paths_defer_every_tail_draw(T):
    """Triad and grid forms send every draw with a word in the lowest bucket to
    the FP64 pass (n_refined counts them), accept what the oracle accepts,
    and the grid form's trace marks exactly the oracle's tail draws."""
    import torch
    seed, pid, E0, bp, r = 3, 2, 1.0, 20.0, 75.0
    for K, N in [(8, 0), (16, 64)]:
        n = 1 << 25
        tails, tot = O.tail_scan(K, seed, pid, 0, n, which=3)
        pt0 = O.make_point(K, E0, bp, r, O.PAPER)
        lm = O.log_M(pt0, 1)
        pt = O.make_point(K, E0, bp, r, O.PAPER, logM=lm)
        mode = T.H3_GRID_BF16X3 if N else T.H3_TRIAD_F32
        S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=pid, logM=lm)], h3_mode=mode,
                      grid_N=N, sample_capacity=1 << 22)
        S.run_ranges([0], [n], seed)
        st = S.stats()[0]
        rec = S.samples(1 << 22)
        S.close()
        assert st["n_refined"] >= tot
        # the tail draws themselves: the GPU accepted exactly those the oracle accepts
        o = O.replay(pt, seed, pid, tails)
        g_acc = set(int(i) for i in rec["idx"]) & set(int(i) for i in tails)
        assert g_acc == set(int(i) for i in tails[o["accept"]])
        if N:
            nw = 4096
            i0 = max(0, int(tails[0]) - 1000)
            S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=pid, logM=lm)], h3_mode=mode,
                          grid_N=N, sample_capacity=1 << 12)
            tr = torch.zeros(2 * nw, dtype=torch.float32, device="cuda")
            S.set_trace(tr, nw)
            S.run_ranges([i0], [nw], seed)
            S.sync()
            S.close()
            tr = tr.cpu().numpy().reshape(nw, 2)
            nan_idx = set((i0 + np.nonzero(np.isnan(tr[:, 0]))[0]).tolist())
            want = set(int(i) for i in tails if i0 <= int(i) < i0 + nw)
            assert nan_idx == want and len(want) >= 1
        print("K=%d N=%d: %d tail draws in 2^25, refined %d" % (K, N, tot, st["n_refined"]))


def test_fast_path_radius_error_bound(T):
    """The FP32 radius -2 ln u of the fast path stays within the error bound
    2^-21 + 2^-21 rho that the accept guard band is built on, over all 2^23
    values of the uniform map."""
    ratio, w = T.tkdv_check_radius_error()
    assert ratio <= 1.0, (ratio, w)
    print("radius: largest error / bound = %.3f at word %#x" % (ratio, w))


def test_warp_form_radius_error_bound(T):
    """The warp form's FP32 radius -2 logf(u) stays within the purely relative
    bound 2^-22 rho its guard band is built on, over all 2^23 values of the
    uniform map."""
    ratio, w = T.tkdv_check_radius_error_log()
    assert ratio <= 1.0, (ratio, w)
    print("log radius: largest error / bound = %.3f at word %#x" % (ratio, w))

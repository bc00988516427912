"""The FP32 decision guard holds on every draw.

A draw outside the guard band is decided in FP32, so exact decisions need the
band to cover the FP32 error of log f/(Mg) on every draw, not only on those
near the threshold.  Here the fast path's log f/(Mg) (replay rows decided in
FP32; the grid form's trace) is compared with the oracle's FP64 value, and
the error must stay below the band, recomputed on the host from the formula
the kernels use (point_table.cpp):
  guard = g_e E/|x| + g_q/|x|^2 + g_a + g_r (|tS| + |tQ| + |tH| + |ln U| + |log M|) + g_h,
with E = sum_m sigma_m / sqrt(rho_m).  The ratio error / guard is printed;
it should sit well below 1.
"""
import math

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
EPS = 2.0**-24


@pytest.fixture(scope="module")
def T():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_16952_gb300 import _build
    _build.build()
    import paper_2411_16952_gb300 as T
    return T


def host_guard(K, prop, bp, E0, r, logM, o, idx, seed, pid, grid_N=0):
    warp = K > 64
    rel = 2.0**-22 if warp else 2.0**-21
    abs_err = 0.0 if warp else 2.0**-21
    gam = 8.0 * (32.0 if warp else 2.0 * K + 16.0) * EPS + 4.0 * rel
    gam_t = 8.0 * (64.0 if warp else 2.0 * K + 16.0) * EPS + 4.0 * rel
    pt = O.make_point(K, E0, bp, r, prop)
    s2 = np.array(pt.sigma2[:K]) if prop == O.PAPER else np.ones(K)
    h3s = 2 * math.pi * (E0 / (2 * math.pi)) ** 1.5
    cS, cH, cQ = -bp / K**2, bp * r / (E0 * K**2) * h3s, (0.0 if prop == O.UNIFORM else float(K))
    ga = 1e-6 + gam * abs(cQ)
    gh = gam_t * abs(cH) * math.sqrt(K) + (2.0**-14 * math.sqrt(2 * K) * abs(cH) if grid_N else 0.0)
    ge = 2 * abs_err * (4 * K**2 * abs(cS) + 6 * math.sqrt(K) * abs(cH) + 2 * abs(cQ))
    gq = abs(cQ) * K * abs_err * (1 + s2.max())
    sig = np.sqrt(s2)
    g = np.empty(len(idx))
    for j, i in enumerate(idx):
        z, _ = O.stream(K, seed, pid, int(i))
        rho = z[:K] ** 2 + z[K:] ** 2
        inv2 = 1.0 / np.sum(s2 * rho)
        esum = np.sum(sig / np.sqrt(rho))
        tS = cS * o["S"][j]
        tH = cH * o["H3"][j] / h3s
        tQ = o["logfg"][j] - tS - tH
        g[j] = (ge * esum * math.sqrt(inv2) + gq * inv2 + ga +
                gam * (abs(tS) + abs(tQ) + abs(tH) + abs(o["lnU"][j]) + abs(logM)) + gh)
    return g


# (K, E0, beta', C3/C2, proposal): the one-thread triad form (K <= 64) and the warp form (K > 64)
REPLAY = [(8, 1.0, 30.0, 50.0, O.PAPER), (16, 1.0, 20.0, 75.0, O.PAPER), (32, 1.0, 40.0, 225.0, O.PAPER),
          (32, 1.0, 20.0, 450.0, O.UNIFORM), (64, 1.0, 40.0, 400.0, O.PAPER), (100, 1.0, 40.0, 225.0, O.PAPER),
          (128, 1.0, 60.0, 150.0, O.PAPER), (128, 1.0, 20.0, 450.0, O.UNIFORM)]


@pytest.mark.parametrize("K,E0,bp,r,prop", REPLAY)
def test_fast_path_error_within_guard(T, K, E0, bp, r, prop):
    seed, pid, lm = 17, 5, 1.5
    rng = np.random.default_rng(K)
    idx = np.concatenate([np.arange(2048), rng.integers(0, 1 << 40, 6144)]).astype(np.uint64)
    tp = T.PROPOSAL_PAPER if prop == O.PAPER else T.PROPOSAL_UNIFORM
    S = T.Sampler(K, [T.make_point(bp, E0, r, tp, point_id=pid, logM=lm)], sample_capacity=16)
    g = S.replay(0, idx, seed)
    S.close()
    fast = g["flags"] == 0
    idx = idx[fast]
    o = O.replay(O.make_point(K, E0, bp, r, prop, logM=lm), seed, pid, idx)
    err = np.abs(g["delta"][fast] - o["delta"])
    band = host_guard(K, prop, bp, E0, r, lm, o, idx, seed, pid)
    ratio = err / band
    assert np.all(ratio < 1.0), (float(ratio.max()), int(idx[np.argmax(ratio)]))
    print("K=%d prop=%d: %d draws, error / guard max %.3g, 99.9%% %.3g" % (
        K, prop, len(idx), ratio.max(), np.quantile(ratio, 0.999)))


@pytest.mark.parametrize("K,N,bp,r", [(16, 64, 20.0, 75.0), (32, 128, 40.0, 225.0), (64, 256, 40.0, 400.0)])
def test_grid_form_error_within_guard(T, K, N, bp, r):
    import torch
    E0, seed, pid, lm, n, i0 = 1.0, 23, 2, 1.5, 1 << 13, 500
    S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=pid, logM=lm)],
                  h3_mode=T.H3_GRID_BF16X3, grid_N=N, sample_capacity=1 << 14)
    tr = torch.zeros(2 * n, dtype=torch.float32, device="cuda")
    S.set_trace(tr, n)
    S.run_ranges([i0], [n], seed)
    S.sync()
    S.close()
    tr = tr.cpu().numpy().reshape(n, 2).astype(np.float64)
    keep = ~np.isnan(tr[:, 0])
    idx = np.arange(i0, i0 + n, dtype=np.uint64)[keep]
    o = O.replay(O.make_point(K, E0, bp, r, O.PAPER, logM=lm), seed, pid, idx)
    err = np.abs(tr[keep, 0] - o["delta"])
    ratio = err / host_guard(K, O.PAPER, bp, E0, r, lm, o, idx, seed, pid, grid_N=N)
    assert np.all(ratio < 1.0), (float(ratio.max()), int(idx[np.argmax(ratio)]))
    print("grid K=%d N=%d: %d draws, error / guard max %.3g, 99.9%% %.3g" % (
        K, N, len(idx), ratio.max(), np.quantile(ratio, 0.999)))

"""sampler_run_static: one sampler run that allocates no device memory.

It exists for callers that cannot call cudaMalloc -- code whose device memory
belongs to another allocator (a framework that reserved the whole pool up
front), latency-critical loops where cudaMalloc/cudaFree would synchronise the
device, plugin hosts that forbid allocation.  It keeps its scratch in a fixed
array inside the library.  Here its output must equal that of the regular
handle API (sampler_run_ranges) on the same index ranges, on two calls in a
row (the second call must not see the first call's leftovers).

This file is named so that pytest collects it last.
"""
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


def logM_k16(proposal=1):
    env = json.load(open(os.path.join(HERE, "golden", "envelopes.json")))["points"]
    return env["K16_E1_b20_r75_p%d" % proposal]["logM"]


def logM_k128(K, E0, bp, r):
    """An envelope for the 128-mode case (both sides of the comparison take
    the same log M): the oracle's largest log f/g over 512 draws plus a
    margin, which accepts a few per cent of the draws."""
    import oracle as O
    pt = O.make_point(K, E0, bp, r, O.PAPER)
    lf = O.replay(pt, 0, 0, np.arange(512, dtype=np.uint64))["logfg"]
    return float(lf.max() + np.log(np.mean(np.exp(lf - lf.max()))) + np.log(20.0))


# (K, proposal, C3/C2, proposals per call): the one-thread form with both
# proposals (uniform: its own kernels) and the 65..128-mode warp form
CASES = [(16, 1, 75.0, None), (16, 0, 75.0, None), (128, 1, 150.0, 1 << 16)]


@pytest.mark.parametrize("K,proposal,r,nmax", CASES)
def test_static_run_matches_handle_api_on_two_calls(T, K, proposal, r, nmax):
    import torch
    E0, bp, seed = 1.0, (20.0 if K == 16 else 60.0), 0
    lm = logM_k16(proposal) if K == 16 else logM_k128(K, E0, bp, r)
    point = T.make_point(bp, E0, r, proposal, point_id=0, logM=lm)
    rb = T.tkdv_record_bytes(K)
    cap = 1 << 14
    buf = torch.zeros(cap * rb, dtype=torch.uint8, device="cuda")
    n0 = nmax or T.STATIC_MAX_PROPOSALS
    ranges = [(0, n0), (n0, n0 - 12345)]
    for idx0, n in ranges:
        st_s, nrec = T.sampler_run_static(K, point, idx0, n, seed, buf, cap)
        rec_s = T.decode_records(buf[: nrec * rb].cpu().numpy(), K)
        S = T.Sampler(K, [point], sample_capacity=cap)
        S.run_ranges([idx0], [n], seed)
        st_h = S.stats()[0]
        rec_h = S.samples(cap)
        S.close()
        for key in ("n_proposals", "n_accepted", "n_refined", "n_near_threshold",
                    "n_envelope_violations", "n_dropped"):
            assert st_s[key] == st_h[key], key
        assert st_s["n_proposals"] == n and st_s["n_accepted"] > 0
        assert np.array_equal(st_s["hist"], st_h["hist"])
        assert np.array_equal(st_s["exceed"], st_h["exceed"])
        assert np.allclose(st_s["sum_u0"], st_h["sum_u0"], rtol=1e-12, atol=1e-12)
        assert nrec == len(rec_h["idx"]) == min(st_h["n_accepted"], cap)
        o_s, o_h = np.argsort(rec_s["idx"]), np.argsort(rec_h["idx"])
        assert np.array_equal(rec_s["idx"][o_s], rec_h["idx"][o_h])
        scale = np.abs(rec_h["H2"][o_h]) + np.abs(r * rec_h["H3"][o_h])
        dH = (rec_s["H2"][o_s] - r * rec_s["H3"][o_s]) - (rec_h["H2"][o_h] - r * rec_h["H3"][o_h])
        assert np.all(np.abs(dH) <= 1e-5 * scale)
        assert np.all(np.abs(rec_s["xhat"][o_s] - rec_h["xhat"][o_h]) <= 2e-6)


def test_static_run_allocates_no_device_memory(T):
    """After a first call (which loads the kernels and looks up the scratch
    array), further calls leave the device's free memory unchanged."""
    import torch
    K = 16
    point = T.make_point(20.0, 1.0, 75.0, T.PROPOSAL_PAPER, logM=logM_k16())
    rb = T.tkdv_record_bytes(K)
    cap = 1 << 12
    buf = torch.zeros(cap * rb, dtype=torch.uint8, device="cuda")
    T.sampler_run_static(K, point, 0, T.STATIC_MAX_PROPOSALS, 1, buf, cap)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for i in range(3):
        T.sampler_run_static(K, point, (i + 1) * T.STATIC_MAX_PROPOSALS, T.STATIC_MAX_PROPOSALS, 1, buf, cap)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_run_checks_the_records_buffer(T):
    """The binding refuses a records buffer the kernels could overrun."""
    import torch
    K = 16
    point = T.make_point(20.0, 1.0, 75.0, T.PROPOSAL_PAPER, logM=logM_k16())
    rb = T.tkdv_record_bytes(K)
    small = torch.zeros(10 * rb, dtype=torch.uint8, device="cuda")
    for bad in (dict(records=small, capacity=11),
                dict(records=torch.zeros(16 * rb, dtype=torch.uint8), capacity=16),
                dict(records=torch.zeros(16 * rb, dtype=torch.int32, device="cuda"), capacity=16),
                dict(records=None, capacity=4)):
        with pytest.raises(T.TkdvError) as ei:
            T.sampler_run_static(K, point, 0, 1024, 0, **bad)
        assert ei.value.code == -1
    st, n = T.sampler_run_static(K, point, 0, 1024, 0, records=small, capacity=10)
    assert st["n_proposals"] == 1024 and n <= 10


def test_static_run_rejects_what_it_cannot_hold(T):
    point = T.make_point(20.0, 1.0, 75.0, T.PROPOSAL_PAPER, logM=logM_k16())
    with pytest.raises(T.TkdvError) as ei:
        T.sampler_run_static(16, point, 0, T.STATIC_MAX_PROPOSALS + 1, 0)
    assert ei.value.code == -8
    no_env = T.make_point(20.0, 1.0, 75.0, T.PROPOSAL_PAPER)
    with pytest.raises(T.TkdvError) as ei:
        T.sampler_run_static(16, no_env, 0, 1024, 0)
    assert ei.value.code == -1

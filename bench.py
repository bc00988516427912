#!/usr/bin/env python
"""Throughput of the GB300 rejection sampler for the truncated-KdV Gibbs measure.

Workload (default): K = 32 modes, grid N = 128, E0 = 1, eight beta' values
log-spaced over [20, 60] with beta' C3/C2 = 9000 (the extreme-event regime of
Table 2), 2^28 proposals per point and step, all eight points in one
persistent launch.  A step is one such run of the whole hot path.

Prints one JSON line (rank 0).  `value` is accepted samples per second of the
whole job; proposals per second and the per-form numbers are alongside.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("accepted samples/sec and proposals/sec at K=32 "
          "(learned+BF16-split vs plain FP32, 1 GB300)")
L2_FLUSH_BYTES = 256 << 20
# bytes sampler_stats copies from the device per point (its integer counters,
# moment sums, 256 histogram and 26 exceedance bins, 128 spectrum sums, 7 SIR
# sums), plus the 8-byte record count and 4-byte status word per call
STAT_BYTES_PER_POINT = 8 * (6 + 1 + 4 + 256 + 26 + 1 + 2 + 128 + 1 + 7)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def alg_ops_per_proposal(K: int, form: str = "triad", grid_N: int = 128) -> int:
    """Ideal thread-instruction count of one proposal.

    Both forms: Philox4x32-10 (ceil(K/2)+1 blocks x 10 rounds x 4: two wide
    multiplies and two 3-input xors) and 40 for log Q, ln U, the ratio and
    the decision.
    triad (scalar FP32 per mode): Box-Muller and sigma scaling (20 per mode),
    the |x|^2, S, Q, u0 accumulations (4 per mode), and the symmetric double
    sum of Eq. (42) in packed FP32x2 pairs (2 per pair k < n-k, 4 for the
    middle term of an even n and 2 for the doubling of an odd one, 4 for the
    outer update); the same count serves the warp form (K > 64).
    grid (the two modes of a Philox block in packed FP32x2 pairs where the
    data allow): per pair of modes 22 for Box-Muller and scaling (4 bit
    shifts, 2 lg2, 2 floors, 2 rsqrt, 4 sin/cos, 8 packed multiply/add),
    4 packed accumulations, 2 table loads and 2 minima of the radius words;
    per value 2.5 for the BF16 hi/lo split (packed residuals) and 0.25 for
    the 16-byte shared-memory stores; 1.5 per mirror pair of grid points
    for 2 C (C^2 + S'^2) (three packed instructions per two pairs); one
    TMEM load per 16 columns of C and of S.  20.5 per mode in all."""
    blocks = (K + 1) // 2 + 1
    if form == "grid":
        return int(40 * blocks + 20.5 * K + 0.75 * grid_N + grid_N // 16 + 40)
    common = 40 * blocks + 20 * K + 4 * K + 40
    triad = sum(2 * ((n - 1) // 2) + (4 if n % 2 == 0 else 2) + 4 for n in range(2, K + 1))
    return common + triad


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per proposal of
# the sampler kernels, from one ncu capture each of the small case
# (--n-per-point 4194304, 8 points: 3.36e7 proposals per launch); the kernels
# read no per-proposal input, so traffic scales with the proposals processed.
# Set to None whenever the kernel changes until it is captured again.
TRAFFIC_PER_PROPOSAL = {
    "grid": (137984.0 / (8 * 4194304),
             "ncu --set full capture prof_grid_k32 (k_sample_grid<32,0,4,4>, 8 x 2^22 proposals)"),
    "triad": (116736.0 / (8 * 4194304),
              "ncu --set full capture prof_triad (k_sample_triad<32,0,256,1,0,1>, 8 x 2^22 proposals)"),
}
# the 64-mode grid kernel: one capture of the upstream run at 2^26 proposals
TRAFFIC_PER_PROPOSAL_K64 = (184576.0 / (1 << 26),
                            "ncu --set full capture prof_grid_k64 (k_sample_grid<64,0,2,2>, 2^26 proposals)")


def alu_peak(n_sms, peaks):
    """Thread instructions per second the SMs can issue: SMs x 128 lanes x
    the maximum SM clock (T-ops/s)."""
    return n_sms * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def tensor_flops_per_proposal(K: int, grid_N: int) -> int:
    """The mirror-pair contraction as issued: three BF16 products (hi hi, hi lo,
    lo hi) of the cosine and of the sine part of a row (K modes rounded up to
    a 16-column MMA step) with an N/2-column basis."""
    kpad = (K + 15) // 16 * 16
    return 3 * 2 * (2 * kpad) * (grid_N // 2)


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(device_index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, t_begin=None, t_end=None):
        """Median SM clock and the throttle reasons seen between the wall-clock
        times t_begin and t_end (datetime; all samples when not given)."""
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        os.unlink(self.f.name)
        if t_begin is not None:
            import datetime as dt
            kept = []
            for r in rows:
                try:
                    ts = dt.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f")
                except ValueError:
                    continue
                if t_begin <= ts <= t_end:
                    kept.append(r)
            rows = kept or rows
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_points(rank, n_per_point):
    from paper_2411_16952_gb300 import workloads
    wl = workloads.extreme_k32(n_per_point)
    # each rank samples its own streams (point ids rank*8 + p): disjoint draws
    return wl, [(bp, r, rank * len(wl["points"]) + p) for p, (bp, r) in enumerate(wl["points"])]


def cpu_baseline(wl, pts, seconds=15.0, sample_points=2):
    """The FP64 oracle, as it stands, on all host cores, on a bounded sample:
    the first `sample_points` points of the workload, sized to ~`seconds`."""
    import oracle as O
    cores = os.cpu_count() or 1
    K, E0 = wl["K"], wl["E0"]
    ops = []
    for bp, r, pid in pts[:sample_points]:
        pt = O.make_point(K, E0, bp, r, O.PAPER)
        pt.logM = _oracle_envelope(K, bp, E0, r, pt)
        ops.append((pt, pid))
    t0 = time.perf_counter()
    O.run_stats(ops[0][0], 0, ops[0][1], 0, 1 << 18, cores)
    per = (time.perf_counter() - t0) / (1 << 18)
    n = int(max(1 << 18, min(1 << 30, seconds / max(per, 1e-12) / len(ops))))
    acc = prop = 0
    t0 = time.perf_counter()
    for pt, pid in ops:
        st = O.run_stats(pt, 0, pid, 0, n, cores)
        acc += st["n_acc"]
        prop += st["n_prop"]
    dt = time.perf_counter() - t0
    return {"value": acc / dt, "unit": "accepted samples/s", "proposals_per_s": prop / dt,
            "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": "%d proposals of each of the first %d points (K=%d, paper proposal), FP64 C oracle, "
                      "%d threads" % (n, len(ops), K, cores)}


def oracle_h_error(T, wl, pts, stream, n=1 << 14):
    """Error of the grid form's H3 (BF16 hi/lo x3 contraction, FP32 cube-sum)
    against the FP64 oracle on a replayed subset: the first and last points of
    the workload (paper proposal), n traced proposals each.  Reports the
    scale-aware relative error |dH| / (|H2| + |C3/C2 H3|) and the error of the
    beta H term of log f/(Mg), |beta' C3/C2 dH3 / (E0 K^2)|."""
    import math
    import torch
    import oracle as O
    K, E0, gN = wl["K"], wl["E0"], wl["grid_N"]
    h3s = 2 * math.pi * (E0 / (2 * math.pi)) ** 1.5
    rel, bh = [], []
    for bp, r, pid in (pts[0], pts[-1]):
        pt = O.make_point(K, E0, bp, r, O.PAPER)
        pt.logM = _oracle_envelope(K, bp, E0, r, pt)
        S = T.Sampler(K, [T.make_point(bp, E0, r, T.PROPOSAL_PAPER, point_id=pid, logM=pt.logM)],
                      h3_mode=T.H3_GRID_BF16X3, grid_N=gN, sample_capacity=1 << 10, stream=stream)
        tr = torch.zeros(2 * n, dtype=torch.float32, device="cuda")
        S.set_trace(tr, n)
        S.run_ranges([0], [n], 11)
        S.sync()
        S.close()
        tr = tr.cpu().numpy().reshape(n, 2).astype(np.float64)
        keep = ~np.isnan(tr[:, 0])
        o = O.replay(pt, 11, pid, np.arange(n, dtype=np.uint64)[keep])
        dH3 = h3s * tr[keep, 1] - o["H3"]
        rel.append(np.abs(r * dH3) / (np.abs(o["H2"]) + np.abs(r * o["H3"])))
        bh.append(np.abs(bp * r / (E0 * K * K) * dH3))
    rel, bh = np.concatenate(rel), np.concatenate(bh)
    return {"h_rel_max": float(rel.max()), "h_rel_median": float(np.median(rel)),
            "beta_h_abs_max": float(bh.max()), "beta_h_abs_median": float(np.median(bh)),
            "tolerance": 1e-5, "proposals": int(rel.size),
            "sample": "grid form (paper proposal), %d traced proposals of the first and last points, "
                      "against the FP64 oracle's replay" % n}


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, per step a bounded
    sample of the same workload (one point per step, cycling)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    from paper_2411_16952_gb300 import workloads
    wl = workloads.extreme_k32(1)
    K, E0 = wl["K"], wl["E0"]
    cores = os.cpu_count() or 1
    pts = []
    for p, (bp, r) in enumerate(wl["points"]):
        pt = O.make_point(K, E0, bp, r, O.PAPER)
        pt.logM = O.log_M(pt, 0) if args.ref_exact_envelope else _oracle_envelope(K, bp, E0, r, pt)
        pts.append((pt, p))
    n = args.ref_proposals
    for i in range(args.warmup):
        pt, pid = pts[i % len(pts)]
        O.run_stats(pt, 0, pid, 0, n, cores)
    acc = prop = 0
    t_all = 0.0
    for i in range(args.steps):
        pt, pid = pts[i % len(pts)]
        t0 = time.perf_counter()
        st = O.run_stats(pt, 0, pid, (i + 1) * n, n, cores)
        t_all += time.perf_counter() - t0
        acc += st["n_acc"]
        prop += st["n_prop"]
    val = acc / t_all
    line = {"metric": METRIC, "value": val, "unit": "accepted samples/s", "impl": "reference",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "proposals_per_s": prop / t_all,
            "config": {"workload": wl["name"], "K": K, "points": len(pts),
                       "proposals_per_step": n, "proposal": "paper"},
            "cpu_baseline": {"value": val, "unit": "accepted samples/s", "cores": cores, "kind": "oracle",
                             "sample": "%d proposals per step, one point per step (cycling over %d), "
                                       "FP64 C oracle on %d threads" % (n, len(pts), cores)},
            "e2e": {"value": val, "unit": "accepted samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _oracle_envelope(K, bp, E0, r, pt):
    """The oracle's own log M (Nelder-Mead, Eq. 45): the cached value that
    tests/golden/make_envelopes.py wrote with the oracle alone, or, for a
    point not in that file, the oracle's search run here (slow at K = 32)."""
    import oracle as O
    path = os.path.join(ROOT, "tests", "golden", "envelopes.json")
    if os.path.exists(path):
        key = "K%d_E%.17g_b%.17g_r%.17g_p%d" % (K, E0, bp, r, O.PAPER)
        pts = json.load(open(path))["points"]
        if key in pts:
            return pts[key]["logM"]
    return O.log_M(pt, 0)


def train_learned(T, K, pts3, grid_N, n_accept, steps, tau, seed, stream, keep=False):
    """Train the learned proposal on n_accept accepted samples per point of
    pts3 [(beta', E0, C3/C2), ...] (paper-proposal sampler, grid form), with
    the tempered loss J_tau.  Per point the corrections are kept only where
    the learned proposal's envelope is below the paper's (its acceptance is
    Prod w_k Z / M with Prod w_k unchanged by mean-zero corrections, so the
    gain is exactly exp(log M_paper - log M_learned)); elsewhere the point
    falls back to the paper's Sigma.  Returns (corrections P x K, info, the
    network handle if keep else None)."""
    from paper_2411_16952_gb300 import learned as L
    t0 = time.perf_counter()
    mlp, corr, hist, rows = L.train(K, pts3, n_accept=n_accept, steps=steps, lr=2e-2, tau=tau, seed=1,
                                    sampler_seed=seed, stream=stream, h3_mode=T.H3_GRID_BF16X3, grid_N=grid_N)
    t_train = time.perf_counter() - t0
    info = []
    for i, p3 in enumerate(pts3):
        gain, lm_p, lm_l = L.predicted_gain(K, p3, corr[i])
        fallback = not gain > 1.0
        info.append({"beta_p": p3[0], "E0": p3[1], "r": p3[2], "gain_trained": gain,
                     "gain": 1.0 if fallback else gain, "fallback_to_paper": fallback,
                     "max_abs_c": float(np.max(np.abs(corr[i])))})
        if fallback:
            corr[i] = 0.0
    if not keep:
        L.close(mlp)
        mlp = None
    return corr, {"train_seconds": t_train, "accepted_rows_per_point": [int(v) for v in rows],
                  "tau": tau, "steps": steps, "loss_first_last": [float(hist[0]), float(hist[-1])],
                  "points": info}, mlp


def k64_pipeline(T, args, stream, peaks, n_sms, rank, learned=True, shift=0):
    """The 64-mode pipeline (learned proposal + BF16 hi/lo grid form, N = 256):
    the upstream ensemble (2^30 proposals, one run), then the downstream beta'
    by bisection on the matching statistic (here the ensemble mean of
    S = H2/E0), 16 candidates per step in one persistent launch of 2^30
    proposals.  Every run is timed with CUDA events on the sampler's stream;
    the per-point precompute (alpha*, envelope search) of each step's
    candidates is host work outside the events and is reported apart."""
    from paper_2411_16952_gb300 import learned as L
    from paper_2411_16952_gb300 import matching as MT
    from paper_2411_16952_gb300 import workloads
    import torch
    pw = workloads.pipeline_k64()
    pw["n_up"] >>= shift
    pw["n_cand"] >>= shift
    K, N, E0 = pw["K"], pw["grid_N"], pw["E0"]
    up = (pw["beta_up"], E0, pw["r_up"])
    train_pts = [up] + [(float(b), E0, pw["r_down"]) for b in np.linspace(pw["lo"], pw["hi"], 7)]
    if learned:
        corr, info, mlp = train_learned(T, K, train_pts, N, pw["learn_accept"], args.learn_steps, args.learn_tau,
                                        rank + 3000, stream, keep=True)
    else:  # the paper's Sigma throughout (c = 0)
        corr = np.zeros((len(train_pts), K))
        info = {"train_seconds": 0.0, "tau": None, "accepted_rows_per_point": [],
                "points": [{"gain": 1.0, "fallback_to_paper": True} for _ in train_pts]}
        mlp = None
    runs = []

    def timed_run(points, budget, seed):
        t_host = time.perf_counter()
        S = T.Sampler(K, points, h3_mode=T.H3_GRID_BF16X3, grid_N=N, sample_capacity=1 << 16, stream=stream)
        S.run_ranges([1 << 62] * len(points), [1] * len(points), seed)  # builds the run's graph
        S.sync()
        S.reset()
        t_host = time.perf_counter() - t_host
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        S.run(budget, seed)
        e1.record(stream)
        st = S.stats()
        S.close()
        ms = e0.elapsed_time(e1)
        runs.append({"points": len(points), "proposals": budget * len(points), "ms": ms, "host_setup_s": t_host,
                     "accepted": int(sum(s["n_accepted"] for s in st))})
        return st

    try:
        st_up = timed_run([T.make_point(*up, T.PROPOSAL_LEARNED, point_id=rank * 4096,
                                        log_var_correction=corr[0])], pw["n_up"], 11)[0]
        target = MT.mean_S(st_up, K)

        def run_batch(betas, pid0, n, seed):
            pts3 = [(float(b), E0, pw["r_down"]) for b in betas]
            c = L.infer(mlp, K, pts3) if mlp is not None else np.zeros((len(pts3), K))
            points = [T.make_point(b, e, r, T.PROPOSAL_LEARNED, point_id=rank * 4096 + 1 + pid0 + j,
                                   log_var_correction=c[j]) for j, (b, e, r) in enumerate(pts3)]
            return timed_run(points, n, seed)

        res = MT.bisect_beta(K, E0, pw["r_down"], MT.mean_S, target, pw["lo"], pw["hi"],
                             n_candidates=pw["n_candidates"], n_steps=pw["steps"],
                             proposals_per_candidate=pw["n_cand"], seed=21, run_batch=run_batch)
        err = None
    except (ValueError, T.TkdvError) as e:  # the statistic did not bracket the target, or a run failed
        res, err = None, str(e)
    finally:
        if mlp is not None:
            L.close(mlp)
    t_s = sum(r["ms"] for r in runs) / 1e3
    props = sum(r["proposals"] for r in runs)
    acc = sum(r["accepted"] for r in runs)
    pps = props / t_s if t_s > 0 else 0.0
    ops = alg_ops_per_proposal(K, "grid", N)
    tf = tensor_flops_per_proposal(K, N) * pps / 1e12
    tpk = float(peaks.get("bf16_tflops_sustained", 1735.3))
    out = {"workload": pw["name"], "K": K, "grid_N": N, "error": err,
           "traffic_per_proposal": TRAFFIC_PER_PROPOSAL_K64[0], "traffic_source": TRAFFIC_PER_PROPOSAL_K64[1],
           "form": "grid_bf16x3_learned" if learned else "grid_bf16x3_paper",
           "proposals_per_s": pps, "accepted_per_s": acc / t_s if t_s > 0 else 0.0, "runs": runs,
           "roofline": {"alu": {"ops_per_proposal": ops, "achieved": ops * pps / 1e12, "peak": alu_peak(n_sms, peaks),
                                "unit": "Tops/s", "frac": ops * pps / 1e12 / alu_peak(n_sms, peaks)},
                        "tensor": {"flops_per_proposal": tensor_flops_per_proposal(K, N), "achieved_tflops": tf,
                                   "peak_tflops": tpk, "frac": tf / tpk,
                                   "note": "mirror-pair BF16 hi/lo x3 contraction flops over the sampler runs' "
                                           "duration, against the sustained cuBLAS BF16 peak"}},
           "learned": {"train_seconds": info["train_seconds"], "tau": info["tau"],
                       "accepted_rows_per_point": info["accepted_rows_per_point"],
                       "gain_exact": [q["gain"] for q in info["points"]],
                       "fallback_to_paper": [q["fallback_to_paper"] for q in info["points"]]}}
    if runs:
        n_up = st_up["n_accepted"]
        sig0 = math.sqrt(E0 / math.pi)
        out["upstream"] = {"beta_p": up[0], "r": up[2], "proposals": runs[0]["proposals"], "ms": runs[0]["ms"],
                           "accepted": n_up, "acceptance": n_up / runs[0]["proposals"], "mean_S": MT.mean_S(st_up, K),
                           "u0": {"mean": st_up["mean"], "var": st_up["var"], "skew": st_up["skew"],
                                  "kurt": st_up["kurt"]},
                           "exceed_2_3_4_sigma0": [int(st_up["exceed"][8]), int(st_up["exceed"][12]),
                                                   int(st_up["exceed"][16])],
                           "sigma0": sig0, "hist_bins_nonzero": int(np.count_nonzero(st_up["hist"])),
                           "envelope_violations": int(st_up["n_envelope_violations"])}
    if res is not None:
        out["downstream"] = {"r": pw["r_down"], "beta_p_found": res["beta"], "bracket": list(res["bracket"]),
                             "target_mean_S": MT.mean_S(st_up, K), "steps": pw["steps"],
                             "candidates_per_step": pw["n_candidates"],
                             "proposals_per_step": pw["n_candidates"] * pw["n_cand"],
                             "ms_per_step": [r["ms"] for r in runs[1:]],
                             "last_step": {"betas": [float(b) for b in res["history"][-1][0]],
                                           "mean_S": [float(v) for v in res["history"][-1][1]]}}
    return out


def measured_gain(st_paper, st_learned, info):
    """Per point: the learned proposal's acceptance over the paper's, measured
    (with its standard error; both from the timed runs, independent streams
    assumed) against the exact value, and the u(0) mean, variance and
    skewness of the two ensembles (the same Gibbs measure: within 3 SE)."""
    out = []
    for sp, sl, pi in zip(st_paper, st_learned, info):
        ap, al = sp["n_accepted"] / sp["n_proposals"], sl["n_accepted"] / sl["n_proposals"]
        ratio = al / ap if ap > 0 else float("nan")
        se = ratio * math.sqrt(1.0 / max(sp["n_accepted"], 1) + 1.0 / max(sl["n_accepted"], 1))
        nn = max(min(sp["n_accepted"], sl["n_accepted"]), 1)
        se_mean = 2 * math.sqrt(sp["var"] / nn)
        se_var = 2 * sp["var"] * math.sqrt(max(sp["kurt"] - 1.0, 1.0) / nn)
        se_skew = 2 * math.sqrt(6.0 / nn)
        out.append({"beta_p": pi["beta_p"], "gain_exact": pi["gain"], "gain_measured": ratio, "gain_se": se,
                    "within_4se": abs(ratio - pi["gain"]) <= 4 * se,
                    "u0_mean": [sp["mean"], sl["mean"]], "u0_var": [sp["var"], sl["var"]],
                    "u0_skew": [sp["skew"], sl["skew"]],
                    "stats_within_3se": bool(abs(sp["mean"] - sl["mean"]) <= 1.5 * se_mean and
                                             abs(sp["var"] - sl["var"]) <= 1.5 * se_var and
                                             abs(sp["skew"] - sl["skew"]) <= 1.5 * se_skew),
                    "envelope_violations": int(sl["n_envelope_violations"])})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-per-point", type=int, default=1 << 28)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-proposals", type=int, default=1 << 22)
    ap.add_argument("--ref-exact-envelope", action="store_true")
    ap.add_argument("--forms", default="", help="comma list of forms to time (default: all)")
    ap.add_argument("--learn-accept", type=int, default=1 << 20, help="accepted samples per point to train on")
    ap.add_argument("--learn-steps", type=int, default=300)
    ap.add_argument("--learn-tau", type=float, default=0.5,
                    help="temperature of the training loss J_tau (0: the plain mean, KL(f || g))")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-learn-accept", type=int, default=1 << 14,
                    help="64-point batch: accepted samples per point to train its network on")
    ap.add_argument("--no-k64", action="store_true", help="skip the 64-mode pipeline")
    ap.add_argument("--only-k64", action="store_true",
                    help="run only the 64-mode pipeline (with --k64-paper: the paper's Sigma, no training) and "
                         "print its JSON object")
    ap.add_argument("--k64-paper", action="store_true")
    ap.add_argument("--k64-shift", type=int, default=0, help="64-mode pipeline: proposals divided by 2^shift")
    ap.add_argument("--no-k128", action="store_true", help="skip the K = 128 measurement")
    ap.add_argument("--k128-n", type=int, default=1 << 24, help="K = 128: proposals per point and step")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2411_16952_gb300 as T
    from paper_2411_16952_gb300 import _build
    _build.build()
    peaks, peak_src = measured_peaks()
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    wl, pts = workload_points(rank, args.n_per_point)
    K, E0, n, gN = wl["K"], wl["E0"], args.n_per_point, wl["grid_N"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.only_k64:
        print(json.dumps({"k64_pipeline": k64_pipeline(T, args, stream, peaks, n_sms, rank,
                                                       learned=not args.k64_paper, shift=args.k64_shift)}))
        return
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    import datetime as dt
    clk = Clocks(local)  # started before any warm-up so that its start-up stays out of the timed steps
    forms = {"triad_f32_paper": (T.H3_TRIAD_F32, T.PROPOSAL_PAPER),
             "grid_bf16x3_paper": (T.H3_GRID_BF16X3, T.PROPOSAL_PAPER),
             "grid_bf16x3_learned": (T.H3_GRID_BF16X3, T.PROPOSAL_LEARNED),
             # SIR with c = 1: the expected copies per proposal equal the
             # rejection acceptance (lambda = exp(log f/(Mg)))
             "sir_triad_paper": (T.H3_TRIAD_F32, T.PROPOSAL_PAPER)}
    if args.forms:
        unknown = set(args.forms.split(",")) - set(forms)
        if unknown:
            raise SystemExit("unknown form(s) %s; known: %s" % (sorted(unknown), sorted(forms)))
        forms = {k: v for k, v in forms.items() if k in args.forms.split(",")}
    headline = next((f for f in ("grid_bf16x3_learned", "grid_bf16x3_paper", "triad_f32_paper") if f in forms),
                    next(iter(forms)))
    learned_info = None
    if "grid_bf16x3_learned" in forms:
        # the learned proposal is trained (outside the timed region) on accepted
        # samples of the same points, generated by the paper-proposal sampler
        pts3 = [(bp, E0, r) for bp, r, _ in pts]
        corr, learned_info, _ = train_learned(T, K, pts3, gN, args.learn_accept, args.learn_steps, args.learn_tau,
                                              rank + 1000, stream)
    results = {}
    stats_by_form = {}
    windows = []
    for fname, (mode, prop) in forms.items():
        if prop == T.PROPOSAL_LEARNED:
            points = [T.make_point(bp, E0, r, prop, point_id=pid, log_var_correction=corr[i])
                      for i, (bp, r, pid) in enumerate(pts)]
        else:
            points = [T.make_point(bp, E0, r, prop, point_id=pid) for bp, r, pid in pts]
        S = T.Sampler(K, points, h3_mode=mode, grid_N=gN if mode == T.H3_GRID_BF16X3 else 0,
                      sample_capacity=1 << 21, stream=stream, sir=fname.startswith("sir"))
        if not args.no_autotune:
            S.autotune(1 << 24)
        seed = 0
        for _ in range(args.warmup):
            S.run(n, seed)
        S.sync()
        S.reset()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t_begin = dt.datetime.now()
        evs = []
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the step events)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            S.run(n, seed)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        windows.append((t_begin, dt.datetime.now()))
        step_ms = [a.elapsed_time(b_) for a, b_ in evs]
        st = S.stats()
        stats_by_form[fname] = st
        acc = sum(s["n_accepted"] for s in st)
        prop_n = sum(s["n_proposals"] for s in st)
        refined = sum(s["n_refined"] for s in st)
        t_s = sum(step_ms) / 1e3
        if ws > 1:
            tt = torch.tensor([t_s], dtype=torch.float64, device="cuda")
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            cnt = torch.tensor([acc, prop_n], dtype=torch.float64, device="cuda")
            torch.distributed.all_reduce(cnt)
            t_s, acc, prop_n = float(tt.item()), int(cnt[0].item()), int(cnt[1].item())
        res = {"accepted_per_s": acc / t_s, "proposals_per_s": prop_n / t_s, "ms_per_step": 1e3 * t_s / args.steps,
               "acceptance": acc / max(prop_n, 1), "refined_fraction": refined / max(prop_n, 1),
               "launch": S.launch_config()}
        if fname == headline:
            # end to end through the public API with host buffers: run, then
            # statistics and the raw accepted records copied into a pinned
            # host buffer every step (sampler_stats, sampler_samples)
            S.reset()
            rec_bytes = T.tkdv_record_bytes(K)
            host_rec = torch.empty((1 << 21) * rec_bytes, dtype=torch.uint8, pin_memory=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d2h = 0
            e2e_acc = 0
            for i in range(args.steps):
                S.reset()
                S.run(n, seed + 1 + i)
                sts = S.stats()
                nrec = S.samples(1 << 21, host_dst=host_rec)
                e2e_acc += sum(s["n_accepted"] for s in sts)
                d2h += nrec * rec_bytes + len(sts) * STAT_BYTES_PER_POINT + 12
            e2e_t = time.perf_counter() - t0
            res["e2e"] = {"value": e2e_acc / e2e_t, "unit": "accepted samples/s",
                          "h2d_bytes_per_step": 8 * 2 * len(pts) + 8, "d2h_bytes_per_step": d2h // args.steps}
        S.close()
        results[fname] = res
    clocks = clk.stop(windows[0][0], windows[-1][1])
    if learned_info is not None and "grid_bf16x3_paper" in stats_by_form:
        learned_info["measured"] = measured_gain(stats_by_form["grid_bf16x3_paper"],
                                                 stats_by_form["grid_bf16x3_learned"], learned_info["points"])

    # the 64-point batch (uneven budgets 2^18..2^26, one persistent launch)
    batch = None
    if not args.no_batch:
        from paper_2411_16952_gb300 import workloads
        bw = workloads.batch_k32()
        bpts = [T.make_point(float(bw["beta_p"][p]), float(bw["E0"][p]), float(bw["r"][p]), T.PROPOSAL_PAPER,
                             point_id=rank * 64 + p) for p in range(64)]
        # the triad form, the grid form with the paper's Sigma, and the grid
        # form with the learned proposal (a network trained on the batch's
        # own points, the paper's Sigma where it does not lower the envelope)
        bforms = {}
        bcorr, binfo = None, None
        if "grid_bf16x3_learned" in forms:
            b3 = [(float(bw["beta_p"][p]), float(bw["E0"][p]), float(bw["r"][p])) for p in range(64)]
            bcorr, binfo, _ = train_learned(T, bw["K"], b3, 128, args.batch_learn_accept, args.learn_steps,
                                            args.learn_tau, rank + 2000, stream)
        for best_form in [f for f in ("triad_f32_paper", "grid_bf16x3_paper", "grid_bf16x3_learned") if f in results]:
            bmode = T.H3_GRID_BF16X3 if best_form.startswith("grid") else T.H3_TRIAD_F32
            pts_b = bpts
            if best_form.endswith("learned"):
                pts_b = [T.make_point(float(bw["beta_p"][p]), float(bw["E0"][p]), float(bw["r"][p]),
                                      T.PROPOSAL_LEARNED, point_id=rank * 64 + p, log_var_correction=bcorr[p])
                         for p in range(64)]
            SB = T.Sampler(bw["K"], pts_b, h3_mode=bmode, grid_N=128 if bmode == T.H3_GRID_BF16X3 else 0,
                           sample_capacity=1 << 22, stream=stream)
            if not args.no_autotune:
                SB.autotune(1 << 20)
            for _ in range(args.warmup):
                SB.run_budgets(bw["budgets"], 7)
            SB.sync()
            SB.reset()
            bev = []
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                SB.run_budgets(bw["budgets"], 7)
                e1.record(stream)
                bev.append((e0, e1))
            torch.cuda.synchronize()
            bms = sum(a.elapsed_time(b_) for a, b_ in bev) / args.steps
            bst = SB.stats()
            bprop = sum(s["n_proposals"] for s in bst)
            bacc = sum(s["n_accepted"] for s in bst)
            bforms[best_form] = {"proposals_per_step": bprop // args.steps, "ms_per_step": bms,
                                 "proposals_per_s": bprop / (bms * args.steps / 1e3),
                                 "accepted_per_s": bacc / (bms * args.steps / 1e3), "launch": SB.launch_config(),
                                 "envelope_violations": int(sum(s["n_envelope_violations"] for s in bst))}
            SB.close()
        if bforms:
            best_form = max(bforms, key=lambda f: bforms[f]["accepted_per_s"])
            batch = dict(bforms[best_form], workload=bw["name"], form=best_form, forms=bforms)
            if binfo is not None:
                g = [q["gain"] for q in binfo["points"]]
                batch["learned"] = {"train_seconds": binfo["train_seconds"], "tau": binfo["tau"],
                                    "accepted_rows_per_point_min": min(binfo["accepted_rows_per_point"]),
                                    "gain_exact_min_median_max": [min(g), float(np.median(g)), max(g)],
                                    "points_falling_back_to_paper": sum(q["fallback_to_paper"] for q in binfo["points"])}
            if "triad_f32_paper" in bforms and "grid_bf16x3_learned" in bforms:
                batch["learned_grid_vs_plain_fp32"] = (bforms["grid_bf16x3_learned"]["accepted_per_s"] /
                                                       bforms["triad_f32_paper"]["accepted_per_s"])

    # K = 128 (one warp per four proposals, the cutoff of Fig. 7): eight points
    k128 = None
    if not args.no_k128:
        from paper_2411_16952_gb300 import workloads
        kw = workloads.speedup_k128(args.k128_n)
        kpts = [T.make_point(b, kw["E0"], r, T.PROPOSAL_PAPER, point_id=rank * 8 + p)
                for p, (b, r) in enumerate(kw["points"])]
        SK = T.Sampler(kw["K"], kpts, sample_capacity=1 << 20, stream=stream)
        if not args.no_autotune:
            SK.autotune(1 << 24)
        for _ in range(args.warmup):
            SK.run(kw["n"], 3)
        SK.sync()
        SK.reset()
        kev = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            SK.run(kw["n"], 3)
            e1.record(stream)
            kev.append((e0, e1))
        torch.cuda.synchronize()
        kms = sum(a.elapsed_time(b_) for a, b_ in kev) / args.steps
        kst = SK.stats()
        kprop = sum(s["n_proposals"] for s in kst)
        kacc = sum(s["n_accepted"] for s in kst)
        kops = alg_ops_per_proposal(kw["K"], "triad")
        kpeak = alu_peak(n_sms, peaks)
        kpps = kprop / (kms * args.steps / 1e3)
        k128 = {"workload": kw["name"], "K": kw["K"], "ms_per_step": kms, "proposals_per_s": kpps,
                "accepted_per_s": kacc / (kms * args.steps / 1e3), "acceptance": kacc / kprop,
                "refined_fraction": sum(s["n_refined"] for s in kst) / kprop,
                "envelope_violations": sum(s["n_envelope_violations"] for s in kst),
                "launch": SK.launch_config(),
                "alu": {"ops_per_proposal": kops, "achieved": kops * kpps / 1e12, "peak": kpeak,
                        "unit": "Tops/s", "frac": kops * kpps / 1e12 / kpeak,
                        "kernel": "k_sample_warp", "note": "same op count and peak as the headline roofline"}}
        SK.close()

    # the 64-mode pipeline (learned + grid form, bisection of the downstream beta')
    k64 = None
    if not args.no_k64 and ws == 1 and "grid_bf16x3_learned" in forms:
        k64 = k64_pipeline(T, args, stream, peaks, n_sms, rank, shift=args.k64_shift)

    h = results[headline]
    form_kind = "grid" if headline.startswith("grid") else "triad"
    ops = alg_ops_per_proposal(K, form_kind, gN)
    step_s = h["ms_per_step"] / 1e3
    props_per_step = h["proposals_per_s"] * step_s
    achieved = ops * props_per_step / step_s / 1e12
    peak = alu_peak(n_sms, peaks)
    tr = TRAFFIC_PER_PROPOSAL.get(form_kind)
    traffic = None if tr is None or tr[0] is None else tr[0] * props_per_step
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": tr[1] if tr else None,
            "algorithmic_bytes_per_launch": h["acceptance"] * props_per_step * T.tkdv_record_bytes(K) + STAT_BYTES_PER_POINT * len(pts),
            "ops_per_proposal": ops, "kernel": "k_sample_%s" % form_kind,
            "note": "ideal thread-instruction count per proposal (bench.py alg_ops_per_proposal); peak = "
                    "%d SMs (device) x 128 lanes x max SM clock (%s sm_max_mhz)" % (n_sms, peak_src)}
    if form_kind == "grid":
        tf = tensor_flops_per_proposal(K, gN) * h["proposals_per_s"] / 1e12
        roof["tensor"] = {"achieved_tflops": tf, "peak_tflops": float(peaks.get("bf16_tflops_sustained", 1735.3)),
                          "frac": tf / float(peaks.get("bf16_tflops_sustained", 1735.3)),
                          "note": "BF16 hi/lo x3 contraction flops of the whole sampler run over its duration, "
                                  "against the sustained cuBLAS BF16 peak (%s)" % peak_src}
    line = {
        "metric": METRIC, "value": h["accepted_per_s"], "unit": "accepted samples/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": h["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x3+f32" if form_kind == "grid" else "f32", "data": "synthetic",
        "proposals_per_s": h["proposals_per_s"], "acceptance": h["acceptance"],
        "headline_form": headline, "forms": results,
        "vs_plain_fp32": h["accepted_per_s"] / results["triad_f32_paper"]["accepted_per_s"]
        if "triad_f32_paper" in results else None,
        "learned": learned_info, "batch_64pts": batch, "k128": k128, "k64_pipeline": k64,
        "config": {"workload": wl["name"], "K": K, "grid_N": gN, "points": len(pts),
                   "proposals_per_point_per_step": n,
                   "proposal": "learned" if headline.endswith("learned") else "paper",
                   "h3_form": "grid_bf16x3" if form_kind == "grid" else "triad_f32",
                   "l2": "256 MiB buffer written between timed steps, outside the step events",
                   "parallelism": "points x index ranges, weak per GPU"},
        "roofline": roof,
        "e2e": h.get("e2e"),
        # kernels of this library launched in the headline's timed region:
        # per step the persistent sampler and its FP64 pass (one CUDA graph)
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the oracle leg: the FP64 oracle timed on the host cores, and the
        # grid form's H error measured against it
        line["cpu_baseline"] = cpu_baseline(wl, pts, args.cpu_seconds)
        if any(f.startswith("grid") for f in results):
            line["h_error_vs_fp64"] = oracle_h_error(T, wl, pts, stream)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

"""Batched bisection of the downstream beta' on a matching statistic.

The method fixes the downstream Gibbs ensemble's inverse temperature by a
statistical matching condition between the upstream and downstream states
(Secs. I and II.A); the paper takes that beta' as given and does not state
the condition.  Here the condition is a function the caller supplies: it maps
one candidate's sampler statistics (and the candidate's beta') to a number,
and the driver finds the beta' where that number equals a target.

Each step samples a batch of candidate beta' values, spread over the current
bracket, in one persistent launch (one sampler handle; each run is one CUDA
graph), evaluates the statistic on every candidate and keeps the sub-bracket
where it crosses the target.  The statistic must be monotone in beta' over
the starting bracket.
"""
from __future__ import annotations

import numpy as np

from . import H3_TRIAD_F32, PROPOSAL_PAPER, Sampler, make_point


def mean_S(stats, K, beta_p=None):
    """Ensemble mean of S = sum_k k^2 s_k = H2 / E0 (Eq. 20) over the accepted
    fields, from the per-mode spectrum sums."""
    n = stats["n_accepted"]
    if n == 0:
        return float("nan")
    k = np.arange(1, K + 1, dtype=np.float64)
    return float(np.dot(k * k, stats["spectrum"][:K]) / n)


def skewness_u0(stats, K=None, beta_p=None):
    """Skewness of the surface displacement u(0) over the accepted fields."""
    return float(stats["skew"])


def _gpu_batch(K, E0, r, proposal, h3_mode, grid_N, capacity):
    def run(betas, point_id0, n, seed):
        pts = [make_point(float(b), E0, r, proposal, point_id=point_id0 + j) for j, b in enumerate(betas)]
        S = Sampler(K, pts, h3_mode=h3_mode, grid_N=grid_N, sample_capacity=capacity)
        try:
            S.run(n, seed)
            return S.stats()
        finally:
            S.close()
    return run


def bisect_beta(K, E0, r, statistic, target, lo, hi, n_candidates=16, n_steps=4, proposals_per_candidate=1 << 24,
                seed=0, proposal=PROPOSAL_PAPER, h3_mode=H3_TRIAD_F32, grid_N=0, run_batch=None):
    """beta' in [lo, hi] where statistic(stats, K, beta') == target.

    statistic: callable(stats_dict, K, beta') -> float, monotone in beta'.
    run_batch: callable(betas, point_id0, n, seed) -> list of stats dicts; by
    default the library's batched sampler (at most 64 candidates).
    Each step keeps the crossing interval widened by half a candidate spacing
    on each side (the bracket shrinks by 2/(n_candidates - 1) per step); the
    estimate is the root of the least-squares line through the last step's
    candidates.  Returns {"beta": estimate, "bracket": (lo, hi), "history":
    [(betas, values), ...]}.  Raises ValueError when the target is not
    bracketed by the starting [lo, hi]."""
    if not (0 <= lo < hi) or n_candidates < 2:
        raise ValueError("need 0 <= lo < hi and at least two candidates")
    run = run_batch or _gpu_batch(K, E0, r, proposal, h3_mode, grid_N, 16)
    lo0, hi0 = lo, hi
    history = []
    for step in range(n_steps):
        betas = np.linspace(lo, hi, n_candidates)
        h = betas[1] - betas[0]
        stats = run(betas, step * n_candidates, proposals_per_candidate, seed + step)
        vals = np.array([statistic(s, K, b) for s, b in zip(stats, betas)], dtype=np.float64)
        history.append((betas, vals))
        g = vals - target
        if not np.all(np.isfinite(g)):
            raise ValueError("statistic is not finite for every candidate (too few accepted samples?)")
        # straight line through all candidates: its root guides the choice
        # among several noisy crossings and replaces a crossing lost to noise
        slope, icpt = np.polyfit(betas, vals, 1)
        b_lin = (target - icpt) / slope if slope != 0 else 0.5 * (lo + hi)
        sign = np.sign(g)
        cross = np.nonzero(sign[:-1] * sign[1:] <= 0)[0]
        if cross.size == 0:
            if step == 0:
                raise ValueError("target %g not bracketed: statistic spans [%g, %g]" % (target, vals.min(), vals.max()))
            mid = float(np.clip(b_lin, betas[0], betas[-1]))
        else:
            j = int(cross[np.argmin(np.abs(0.5 * (betas[cross] + betas[cross + 1]) - b_lin))])
            mid = 0.5 * (betas[j] + betas[j + 1])
        # next bracket: the crossing interval widened by half a spacing on each
        # side, so that sampling noise at its ends cannot lose the root
        lo, hi = max(lo0, mid - h), min(hi0, mid + h)
    betas, vals = history[-1]
    slope, icpt = np.polyfit(betas, vals, 1)
    beta = float(np.clip((target - icpt) / slope, lo, hi)) if slope != 0 else 0.5 * (lo + hi)
    return {"beta": beta, "bracket": (lo, hi), "history": history}

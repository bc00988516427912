"""Learned proposal: training and use (driver around the library's MLP kernels).

The network maps a parameter point to per-mode log-variance corrections c_k of
the paper's proposal (sigma_k'^2 = sigma_k^2 e^{c_k}).  Training data are
accepted samples of the paper-proposal sampler; every step (forward, loss,
backward, Adam) runs in the library's CUDA kernels.  The corrected proposal
keeps the closed-form density of Eqs. (33)-(38), and the sampler recomputes
the envelope M for it, so the accept test stays exact; its gain over the
paper proposal is exp(log M_paper - log M_learned) in acceptance, because the
corrections have mean zero (prod_k w'_k = prod_k w_k).
"""
from __future__ import annotations

import numpy as np

from . import (PROPOSAL_LEARNED, PROPOSAL_PAPER, Sampler, make_point, tkdv_log_M, tkdv_mlp_create,
               tkdv_mlp_destroy, tkdv_mlp_features, tkdv_mlp_infer, tkdv_mlp_rows, tkdv_mlp_set_data_records,
               tkdv_mlp_step, tkdv_record_bytes)


def collect_accepted(K, points, n_accept, seed=0, pilot=1 << 20, max_proposals=1 << 36, h3_mode=0, grid_N=0,
                     stream=None):
    """Run the paper-proposal sampler on `points` [(beta', E0, C3/C2), ...] until
    every point has n_accept accepted records; returns (sampler, records
    device buffer (torch uint8), record count, per-point alpha*, sigma^2).
    A pilot run measures each point's acceptance, and later runs give each
    point the budget its remaining records need (30 % spare), so that points
    of very different acceptance share one record ring of 2 n_accept records
    per point without one crowding the others out."""
    import torch
    pts = [make_point(bp, E0, r, PROPOSAL_PAPER, point_id=p) for p, (bp, E0, r) in enumerate(points)]
    P = len(points)
    cap = n_accept * P * 2
    S = Sampler(K, pts, h3_mode=h3_mode, grid_N=grid_N, sample_capacity=cap, stream=stream)
    budgets = np.full(P, pilot, dtype=np.uint64)
    used = np.zeros(P, dtype=np.uint64)
    while True:
        S.run_budgets(budgets, seed)
        used += budgets
        acc = np.array([s["n_accepted"] for s in S.stats()])
        need = (acc < n_accept) & (used < max_proposals)
        if not need.any():
            break
        rate = np.maximum(acc, 1) / used.astype(np.float64)
        want = np.ceil((n_accept - acc) * 1.3 / rate)
        budgets = np.where(need, np.clip(want, pilot, min(1 << 32, max_proposals)), 0).astype(np.uint64)
    rb = tkdv_record_bytes(K)
    buf = torch.empty(cap * rb, dtype=torch.uint8, device="cuda")
    n = S.samples(cap, device_dst=buf)
    info = [S.point_info(p) for p in range(P)]
    return S, buf, n, info


def train(K, points, n_accept=1 << 14, steps=300, lr=2e-2, tau=1.0, seed=0, sampler_seed=0, stream=None,
          mlp=None, h3_mode=0, grid_N=0):
    """Train the MLP on accepted samples of `points`; returns (mlp handle,
    per-point corrections c (P x K), loss history, training rows per point).
    The samples come from the paper-proposal sampler in the given H3 form."""
    S, buf, n, info = collect_accepted(K, points, n_accept, seed=sampler_seed, stream=stream, h3_mode=h3_mode,
                                       grid_N=grid_N)
    P = len(points)
    feats = np.array([tkdv_mlp_features(K, bp, E0, r) for bp, E0, r in points])
    w_paper = [1.0 / np.asarray(s2) for (_, _, s2) in info]
    zcoef = np.array([[bp / (E0 * K * K), r] for bp, E0, r in points])
    m = mlp if mlp is not None else tkdv_mlp_create(seed)
    tkdv_mlp_set_data_records(m, [K] * P, feats, w_paper, zcoef, buf, n, K, n_accept)
    S.close()
    del buf
    hist = []
    for _ in range(steps):
        hist.append(tkdv_mlp_step(m, lr, tau, True))
    hist.append(tkdv_mlp_step(m, lr, tau, False))
    c = tkdv_mlp_infer(m, feats, [K] * P)[:, :K]
    return m, c, np.array(hist), tkdv_mlp_rows(m, P)


def infer(mlp, K, points):
    """Corrections c (P x K) of the trained network for points [(beta', E0, C3/C2), ...]."""
    feats = np.array([tkdv_mlp_features(K, bp, E0, r) for bp, E0, r in points])
    return tkdv_mlp_infer(mlp, feats, [K] * len(points))[:, :K]


def learned_points(K, points, c, point_id0=0):
    """tkdv_point structs of the learned proposal for `points` with corrections c."""
    return [make_point(bp, E0, r, PROPOSAL_LEARNED, point_id=point_id0 + p, log_var_correction=c[p])
            for p, (bp, E0, r) in enumerate(points)]


def predicted_gain(K, point, c):
    """Acceptance of the learned proposal over the paper's: exp(log M_paper - log M_learned)
    (the corrections have mean zero, so prod_k w'_k = prod_k w_k)."""
    from . import tkdv_alpha_star
    bp, E0, r = point
    a = tkdv_alpha_star(K, bp)
    k = np.arange(1, K + 1)
    s2 = 1.0 / (1.0 + a * bp * k * k / K**3)
    lm_p = tkdv_log_M(K, bp, E0, r, s2)
    lm_l = tkdv_log_M(K, bp, E0, r, s2 * np.exp(np.asarray(c[:K])))
    return float(np.exp(lm_p - lm_l)), lm_p, lm_l


def close(m):
    tkdv_mlp_destroy(m)

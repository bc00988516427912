"""Write tests/golden/learned_corrections.json: learned-proposal corrections
c_k and their envelopes, made with the oracle alone.

For two points of the 32-mode extreme-event workload (E0 = 1, beta' = 20 and
60 at beta' C3/C2 = 9000), the oracle's paper-proposal sampler draws accepted
samples; the oracle's FP64 network (oracle/mlp.py, 4 -> 64 -> 64 -> 64) is
trained on them by Adam on the tempered loss J_tau; its gauge-fixed output is
the correction c (sigma_k'^2 = sigma_k^2 e^{c_k}); and the oracle's
Nelder-Mead gives log M (Eq. 45) of the diagonal proposal with those
variances.  The GPU test of the grid form with the learned proposal takes c
and log M from this file.  Calls only oracle/.

    python tests/golden/make_learned.py
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from oracle import mlp as OM  # noqa: E402

K, E0, LAM = 32, 1.0, 9000.0
BETAS = (20.0, 60.0)
N_ACCEPT = 1 << 11
TAU = 0.5
STEPS, LR = 300, 2e-2


def envelope_cache():
    return json.load(open(os.path.join(HERE, "envelopes.json")))["points"]


def key(bp, r, prop):
    return "K%d_E%.17g_b%.17g_r%.17g_p%d" % (K, E0, bp, r, prop)


def accepted(pt, pid, n_accept):
    """(s (n, K), z (n,)) of the first n_accept accepted samples of point pid."""
    s_rows, z_rows = [], []
    idx0, step = 0, 1 << 24
    while sum(len(s) for s in s_rows) < n_accept:
        _, rec = O.run_accepted(pt, 0, pid, idx0, step, cap=1 << 16)
        xh = rec["xhat"]
        s_rows.append(xh[:, :K] ** 2 + xh[:, K:2 * K] ** 2)
        z_rows.append(-(pt.beta_p / (E0 * K * K)) * (rec["H2"] - pt.r * rec["H3"]))
        idx0 += step
    return np.concatenate(s_rows)[:n_accept], np.concatenate(z_rows)[:n_accept]


def adam(theta, grads, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    for name in theta:
        m, v = state.setdefault(name, (np.zeros_like(theta[name]), np.zeros_like(theta[name])))
        g = grads[name]
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        state[name] = (m, v)
        theta[name] = theta[name] - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)


def main():
    env = envelope_cache()
    pts, s_list, z_list, wp, feats = [], [], [], [], []
    for p, bp in enumerate(BETAS):
        r = LAM / bp
        pt = O.make_point(K, E0, bp, r, O.PAPER, logM=env[key(bp, r, O.PAPER)]["logM"])
        s, z = accepted(pt, p, N_ACCEPT)
        pts.append(pt)
        s_list.append(s)
        z_list.append(z)
        wp.append(1.0 / np.array(pt.sigma2[:K]))
        feats.append(OM.features(K, bp, E0, r))
    feats = np.array(feats)
    theta = OM.init_theta(1)
    state = {}
    hist = []
    for t in range(1, STEPS + 1):
        J, g = OM.loss_and_grad(theta, feats, [K] * len(BETAS), wp, s_list, z_list, TAU)
        hist.append(J)
        adam(theta, g, state, LR, t)
    out, _ = OM.forward(theta, feats)
    res = {}
    for p, bp in enumerate(BETAS):
        r = LAM / bp
        c = OM.gauge(out[p], K)
        s2 = np.array(pts[p].sigma2[:K]) * np.exp(c)
        pd = O.make_point(K, E0, bp, r, O.DIAG, sigma2=s2)
        lm = O.log_M(pd, 4)
        res["b%.17g" % bp] = {"K": K, "E0": E0, "beta_p": bp, "r": r, "c": c.tolist(), "sigma2": s2.tolist(),
                              "logM": lm, "logM_paper": pts[p].logM,
                              "predicted_gain": math.exp(pts[p].logM - lm)}
    with open(os.path.join(HERE, "learned_corrections.json"), "w") as f:
        json.dump({"_source": "oracle only: oracle.run_accepted samples, oracle/mlp.py network trained by Adam "
                              "on J_tau (tau = %g, %d steps, %d accepted samples per point), oracle.log_M of "
                              "the diagonal proposal; written by make_learned.py" % (TAU, STEPS, N_ACCEPT),
                   "loss_first_last": [hist[0], hist[-1]], "points": res}, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()

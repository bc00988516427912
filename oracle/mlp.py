"""FP64 oracle of the learned proposal (MLP inference, loss and gradients).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The learned proposal keeps the paper's closed-form proposal density (Eqs.
33-38): a centred Gaussian with pair variances sigma_k'^2, projected onto the
sphere, has density g(xh) = prod_k w'_k * Q(xh)^-K against the uniform measure
mu0, with w'_k = 1/sigma_k'^2 and Q = sum_k w'_k s_k, s_k = xh_k^2 + xh_{K+k}^2.
The network only moves the variances: sigma_k'^2 = sigma_k^2(paper) e^{c_k}, so
w'_k = w_k e^{-c_k}.  g is unchanged by w' -> lambda w', so c is gauge-fixed to
mean zero over k = 1..K.

Network: 4 -> 64 -> 64 -> 64, tanh hidden layers, linear output; weights are
BF16 values (held here as float64), biases float64.  Output entries k > K
are ignored.

Loss of one parameter point, over accepted samples i = 1..n (draws from f):
    ell_i = -log g(xh_i) = K ln Q_i - sum_k ln w'_k
    J     = mean_i ell_i                               (tau = inf: KL(f || g) + const)
    J_tau = tau * log mean_i exp((z_i + ell_i) / tau)  (z_i = -beta H_i = log f + const)
As tau -> 0, J_tau tends to the largest log(f/g) over the samples, the
quantity that sets the acceptance rate 1/sup(f/g).
"""
from __future__ import annotations

import math

import numpy as np

H = 64
KOUT = 64


def features(K, beta_p, E0, r):
    """Network input of one parameter point (the paper's K, E0, beta', C3/C2;
    beta' C3/C2 is the H3 prefactor that Tables 1-2 step through)."""
    lam = beta_p * r
    return np.array([math.log(max(beta_p, 1e-3)) / math.log(100.0), math.log(E0),
                     math.log1p(max(lam, 0.0) / 100.0) / math.log(100.0), K / 64.0])


def unpack(theta):
    """theta: dict with W1 (64x4), b1 (64), W2 (64x64), b2, W3 (64x64), b3."""
    return theta["W1"], theta["b1"], theta["W2"], theta["b2"], theta["W3"], theta["b3"]


def forward(theta, f):
    """f: (P, 4) -> c_raw (P, 64), cache."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    a1 = f @ W1.T + b1
    h1 = np.tanh(a1)
    a2 = h1 @ W2.T + b2
    h2 = np.tanh(a2)
    out = h2 @ W3.T + b3
    return out, (f, h1, h2)


def gauge(c_raw, K):
    """Mask k > K and subtract the mean over k <= K."""
    c = np.array(c_raw[..., :K], dtype=np.float64)
    return c - c.mean(axis=-1, keepdims=True)


def point_loss(c, w_paper, s, z=None, tau=None):
    """Loss J (or J_tau) of one point and dJ/dc (length K).
    c: (K,) gauge-fixed log-variance corrections; w_paper: (K,) 1/sigma_k^2(paper);
    s: (n, K) pair energies of the accepted samples; z: (n,) -beta H_i."""
    K = c.shape[0]
    w = w_paper * np.exp(-c)
    Q = s @ w
    ell = K * np.log(Q) - np.sum(np.log(w))
    if tau is None or not np.isfinite(tau):
        p = np.full(len(ell), 1.0 / len(ell))
        J = float(np.mean(ell))
    else:
        a = (z + ell) / tau
        m = a.max()
        e = np.exp(a - m)
        p = e / e.sum()
        J = float(tau * (m + math.log(e.mean())))
    # d ell_i / d c_k = 1 - K w_k s_ik / Q_i
    g = 1.0 - K * (p / Q) @ (s * w)
    return J, g


def loss_and_grad(theta, feats, Ks, w_papers, s_list, z_list=None, tau=None):
    """Total loss over points (sum) and the gradient with respect to every
    parameter, by backpropagation through the gauge fixing and the MLP."""
    out, (f, h1, h2) = forward(theta, feats)
    P = feats.shape[0]
    dout = np.zeros_like(out)
    total = 0.0
    for p in range(P):
        K = Ks[p]
        c = gauge(out[p], K)
        z = None if z_list is None else z_list[p]
        J, g = point_loss(c, w_papers[p], s_list[p], z, tau)
        total += J
        dc = g - g.mean()  # through c = c_raw - mean(c_raw)
        dout[p, :K] = dc
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    grads = {}
    grads["W3"] = dout.T @ h2
    grads["b3"] = dout.sum(0)
    dh2 = dout @ W3
    da2 = dh2 * (1 - h2 * h2)
    grads["W2"] = da2.T @ h1
    grads["b2"] = da2.sum(0)
    dh1 = da2 @ W2
    da1 = dh1 * (1 - h1 * h1)
    grads["W1"] = da1.T @ f
    grads["b1"] = da1.sum(0)
    return total, grads


def init_theta(seed=0, scale=0.3):
    """Random hidden layers, zero output layer: c = 0 (the paper proposal) at start."""
    g = np.random.default_rng(seed)
    return {"W1": g.normal(0, scale, (H, 4)), "b1": np.zeros(H),
            "W2": g.normal(0, scale / math.sqrt(H) * 4, (H, H)), "b2": np.zeros(H),
            "W3": np.zeros((KOUT, H)), "b3": np.zeros(KOUT)}


def bf16_round(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    x = np.asarray(a, dtype=np.float32).copy()
    u = x.view(np.uint32)
    u = (u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return u.view(np.float32).astype(np.float64)

"""Pins of the learned-proposal oracle (oracle/mlp.py)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp


def random_theta(seed):
    g = np.random.default_rng(seed)
    th = mlp.init_theta(seed)
    th["W3"] = g.normal(0, 0.05, th["W3"].shape)
    th["b3"] = g.normal(0, 0.05, 64)
    th["b1"] = g.normal(0, 0.1, 64)
    return th


def sphere_s(rng, n, K, sigma2=None):
    """Pair energies of projected Gaussian draws (uniform on the sphere if sigma2 is None)."""
    z = rng.standard_normal((n, 2 * K))
    if sigma2 is not None:
        sd = np.sqrt(np.concatenate([sigma2, sigma2]))
        z = z * sd
    x = z / np.linalg.norm(z, axis=1, keepdims=True)
    return x[:, :K] ** 2 + x[:, K:] ** 2


def test_proposal_density_is_normalised():
    """g(xh) = prod_k w_k Q^-K integrates to one against mu0 (Eqs. 33-38): its mean
    over uniform points of the sphere is 1."""
    rng = np.random.default_rng(0)
    for K in (4, 8):
        w = np.exp(rng.normal(0, 0.4, K))
        s = sphere_s(rng, 400000, K)
        gvals = np.prod(w) * (s @ w) ** (-K)
        assert abs(gvals.mean() - 1) < 5 * gvals.std() / math.sqrt(len(gvals))


def test_nll_matches_a_gaussian_fit():
    """Draws from a projected Gaussian with variances sigma2: the per-mode
    correction that minimises the mean NLL starting from sigma2 * e^{c} is c = 0
    (the gradient vanishes there), and is nonzero from any other start."""
    rng = np.random.default_rng(1)
    K = 8
    s2 = np.exp(rng.normal(0, 0.5, K))
    s = sphere_s(rng, 200000, K, s2)
    J0, g0 = mlp.point_loss(np.zeros(K), 1.0 / s2, s)
    assert np.max(np.abs(g0)) < 0.02
    J1, g1 = mlp.point_loss(np.zeros(K), np.ones(K), s)
    assert J1 > J0 and np.max(np.abs(g1)) > 0.1


@pytest.mark.parametrize("tau", [None, 1.0, 0.3])
def test_gradient_by_central_differences(tau):
    rng = np.random.default_rng(2)
    th = random_theta(3)
    Ks = [8, 16]
    feats = np.array([mlp.features(8, 20.0, 1.0, 60.0), mlp.features(16, 40.0, 0.7, 30.0)])
    wp = [np.exp(rng.normal(0, 0.3, K)) for K in Ks]
    s_list = [sphere_s(rng, 500, K) for K in Ks]
    z_list = [rng.normal(0, 1, 500) for _ in Ks]
    J, grads = mlp.loss_and_grad(th, feats, Ks, wp, s_list, z_list, tau)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = th[name].reshape(-1)
        for j in rng.choice(flat.size, 6, replace=False):
            old = flat[j]
            flat[j] = old + h
            Jp, _ = mlp.loss_and_grad(th, feats, Ks, wp, s_list, z_list, tau)
            flat[j] = old - h
            Jm, _ = mlp.loss_and_grad(th, feats, Ks, wp, s_list, z_list, tau)
            flat[j] = old
            fd = (Jp - Jm) / (2 * h)
            an = grads[name].reshape(-1)[j]
            assert abs(fd - an) <= 1e-6 * (1 + abs(fd)), (name, j, fd, an)


def test_gauge_invariance_and_zero_start():
    rng = np.random.default_rng(4)
    K = 8
    wp = np.exp(rng.normal(0, 0.3, K))
    s = sphere_s(rng, 1000, K)
    c = rng.normal(0, 0.2, K)
    c -= c.mean()
    J, _ = mlp.point_loss(c, wp, s)
    J2, _ = mlp.point_loss(c + 0.7, wp, s)  # w' -> e^{-0.7} w' leaves g unchanged
    assert abs(J - J2) < 1e-10
    th = mlp.init_theta(0)
    out, _ = mlp.forward(th, mlp.features(K, 20.0, 1.0, 60.0)[None, :])
    assert np.all(mlp.gauge(out[0], K) == 0)  # zero output layer: the paper proposal


def test_tempered_loss_limits():
    rng = np.random.default_rng(5)
    K = 8
    wp = np.ones(K)
    s = sphere_s(rng, 2000, K)
    z = rng.normal(0, 1, 2000)
    ell = K * np.log(s @ wp)
    Jmean, _ = mlp.point_loss(np.zeros(K), wp, s, z, None)
    assert abs(Jmean - ell.mean()) < 1e-12
    Jsmall, _ = mlp.point_loss(np.zeros(K), wp, s, z, 1e-3)
    assert abs(Jsmall - np.max(z + ell)) < 0.02

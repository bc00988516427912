"""Property-based pins of the oracle over the whole mode range K = 1..128
(hypothesis draws K, E0 and a state on the sphere):

* the double sum of Eq. (42), the triple sum of Eq. (41) and the grid
  cubature of Eq. (2) with N = 3K + 1 points give the same H3;
* |u(xi)| <= sqrt(2 K E0 / pi) (Cauchy-Schwarz, attained by the Dirichlet
  kernel of Eq. 46), and H2 = E0 S with 1 <= S <= K^2;
* H3 is odd under xhat -> -xhat and invariant under the translation
  xi -> xi + s, which rotates mode k by the angle k s.
"""
import math

import numpy as np
import pytest

import oracle as O

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")


def sphere(seed, K):
    x = np.random.default_rng(seed).standard_normal(2 * K)
    return x / np.linalg.norm(x)


@hyp.settings(max_examples=60, deadline=None)
@hyp.given(K=st.integers(1, 128), E0=st.floats(0.1, 5.0), seed=st.integers(0, 2**32 - 1),
           s=st.floats(-math.pi, math.pi), xi=st.floats(-math.pi, math.pi))
def test_hamiltonian_forms_and_bounds(K, E0, seed, s, xi):
    xh = sphere(seed, K)
    d = O.H3_double(K, E0, xh)
    scale = 1e-12 * (1.0 + K ** 1.5) * E0 ** 1.5
    assert abs(O.H3_triple(K, E0, xh) - d) <= scale
    assert abs(O.H3_grid(K, E0, xh, 3 * K + 1) - d) <= scale
    H2 = O.H2(K, E0, xh)
    assert E0 * (1 - 1e-12) <= H2 <= E0 * K * K * (1 + 1e-12)
    assert abs(O.u_at(K, E0, xh, xi)) <= math.sqrt(2 * K * E0 / math.pi) * (1 + 1e-12)
    assert abs(O.H3_double(K, E0, -xh) + d) <= scale
    uk = xh[:K] - 1j * xh[K:]
    rot = uk * np.exp(1j * np.arange(1, K + 1) * s)
    xs = np.concatenate([rot.real, -rot.imag])
    assert abs(O.H3_double(K, E0, xs) - d) <= scale
    assert abs(O.u_at(K, E0, xs, xi) - O.u_at(K, E0, xh, xi + s)) <= 1e-12 * math.sqrt(K * E0)

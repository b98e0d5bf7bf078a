"""Identities behind a 132-byte-per-voxel schedule of the ADMM pass (Eq. 28, Eq. 30), checked on
the oracle's operators. Such a schedule keeps a = div^- A* e and b = div^- A* v per voxel, so
that the forward FFT pass reads 8 bytes instead of the 12 state components (d = a - b / rho), and
has the update pass produce the next a and b. These tests pin the algebra that makes that
possible:

* P_K leaves the divergence of A* unchanged: div^- A* xi^{k+1/2} = div^- A* w for w = e - v / rho,
  because A* P_K(w) = grad^+ phi + xi_bar with div^- grad^+ phi = div^- A* w (zero mean).
* Hence div^- A* z = rho a - beta b for the pre-projection point z = v + rho (alpha xi^{k+1/2}
  - beta e), alpha = 2 (1 - delta), beta = 1 - 2 delta, with no stencil on the new state.
* Only the clip excess c = z - P_C(z) needs one: a' = div^- A* c / rho, b' = rho a - beta b -
  div^- A* c.
"""

import numpy as np
import pytest

from oracle import ccmf_oracle as O

SHAPES = [(4, 5, 6), (8, 8, 8), (3, 7, 5)]


def dA(w):
    return O.div_minus(O.op_A_adj(w))


def state(shape, seed):
    rng = np.random.default_rng(seed)
    gamma = rng.uniform(0.2, 1.5, shape)
    e = rng.standard_normal((6,) + shape)
    v = rng.standard_normal((6,) + shape)
    return gamma, e, v


@pytest.mark.parametrize("shape", SHAPES)
def test_projection_keeps_divergence(shape):
    _, e, v = state(shape, 11)
    rho = 0.7
    xi_bar = np.array([0.36, 0.48, 0.8])
    w = e - v / rho
    xi_half = O.project_K(w, xi_bar)
    # A* of the projection is a gradient plus the prescribed mean flux (Eq. 28)
    u = O.op_A_adj(xi_half) - O.const_field(xi_bar, shape)
    phi = O.laplacian_pinv(O.div_minus(u))
    np.testing.assert_allclose(u, O.grad_plus(phi), rtol=0, atol=1e-11)
    np.testing.assert_allclose(dA(xi_half), dA(w), rtol=0, atol=1e-11)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("delta", [0.25, 0.5])
def test_next_divergences_from_a_b_and_clip_excess(shape, delta):
    gamma, e, v = state(shape, 12)
    rho = 1.3
    xi_bar = np.array([0.0, 0.6, 0.8])
    alpha, beta = 2.0 * (1.0 - delta), 1.0 - 2.0 * delta
    a, b = dA(e), dA(v)
    xi_half, e_new, v_new = O.admm_step(e, v, rho, gamma, xi_bar, delta)
    z = v + rho * (alpha * xi_half - beta * e)
    np.testing.assert_allclose(dA(z), rho * a - beta * b, rtol=0, atol=1e-10)
    c = z - O.project_C(z, gamma)
    assert np.any(np.abs(c) > 0)   # the clip is active somewhere, so the test is not vacuous
    np.testing.assert_allclose(dA(e_new), dA(c) / rho, rtol=0, atol=1e-10)
    np.testing.assert_allclose(dA(v_new), rho * a - beta * b - dA(c), rtol=0, atol=1e-10)
    # the next forward pass's input: d' = a' - b' / rho' for any rho'
    rho_next = 0.9
    np.testing.assert_allclose(dA(e_new - v_new / rho_next), dA(c) / rho - (rho * a - beta * b - dA(c)) / rho_next,
                               rtol=0, atol=1e-10)

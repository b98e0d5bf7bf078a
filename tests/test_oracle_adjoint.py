"""Pins of the oracle gradient (reverse mode through K replayed updates of Eq. 30):
central finite differences of the same replayed map, a directional derivative
that crosses no projection kink, and the envelope derivative |xi*| / N at
convergence (Danskin on the min-cut value of Eq. 21)."""

import numpy as np
import pytest

# rho^0 = 0.9 min(gamma): with rho^0 = min(gamma) the first update puts the weakest voxel exactly
# on the kink |z| = gamma of the projection, where a central difference straddles two branches.

from oracle import ccmf_adjoint as D
from oracle import ccmf_oracle as O
from paper_2103_05968_gb300 import microstructure as M


@pytest.mark.parametrize("seed,shape,xi", [(1, (5, 4, 6), [0, 0, 1]), (2, (6, 6, 3), [0.36, 0.48, 0.8])])
def test_gradient_matches_central_differences(seed, shape, xi):
    g = M.uniform_random(shape, 0.5, 1.5, seed)
    rho = D.record_rho(g, xi, 25, O.Params(rho0=0.9 * float(g.min())))
    J, grad = D.gradient(g, xi, rho)
    rng = np.random.default_rng(seed + 10)
    for _ in range(3):
        eta = rng.standard_normal(shape)
        h = 1e-6
        jp, _, _, _ = D.forward_replay(g + h * eta, xi, rho, keep=False)
        jm, _, _, _ = D.forward_replay(g - h * eta, xi, rho, keep=False)
        fd = (jp - jm) / (2 * h)
        ad = float(np.sum(grad * eta))
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-3)


def test_gradient_single_voxel_derivative():
    """One voxel at a time on a tiny grid (every component of the gradient)."""
    g = M.uniform_random((3, 2, 4), 0.6, 1.4, 7)
    xi = [0.6, 0.0, 0.8]
    rho = D.record_rho(g, xi, 15, O.Params(rho0=0.9 * float(g.min())))
    _, grad = D.gradient(g, xi, rho)
    h = 1e-7
    for idx in np.ndindex(g.shape):
        gp = g.copy()
        gm = g.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (D.forward_replay(gp, xi, rho, keep=False)[0] - D.forward_replay(gm, xi, rho, keep=False)[0]) / (2 * h)
        assert abs(fd - grad[idx]) <= 1e-6 * max(abs(fd), 1e-3)


def test_envelope_gradient_at_convergence():
    """At convergence the gradient approaches |xi*(x)| / N (Danskin on Eq. 21)."""
    g = M.single_sphere((16, 16, 16), (8.0, 8.0, 8.0), 4.0, 0.1, 1.0)
    xi = [0, 0, 1]
    r = O.solve(g, xi, O.Params(tol=1e-7, max_iter=20000))
    assert r.converged
    rho = [h[1] for h in r.history]
    _, grad = D.gradient(g, xi, rho)
    env = np.sqrt(np.sum(r.cut ** 2, axis=0)) / g.size
    cos = float(np.sum(grad * env) / np.sqrt(np.sum(grad ** 2) * np.sum(env ** 2)))
    assert cos > 0.99
    # 1-homogeneity of the optimal value (Euler): sum_x gamma dJ/dgamma = gamma_eff
    assert abs(float(np.sum(g * grad)) - r.gamma_eff) < 1e-3 * r.gamma_eff

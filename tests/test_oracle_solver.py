"""Pins of the oracle's ADMM (Eq. 30) against closed forms, the dense barrier
solver of the face-based problem, the paper's single-sphere result (Sec. 4.2)
and invariances of the problem."""

import json
import math
import os

import numpy as np
import pytest

from oracle import ccmf_oracle as O
from oracle import dense_maxflow as D
from paper_2103_05968_gb300 import microstructure as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_homogeneous_any_normal():
    g = np.full((6, 7, 8), 1.7)
    for xi in ([0.6, 0.8, 0.0], [1.0, 2.0, 2.0], [0.0, 0.0, -1.0]):
        r = O.solve(g, xi, O.Params(tol=1e-9))
        assert r.converged
        assert abs(r.gamma_eff - 1.7) < 1e-8
        assert abs(r.gamma_primal - 1.7) < 1e-8


def test_laminate_closed_forms():
    layers = np.random.default_rng(1).uniform(0.5, 2.0, 8)
    g = M.laminate(4, 4, layers)
    r = O.solve(g, [0, 0, 1], O.Params(tol=1e-9, max_iter=50000))
    assert abs(r.gamma_eff - layers.min()) < 1e-6 * layers.min()      # stacking axis: weakest layer
    r = O.solve(g, [1, 0, 0], O.Params(tol=1e-9))
    assert abs(r.gamma_eff - layers.mean()) < 1e-9                      # in plane: thickness mean
    r = O.solve(g, [0, 0.6, 0.8], O.Params(tol=1e-9, max_iter=50000))
    assert layers.min() - 1e-8 <= r.gamma_eff <= layers.mean() + 1e-8


def test_axis_normal_bounds_random_columns():
    """mean_ij(min_k gamma) <= gamma_eff(e3) <= min_k mean_ij gamma (the bounds of the golden note)."""
    g = M.uniform_random((5, 4, 6), 0.4, 1.6, 21)
    r = O.solve(g, [0, 0, 1], O.Params(tol=1e-5, max_iter=3000), record_history=False)
    lo = g.min(axis=2).mean()
    hi = g.mean(axis=(0, 1)).min()
    assert lo - 1e-4 <= r.gamma_eff <= hi + 1e-4
    assert lo - 1e-4 <= r.gamma_primal <= hi + 1e-4


@pytest.mark.parametrize("seed,xi", [(3, [0.3, -0.5, 0.8]), (4, [0.0, 0.0, 1.0]), (5, [1.0, 1.0, 0.0])])
def test_dense_barrier_agreement(seed, xi):
    """The converged ADMM value equals the maximum flow of the face-based problem (Eq. 6 - Eq. 8)."""
    g = M.uniform_random((4, 4, 4), 0.5, 2.0, seed)
    val, _, gap = D.max_flow(g, xi, gap_tol=1e-10)
    r = O.solve(g, xi, O.Params(tol=1e-10, max_iter=100000))
    assert r.converged
    assert abs(r.gamma_eff - val) <= 1e-8 * val + gap
    assert abs(r.gamma_primal - val) <= 1e-8 * val + gap


@pytest.mark.slow
@pytest.mark.parametrize("n,seed,xi", [(6, 41, [0.3, -0.5, 0.8]), (8, 42, [0.0, 0.0, 1.0])])
def test_dense_barrier_agreement_6_and_8(n, seed, xi):
    """The same agreement on 6^3 and 8^3 grids (648 and 1536 face unknowns)."""
    g = M.uniform_random((n, n, n), 0.5, 2.0, seed)
    val, _, gap = D.max_flow(g, xi, gap_tol=1e-9)
    r = O.solve(g, xi, O.Params(tol=1e-10, max_iter=200000), record_history=False)
    assert r.converged
    assert abs(r.gamma_eff - val) <= 1e-8 * val + gap
    assert abs(r.gamma_primal - val) <= 1e-8 * val + gap


def test_dense_barrier_anisotropic_grid():
    g = M.random_two_phase((2, 3, 5), 0.4, 0.2, 1.0, 6)
    xi = [0.2, 0.4, -0.9]
    val, _, gap = D.max_flow(g, xi, gap_tol=1e-10)
    r = O.solve(g, xi, O.Params(tol=1e-10, max_iter=200000))
    assert abs(r.gamma_eff - val) <= 1e-7 * val + gap
    assert abs(r.gamma_primal - val) <= 1e-7 * val + gap


def test_config_single_sphere_32_closed_form():
    gold = json.load(open(os.path.join(GOLDEN, "single_sphere_32_e3.json")))
    g = M.single_sphere(gold["n"], gold["centre"], gold["radius"], gold["gamma_sphere"], gold["gamma_matrix"])
    assert int(np.sum(g == gold["gamma_sphere"])) == gold["sphere_voxels"]
    assert int(np.sum(g[:, :, 15] == gold["gamma_sphere"])) == gold["central_layer_voxels"]
    exact = gold["gamma_eff"]
    assert exact == 1.0 - 0.9 * gold["central_layer_voxels"] / 1024.0
    r = O.solve(g, gold["xi_bar"], O.Params(tol=1e-6))
    assert r.converged
    assert exact - 1e-9 <= r.gamma_primal <= exact + 5e-6       # the min-cut value is an upper bound
    assert abs(r.gamma_eff - exact) <= 5e-6                      # reported max-flow value


@pytest.mark.slow
def test_paper_single_sphere_64():
    """Sec. 4.2: gamma_eff = gamma_matrix for the tougher centred ball (printed result)."""
    gold = json.load(open(os.path.join(GOLDEN, "single_sphere_64.json")))
    g = M.single_sphere(gold["n"], gold["centre"], gold["radius"], gold["gamma_sphere"], gold["gamma_matrix"])
    p = O.Params(tol=gold["tol"], rho_rule=O.RHO_CONST, rho0=float(g.min()))
    r = O.solve(g, gold["xi_bar"], p, record_history=False)
    assert r.converged
    assert abs(r.gamma_eff / gold["gamma_matrix"] - gold["gamma_eff_over_gamma_matrix"]) < 1e-3


def test_multiplier_feasible_every_iteration():
    g = M.random_two_phase((6, 5, 4), 0.3, 0.1, 1.0, 7)
    xi = np.array([0.48, 0.6, 0.64])
    e = O.op_A(O.const_field(xi, g.shape))
    v = np.zeros((6,) + g.shape)
    rho = O.initial_rho(g, O.Params())
    for _ in range(30):
        _, e, v = O.admm_step(e, v, rho, g, xi, 0.25)
        assert np.all(np.sqrt(np.sum(v * v, axis=0)) <= g * (1 + 1e-12) + 1e-14)


def test_scaling_equivariance():
    """gamma -> 2 gamma (rho^0 proportional to gamma): xi and e unchanged, v doubled."""
    g = M.random_two_phase((6, 6, 6), 0.3, 0.25, 1.0, 8)
    xi = [0.0, 0.6, 0.8]
    p = O.Params(fixed_iters=40)
    a = O.solve(g, xi, p)
    b = O.solve(2.0 * g, xi, p)
    np.testing.assert_array_equal(a.e, b.e)
    np.testing.assert_array_equal(2.0 * a.v, b.v)
    assert b.gamma_eff == 2.0 * a.gamma_eff


def test_normal_sign_translation_permutation():
    g = M.random_two_phase((6, 5, 4), 0.3, 0.25, 1.0, 9)
    xi = np.array([0.36, 0.48, 0.8])
    p = O.Params(tol=1e-8, max_iter=20000)
    a = O.solve(g, xi, p)
    b = O.solve(g, -xi, p)
    assert abs(a.gamma_eff - b.gamma_eff) < 1e-7
    c = O.solve(np.roll(g, (2, 1, 3), axis=(0, 1, 2)), xi, p)
    assert abs(a.gamma_eff - c.gamma_eff) < 1e-7
    gp = np.transpose(g, (2, 0, 1))
    d = O.solve(gp, xi[[2, 0, 1]], p)
    assert abs(a.gamma_eff - d.gamma_eff) < 1e-7


def test_translation_fixed_iters_fields_shift():
    g = M.random_two_phase((6, 5, 4), 0.3, 0.25, 1.0, 10)
    xi = [0.36, 0.48, 0.8]
    p = O.Params(fixed_iters=15)
    a = O.solve(g, xi, p)
    c = O.solve(np.roll(g, (2, 1, 3), axis=(0, 1, 2)), xi, p)
    np.testing.assert_allclose(np.roll(a.e, (2, 1, 3), axis=(1, 2, 3)), c.e, atol=1e-12)
    np.testing.assert_allclose(np.roll(a.v, (2, 1, 3), axis=(1, 2, 3)), c.v, atol=1e-12)


def test_two_dimensional_column_min_cut():
    """N1 = N2 = 1: a single column along z; the cut sits in the weakest voxel."""
    col = np.array([1.0, 0.7, 0.45, 0.9, 1.2])[None, None, :]
    r = O.solve(col, [0, 0, 1], O.Params(tol=1e-10, max_iter=100000))
    assert abs(r.gamma_eff - 0.45) < 1e-8


def test_resume_is_bit_identical():
    g = M.random_two_phase((5, 6, 4), 0.3, 0.25, 1.0, 11)
    xi = [0.0, 0.6, 0.8]
    full = O.solve(g, xi, O.Params(fixed_iters=30))
    half = O.solve(g, xi, O.Params(fixed_iters=12))
    rest = O.solve(g, xi, O.Params(fixed_iters=18), e0=half.e, v0=half.v, rho0_state=half.rho)
    np.testing.assert_array_equal(full.e, rest.e)
    np.testing.assert_array_equal(full.v, rest.v)
    assert full.rho == rest.rho


def test_penalty_rules_agree():
    """BB and LTD (text after Eq. 30), the constant lower-bound penalty (Sec. 4.3) and residual
    balancing (Sec. 4.3 appendix) approach the same optimum, inside the axis-normal bounds."""
    g, _ = M.boolean_spheres((10, 10, 10), 2.0, 0.2, 0.3, 1.0, 12)
    lo = g.min(axis=2).mean()
    hi = g.mean(axis=(0, 1)).min()
    vals = []
    for rule in (O.RHO_BB, O.RHO_LTD, O.RHO_CONST, O.RHO_RB):
        r = O.solve(g, [0, 0, 1], O.Params(tol=1e-4, max_iter=3000, rho_rule=rule), record_history=False)
        assert lo - 1e-9 <= r.gamma_eff and r.gamma_primal <= hi + 1e-9
        vals.append(r.gamma_eff)
    assert max(vals) - min(vals) < 2e-3 * vals[0]


def test_strong_duality_at_convergence():
    g, _ = M.boolean_spheres((12, 12, 12), 2.0, 0.2, 0.3, 1.0, 13)
    r = O.solve(g, [0, 0, 1], O.Params(tol=1e-8, max_iter=50000))
    assert r.converged
    assert abs(r.gamma_primal - r.gamma_dual) < 1e-6


def test_residual_balancing_direction():
    """Residual balancing (He et al., the fourth strategy of the Sec. 4.3 study): a primal
    residual more than 10x the dual residual rho |e^{k+1} - e^k| raises rho by the step
    factor, a dual residual more than 10x the primal one lowers it, anything between keeps it.
    Here |e^{k+1} - e^k| = 0.5 in every component (L2 norm over 6 components: sqrt(6 * 0.25))."""
    shape = (2, 2, 2)
    e_old = np.zeros((6,) + shape)
    e_new = np.full((6,) + shape, 0.5)
    v = np.zeros((6,) + shape)
    p = O.Params(rho_step_max=2.0)
    rho = 0.4
    s = rho * np.sqrt(6 * 0.25)          # dual residual, 0.4899
    assert O.next_rho(rho, O.RHO_RB, e_old, e_new, v, v, p, primal_res=11 * s) == 0.8
    assert O.next_rho(rho, O.RHO_RB, e_old, e_new, v, v, p, primal_res=s / 11) == 0.2
    assert O.next_rho(rho, O.RHO_RB, e_old, e_new, v, v, p, primal_res=s) == 0.4
    assert O.next_rho(rho, O.RHO_RB, e_old, e_new, v, v, p, primal_res=9 * s) == 0.4

"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case swaps one oracle function for a plausible wrong version and checks
that the corresponding pin (face-based problem, closed form or dense solver)
no longer holds. The oracle module is restored after every case.
"""

import numpy as np
import pytest

from oracle import ccmf_oracle as O
from oracle import dense_maxflow as D
from paper_2103_05968_gb300 import microstructure as M


def _face_pin_holds():
    shape = (4, 5, 6)
    u = np.random.default_rng(1).standard_normal((3,) + shape)
    B, G = D.build_problem(shape)
    f = u.reshape(-1)
    au = O.op_A(u)
    ok_bound = np.allclose((G @ (f * f)).reshape(shape), 2.0 * np.sum(au * au, axis=0), rtol=1e-12)
    ok_div = np.allclose((B @ f).reshape(shape), O.div_minus(u), atol=1e-12)
    return ok_bound and ok_div


def _dense_pin_holds():
    g = M.uniform_random((3, 3, 4), 0.5, 2.0, 3)
    xi = [0.3, -0.5, 0.8]
    val, _, gap = D.max_flow(g, xi, gap_tol=1e-9)
    r = O.solve(g, xi, O.Params(tol=1e-9, max_iter=20000), record_history=False)
    return abs(r.gamma_eff - val) <= 1e-6 * val + gap and abs(r.gamma_primal - val) <= 1e-6 * val + gap


def _homogeneous_pin_holds():
    r = O.solve(np.full((4, 4, 4), 1.3), [0.6, 0.8, 0.0], O.Params(tol=1e-9, max_iter=2000),
                record_history=False)
    return abs(r.gamma_eff - 1.3) < 1e-7 and abs(r.gamma_primal - 1.3) < 1e-7


def _column_step_pin_holds():
    """The literal single step of Eq. 30 on the two-voxel column (test_oracle_trajectory)."""
    r2 = 0.5 ** 0.5
    e = np.array([[1.0, 0.0], [0.0, 0.0], [0.5, -0.5], [0.0, 1.0], [0.0, 0.0], [0.5, 1.5]]).reshape(6, 1, 1, 2)
    c = 1.5 * r2
    v_lit0 = np.array([0.25, 0.0, c - 0.25, -0.75, 0.0, c - 0.25])   # voxel 0: z unclipped
    half, _, v_new = O.admm_step(e, np.zeros_like(e), 1.0, np.array([100.0, 0.5]).reshape(1, 1, 2),
                                 np.array([0.0, 0.0, 1.0]), 0.25)
    ok_half = np.allclose(half.reshape(6, 2)[:, 0], [0.5, 0.0, r2, -0.5, 0.0, r2], atol=1e-14)
    return ok_half and np.allclose(v_new.reshape(6, 2)[:, 0], v_lit0, atol=1e-14)


def _bb_ratio_pin_holds():
    """de = (1, 0, ..), dv = (1, 1, ..) per voxel: <dv, de> / |de|^2 = 1 (test_oracle_trajectory)."""
    one = np.zeros((6, 2, 1, 2))
    one[0] = 1.0
    dv = one.copy()
    dv[1] = 1.0
    z = np.zeros_like(one)
    return abs(O.next_rho(0.8, O.RHO_BB, z, one, z, dv, O.Params()) - 1.0) < 1e-15


def _ltd_ratio_pin_holds():
    """|v| = 1, |e| = 2 per voxel: |v| / |e| = 0.5 (test_oracle_trajectory)."""
    e = np.zeros((6, 2, 1, 2))
    e[1] = 2.0
    v = np.zeros_like(e)
    v[0], v[5] = 0.6, 0.8
    z = np.zeros_like(e)
    return abs(O.next_rho(0.7, O.RHO_LTD, z, e, z, v, O.Params()) - 0.5) < 1e-15


def _laplacian_pin_holds():
    d = np.random.default_rng(2).standard_normal((5, 6, 7))
    d -= d.mean()
    return np.allclose(O.div_minus(O.grad_plus(O.laplacian_pinv(d))), d, atol=1e-10)


_admm_step = O.admm_step
_next_rho = O.next_rho


def _next_rho_other_bb(rho, rule, e_old, e_new, v_old, v_new, params, primal_res=None):
    """The other Barzilai-Borwein step |dv|^2 / <dv, de> in place of <dv, de> / |de|^2."""
    if rule != O.RHO_BB:
        return _next_rho(rho, rule, e_old, e_new, v_old, v_new, params, primal_res)
    de, dv = e_new - e_old, v_new - v_old
    s_ve, s_ee, s_vv = O.inner(dv, de), O.inner(de, de), O.inner(dv, dv)
    if s_ve > 0.0 and s_ee > 0.0 and s_vv > 0.0 and s_ve / np.sqrt(s_vv * s_ee) > params.bb_corr_min:
        return min(max(s_vv / s_ve, rho / params.rho_step_max), rho * params.rho_step_max)
    return rho


def _next_rho_ltd_inverted(rho, rule, e_old, e_new, v_old, v_new, params, primal_res=None):
    """Lorenz-Tran-Dinh as |e| / |v| instead of |v| / |e|."""
    if rule != O.RHO_LTD:
        return _next_rho(rho, rule, e_old, e_new, v_old, v_new, params, primal_res)
    nv, ne = O.l2_norm(v_new), O.l2_norm(e_new)
    if nv > 0.0 and ne > 0.0:
        return min(max(ne / nv, rho / params.rho_step_max), rho * params.rho_step_max)
    return rho


MUTATIONS = {
    "relaxation_delta_swapped": ("admm_step", lambda e, v, rho, g, xi, delta: _admm_step(e, v, rho, g, xi, 1.0 - delta),
                                 _column_step_pin_holds),
    "relaxation_dropped": ("admm_step", lambda e, v, rho, g, xi, delta: _admm_step(e, v, rho, g, xi, 0.5),
                           _column_step_pin_holds),
    "bb_other_step": ("next_rho", _next_rho_other_bb, _bb_ratio_pin_holds),
    "ltd_inverted": ("next_rho", _next_rho_ltd_inverted, _ltd_ratio_pin_holds),
    "shift_back_wrong_direction": ("shift_back", lambda u: np.stack([np.roll(u[a], -1, axis=a) for a in range(3)]),
                                   _face_pin_holds),
    "A_missing_sqrt_half": ("op_A", lambda u: np.concatenate([u, O.shift_back(u)]), _homogeneous_pin_holds),
    "A_adj_unshifted": ("op_A_adj", lambda w: (w[:3] + w[3:]) * (0.5 ** 0.5), _dense_pin_holds),
    "grad_plus_backward": ("grad_plus", lambda p: np.stack([p - np.roll(p, 1, axis=a) for a in range(3)]),
                           _laplacian_pin_holds),
    "symbol_missing_factor_4": ("laplacian_symbol",
                                lambda shape: sum(-np.sin(np.pi * np.arange(m) / m).reshape(
                                    [-1 if b == a else 1 for b in range(3)]) ** 2 for a, m in enumerate(shape)),
                                _laplacian_pin_holds),
    "projection_C_no_clip": ("project_C", lambda z, g: z, _dense_pin_holds),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, wrong, pin = MUTATIONS[name]
    assert pin(), "pin must hold for the correct oracle"
    monkeypatch.setattr(O, attr, wrong)
    try:
        held = pin()
    except (FloatingPointError, np.linalg.LinAlgError, ValueError, OverflowError):
        held = False
    assert not held, f"planted mistake {name} was not caught"

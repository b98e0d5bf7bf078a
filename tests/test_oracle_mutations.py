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


def _laplacian_pin_holds():
    d = np.random.default_rng(2).standard_normal((5, 6, 7))
    d -= d.mean()
    return np.allclose(O.div_minus(O.grad_plus(O.laplacian_pinv(d))), d, atol=1e-10)


MUTATIONS = {
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

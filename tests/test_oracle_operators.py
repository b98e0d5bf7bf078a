"""Pins of the oracle's operators against identities the paper states and the
face-based form of the CCMF problem (Sec. 2.2, Eq. 6 - Eq. 8), which the dense
module builds without any of the oracle's operators."""

import math

import numpy as np
import pytest

from oracle import ccmf_oracle as O
from oracle import dense_maxflow as D
from paper_2103_05968_gb300 import microstructure as M

SHAPES = [(4, 5, 6), (3, 1, 7), (8, 8, 8)]


def rnd(shape, seed, comps=None):
    rng = np.random.default_rng(seed)
    full = shape if comps is None else (comps,) + tuple(shape)
    return rng.standard_normal(full)


@pytest.mark.parametrize("shape", SHAPES)
def test_shift_inverse_and_adjoint(shape):
    u = rnd(shape, 1, 3)
    w = rnd(shape, 2, 3)
    assert np.array_equal(O.shift_forward(O.shift_back(u)), u)          # S* S = Id (Sec. 3.1)
    assert math.isclose(O.inner(O.shift_back(u), w), O.inner(u, O.shift_forward(w)), rel_tol=1e-13)


@pytest.mark.parametrize("shape", SHAPES)
def test_A_isometry_and_projector(shape):
    u = rnd(shape, 3, 3)
    w = rnd(shape, 4, 6)
    np.testing.assert_allclose(O.op_A_adj(O.op_A(u)), u, atol=1e-14)     # A* A = Id (after Eq. 17)
    assert math.isclose(O.inner(O.op_A(u), w), O.inner(u, O.op_A_adj(w)), rel_tol=1e-12)
    P = lambda x: O.op_A(O.op_A_adj(x))
    np.testing.assert_allclose(P(P(w)), P(w), atol=1e-13)               # A A* projector


@pytest.mark.parametrize("shape", SHAPES)
def test_face_form_matches_compact_form(shape):
    """Eq. 7 (six face flows per voxel) equals 2 |A u|^2 (Eq. 10 / Eq. 15), and the
    mass balance of Eq. 6 equals div^- (Sec. 2.2): catches a wrong shift direction."""
    u = rnd(shape, 5, 3)
    B, G = D.build_problem(shape)
    f = u.reshape(3, -1).reshape(-1)
    face_sq = (G @ (f * f)).reshape(shape)
    au = O.op_A(u)
    np.testing.assert_allclose(face_sq, 2.0 * np.sum(au * au, axis=0), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose((B @ f).reshape(shape), O.div_minus(u), atol=1e-12)


@pytest.mark.parametrize("shape", SHAPES)
def test_grad_div_adjoint(shape):
    phi = rnd(shape, 6)
    u = rnd(shape, 7, 3)
    assert math.isclose(O.inner(O.grad_plus(phi), u), -O.inner(phi, O.div_minus(u)), rel_tol=1e-12)


@pytest.mark.parametrize("shape", SHAPES + [(5, 3, 15), (6, 10, 15)])
def test_laplacian_pinv_against_real_space(shape):
    """The FFT symbol solve inverts div^- grad^+ applied in real space (rolls)."""
    d = rnd(shape, 8)
    d -= d.mean()
    phi = O.laplacian_pinv(d)
    np.testing.assert_allclose(O.div_minus(O.grad_plus(phi)), d, atol=1e-11)
    assert abs(phi.mean()) < 1e-13


@pytest.mark.parametrize("shape", [(4, 5, 6), (6, 10, 15)])
def test_gamma_operator(shape):
    u = rnd(shape, 9, 3)
    w = rnd(shape, 10, 3)
    gu = O.op_Gamma(u)
    np.testing.assert_allclose(O.op_Gamma(gu), gu, atol=1e-12)                       # projector
    assert math.isclose(O.inner(gu, w), O.inner(u, O.op_Gamma(w)), rel_tol=1e-11)     # self-adjoint
    np.testing.assert_allclose(O.div_minus(u - gu), 0.0, atol=1e-11)                 # range: div-free complement
    phi = rnd(shape, 11)
    g = O.grad_plus(phi)
    np.testing.assert_allclose(O.op_Gamma(g), g, atol=1e-11)                         # fixes gradients


@pytest.mark.parametrize("shape", [(4, 5, 6), (6, 10, 15)])
def test_project_K(shape):
    xi_bar = np.array([0.36, -0.48, 0.8])
    w = rnd(shape, 12, 6)
    pk = O.project_K(w, xi_bar)
    # membership in K (Sec. 3.1): A* xi - xi_bar is a gradient, i.e. fixed by Gamma, with zero mean
    r = O.op_A_adj(pk) - O.const_field(xi_bar, shape)
    np.testing.assert_allclose(O.op_Gamma(r), r, atol=1e-11)
    np.testing.assert_allclose(r.reshape(3, -1).mean(axis=1), 0.0, atol=1e-13)
    np.testing.assert_allclose(O.project_K(pk, xi_bar), pk, atol=1e-11)               # idempotent
    # nearest point: <w - P w, xi - P w> = 0 for xi in the affine set K
    psi = rnd(shape, 13)
    extra = rnd(shape, 14, 6)
    xi = O.op_A(O.const_field(xi_bar, shape) + O.grad_plus(psi)) + extra - O.op_A(O.op_A_adj(extra))
    assert abs(O.inner(w - pk, xi - pk)) < 1e-10 * (1 + O.l2_norm(w) * O.l2_norm(xi))
    assert O.l2_norm(w - pk) <= O.l2_norm(w - xi) + 1e-12


def test_project_C():
    shape = (5, 4, 3)
    rng = np.random.default_rng(15)
    gamma = rng.uniform(0.0, 2.0, shape)
    gamma[0, 0, 0] = 0.0
    z = rng.standard_normal((6,) + shape) * 2.0
    p = O.project_C(z, gamma)
    assert np.all(np.sqrt(np.sum(p * p, axis=0)) <= gamma * (1 + 1e-15))
    np.testing.assert_allclose(O.project_C(p, gamma), p, rtol=1e-15, atol=1e-15)
    assert np.all(p[:, 0, 0, 0] == 0.0)
    # nearest point against random points of C_gamma
    for s in range(5):
        q = rng.standard_normal((6,) + shape)
        q *= (gamma * rng.random(shape) / np.sqrt(np.sum(q * q, axis=0)))[None]
        assert np.all(np.sum((z - p) ** 2, axis=0) <= np.sum((z - q) ** 2, axis=0) + 1e-12)


def test_disk_composite_generator():
    """The 2-D stand-in of the Sec. 4.3 composite: 32 disks, no two closer than a diameter
    (periodic distance), voxel filler fraction within 1 % of the requested 50 %."""
    g, c = M.disks_2d(128, 32, 0.5, 10.0, 1.0, seed=599)
    assert g.shape == (128, 128, 1) and len(c) == 32
    r = np.sqrt(0.5 * 128 * 128 / (32 * np.pi))
    d = np.abs(c[:, None, :] - c[None, :, :])
    d = np.minimum(d, 128 - d)
    dist = np.sqrt((d ** 2).sum(-1))[np.triu_indices(32, 1)]
    assert dist.min() >= 2 * r
    assert abs(float((g > 1).mean()) - 0.5) < 0.01


def test_boolean_and_fibre_generators():
    """Generator statistics: the voxel volume fraction is reached and overshot by at most about
    one added body (balls of the Boolean model, fibres of the random sequential addition)."""
    g, nb = M.boolean_spheres((48, 48, 48), 4.0, 0.2, 0.3, 1.0, seed=7)
    frac = float((g < 1.0).mean())
    ball = 4.0 / 3.0 * np.pi * 4.0 ** 3 / 48 ** 3
    assert 0.2 <= frac <= 0.2 + ball
    gf, nf = M.short_fibres((64, 64, 64), 4.0, 8.0, 0.06, 3.0, 1.0, seed=5)
    ff = float((gf > 1.0).mean())
    cyl = np.pi * 2.0 ** 2 * 32.0 / 64 ** 3
    assert nf > 0 and 0.06 <= ff <= 0.06 + 1.5 * cyl


def test_relaxed_and_infinite_contrast_generators():
    """Relaxed balls do not overlap (periodic distances >= sum of radii); the porous cell hits
    its porosity with gamma 0 in the pores; the sand-binder cell has the phase fractions of
    Sec. 4.6 (grains 58.6 %, binder 1.3 %, the rest the third phase)."""
    r = np.full(30, 4.0)
    x = M.relaxed_spheres((32, 32, 32), r, seed=3)
    d = x[:, None, :] - x[None, :, :]
    d -= 32.0 * np.round(d / 32.0)
    dist = np.sqrt(np.sum(d * d, axis=-1)) + np.eye(30) * 1e9
    assert dist.min() >= 8.0 - 2e-3
    g, por = M.porous_spheres((48, 48, 48), 20, 0.4, seed=2)
    assert abs(por - 0.4) < 0.01 and g.min() == 0.0 and g.max() == 1.0
    labels, fr = M.sand_binder((48, 48, 48), 6.0, 0.586, 0.013, seed=6)
    assert abs(fr["grain"] - 0.586) < 0.02 and abs(fr["binder"] - 0.013) < 1e-3
    assert abs(fr["matrix"] + fr["grain"] + fr["binder"] - 1.0) < 1e-12

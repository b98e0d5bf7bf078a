"""Pins of one step of the damped ADMM (Eq. 30) and of the penalty rules that follow it.

Equal-iteration GPU parity rests on the oracle's trajectory, so the trajectory itself is
fixed here by values derived by hand from the paper, not by re-running the oracle:

* a single step of Eq. 30 on a 1 x 1 x 2 column, where the projection onto K_xi_bar
  (Eq. 28) has a closed form, checked against literal numbers for xi^{k+1/2}, the relaxed
  xi^{k+1}, the pre-projection point z = v + rho xi^{k+1}, e^{k+1} and v^{k+1};
* the same closed form on random columns (any length, any rho, delta, normal);
* delta = 1/2 turning Eq. 30 into the undamped scheme printed just before it;
* the Barzilai-Borwein and Lorenz-Tran-Dinh ratios (text after Eq. 30) and the safeguard
  of reading R3 on small hand-made fields with literal expected values.

On a column (N1 = N2 = 1) the x and y shifts are the identity, so for w = e - v/rho and
u = A* w (Eq. 17): u_x = (w1x + w2x)/sqrt2, u_y likewise, u_z[k] = (w1z[k] + w2z[k+1])/sqrt2,
and div^- u = u_z[k] - u_z[k-1]. The forward gradients of periodic sequences are exactly the
sequences with zero mean, so the potential of Eq. 28 satisfies grad^+ phi = u_z - mean(u_z).
Hence y = u - grad^+ phi - xi_bar = (u_x - xi_x, u_y - xi_y, mean(u_z) - xi_z), constant along
z in its last component, and xi^{k+1/2} = w - A y with A y = (y, y)/sqrt2.
"""

import math

import numpy as np

from oracle import ccmf_oracle as O

R2 = 1.0 / math.sqrt(2.0)


def column_step_by_hand(e, v, rho, gamma, xi_bar, delta):
    """Eq. 30 on a 1 x 1 x n column, written out with the column closed form of P_K."""
    w = e - v / rho
    u_x = (w[0] + w[3]) * R2
    u_y = (w[1] + w[4]) * R2
    u_z = (w[2] + np.roll(w[5], -1)) * R2            # w2z at k + 1
    y = [u_x - xi_bar[0], u_y - xi_bar[1], np.full_like(u_z, u_z.mean() - xi_bar[2])]
    xi_half = np.stack([w[c] - y[c % 3] * R2 for c in range(6)])
    xi = 2.0 * (1.0 - delta) * xi_half - (1.0 - 2.0 * delta) * e
    z = v + rho * xi
    nz = np.sqrt(np.sum(z * z, axis=0))
    scale = np.where(nz > gamma, gamma / np.where(nz > 0, nz, 1.0), 1.0)
    v_new = z * scale
    e_new = (z - v_new) / rho
    return xi_half, xi, z, e_new, v_new


def _as_grid(a):
    """(6, n) column arrays -> the oracle's (6, 1, 1, n) layout."""
    return np.asarray(a, dtype=np.float64).reshape(a.shape[0], 1, 1, -1)


def test_single_step_on_a_two_voxel_column_literal_values():
    """e^k = w given, v^k = 0, rho = 1, delta = 1/4, xi_bar = e_z, gamma = (100, 0.5).

    By hand (components ordered w1x, w1y, w1z, w2x, w2y, w2z; voxels k = 0, 1):
      mean(u_z) = (mean w1z + mean w2z)/sqrt2 = (0 + 1)/sqrt2, so y_z = 1/sqrt2 - 1 and
      xi^{k+1/2}_{1z} = w1z - y_z/sqrt2 = w1z - 1/2 + 1/sqrt2, likewise for w2z;
      xi^{k+1/2}_{1x} = (w1x - w2x)/2, xi^{k+1/2}_{2x} = (w2x - w1x)/2 (xi_x = 0);
      xi^{k+1} = 3/2 xi^{k+1/2} - 1/2 e^k; z = xi^{k+1}; voxel 0 is not clipped (|z| < 100),
      voxel 1 is clipped to radius 0.5.
    """
    e = np.array([[1.0, 0.0], [0.0, 0.0], [0.5, -0.5], [0.0, 1.0], [0.0, 0.0], [0.5, 1.5]])
    v = np.zeros_like(e)
    gamma = np.array([100.0, 0.5])
    xi_bar = np.array([0.0, 0.0, 1.0])
    xi_half_lit = np.array([[0.5, -0.5], [0.0, 0.0], [R2, -1.0 + R2],
                            [-0.5, 0.5], [0.0, 0.0], [R2, 1.0 + R2]])
    c = 1.5 * R2
    xi_lit = np.array([[0.25, -0.75], [0.0, 0.0], [c - 0.25, c - 1.25],
                       [-0.75, 0.25], [0.0, 0.0], [c - 0.25, c + 0.75]])
    z1 = xi_lit[:, 1]
    n1 = math.sqrt(0.75 ** 2 + 0.25 ** 2 + (c - 1.25) ** 2 + (c + 0.75) ** 2)
    assert abs(n1 - 1.98478) < 1e-5                     # |z| at voxel 1 > gamma = 0.5
    v_new_lit = np.stack([xi_lit[:, 0], z1 * (0.5 / n1)], axis=1)
    e_new_lit = np.stack([np.zeros(6), z1 * (1.0 - 0.5 / n1)], axis=1)

    # the closed form reproduces the literal values ...
    xh, xi, z, en, vn = column_step_by_hand(e, v, 1.0, gamma, xi_bar, 0.25)
    np.testing.assert_allclose(xh, xi_half_lit, atol=1e-15)
    np.testing.assert_allclose(xi, xi_lit, atol=1e-15)
    np.testing.assert_allclose(z, xi_lit, atol=1e-15)
    # ... and so does the oracle's step
    o_half, o_e, o_v = O.admm_step(_as_grid(e), _as_grid(v), 1.0, gamma.reshape(1, 1, 2), xi_bar, 0.25)
    np.testing.assert_allclose(o_half.reshape(6, 2), xi_half_lit, atol=1e-14)
    np.testing.assert_allclose(o_e.reshape(6, 2), e_new_lit, atol=1e-14)
    np.testing.assert_allclose(o_v.reshape(6, 2), v_new_lit, atol=1e-14)
    # xi^{k+1/2} lies in K_xi_bar: A* xi - xi_bar = (0, 0, (1/sqrt2, -1/sqrt2)), a mean-free z part
    az = (o_half.reshape(6, 2)[2] + np.roll(o_half.reshape(6, 2)[5], -1)) * R2
    np.testing.assert_allclose(az - 1.0, [R2, -R2], atol=1e-15)


def test_single_step_random_columns():
    """The column closed form against the oracle for random states, rho, delta and normals,
    with a mix of clipped and unclipped voxels."""
    rng = np.random.default_rng(30)
    for n in (1, 2, 3, 7, 16):
        for _ in range(4):
            e = rng.standard_normal((6, n))
            v = rng.standard_normal((6, n))
            gamma = rng.uniform(0.2, 3.0, n)
            xi_bar = rng.standard_normal(3)
            xi_bar /= np.linalg.norm(xi_bar)
            rho = float(rng.uniform(0.1, 5.0))
            delta = float(rng.uniform(0.05, 0.95))
            xh, _, _, en, vn = column_step_by_hand(e, v, rho, gamma, xi_bar, delta)
            o_half, o_e, o_v = O.admm_step(_as_grid(e), _as_grid(v), rho, gamma.reshape(1, 1, n), xi_bar, delta)
            np.testing.assert_allclose(o_half.reshape(6, n), xh, atol=1e-12)
            np.testing.assert_allclose(o_e.reshape(6, n), en, atol=1e-12)
            np.testing.assert_allclose(o_v.reshape(6, n), vn, atol=1e-12)


def test_delta_half_is_the_undamped_scheme():
    """delta = 1/2 gives xi^{k+1} = xi^{k+1/2}: the scheme printed before Eq. 30,
    xi^{k+1} = A xi_bar - (1/rho) M (v^k - rho e^k), e^{k+1} = [z - P_C(z)]/rho with
    z = v^k + rho xi^{k+1}, v^{k+1} = v^k + rho (xi^{k+1} - e^{k+1})."""
    rng = np.random.default_rng(31)
    shape = (4, 5, 3)
    gamma = rng.uniform(0.3, 1.5, shape)
    xi_bar = np.array([0.48, 0.6, 0.64])
    e = rng.standard_normal((6,) + shape) * 0.5
    v = rng.standard_normal((6,) + shape) * 0.5
    rho = 0.7
    xi = O.op_A(O.const_field(xi_bar, shape)) - O.op_M(v - rho * e) / rho
    z = v + rho * xi
    e_plain = (z - O.project_C(z, gamma)) / rho
    v_plain = v + rho * (xi - e_plain)
    xh, en, vn = O.admm_step(e, v, rho, gamma, xi_bar, 0.5)
    np.testing.assert_allclose(xh, xi, atol=1e-13)
    np.testing.assert_allclose(en, e_plain, atol=1e-13)
    np.testing.assert_allclose(vn, v_plain, atol=1e-13)


def _fields(a, b, shape=(2, 1, 2)):
    """A 6-component field whose voxels alternate between the 6-vectors a and b."""
    f = np.empty((6,) + shape)
    flat = f.reshape(6, -1)
    for p in range(flat.shape[1]):
        flat[:, p] = a if p % 2 == 0 else b
    return f


def test_barzilai_borwein_ratio_literal():
    """BB (text after Eq. 30): rho = <dv, de> / |de|^2 with the R3 safeguard.

    Per voxel de = (1, 0, 0, 0, 0, 0) and dv = (1, 1, 0, 0, 0, 0): <dv, de> = 1, |de|^2 = 1,
    |dv|^2 = 2, correlation 1/sqrt2 > 0.2, so rho_BB = 1. (The other Barzilai-Borwein step,
    |dv|^2 / <dv, de> = 2, differs.)"""
    p = O.Params(bb_corr_min=0.2, rho_step_max=2.0)
    e0 = _fields([0.25, 0.125, 0, 0, 0, 0.375], [0.25, 0.125, 0, 0, 0, 0.375])
    e1 = e0 + _fields([1, 0, 0, 0, 0, 0], [1, 0, 0, 0, 0, 0])
    v0 = _fields([0.0, 0.5, 0.125, 0, 0, 0], [0.0, 0.5, 0.125, 0, 0, 0])
    v1 = v0 + _fields([1, 1, 0, 0, 0, 0], [1, 1, 0, 0, 0, 0])
    assert abs(O.next_rho(0.8, O.RHO_BB, e0, e1, v0, v1, p) - 1.0) < 1e-15
    assert abs(O.next_rho(0.3, O.RHO_BB, e0, e1, v0, v1, p) - 0.6) < 1e-15      # clamped to 2 x 0.3
    assert abs(O.next_rho(3.0, O.RHO_BB, e0, e1, v0, v1, p) - 1.5) < 1e-15      # clamped to 3 / 2
    # mixed voxels: de = (2,0,..) | (0,1,..), dv = (1,0,..) | (0,3,..):
    # <dv,de> = (2 + 3)/2, |de|^2 = (4 + 1)/2 -> rho_BB = 1; |dv|^2 = (1 + 9)/2, corr = 5/sqrt(50)
    e2 = e0 + _fields([2, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0])
    v2 = v0 + _fields([1, 0, 0, 0, 0, 0], [0, 3, 0, 0, 0, 0])
    assert abs(O.next_rho(0.9, O.RHO_BB, e0, e2, v0, v2, p) - 1.0) < 1e-15
    # safeguard: correlation below the threshold, or <dv, de> <= 0, keeps rho
    v3 = v0 + _fields([0.1, 5, 0, 0, 0, 0], [0.1, 5, 0, 0, 0, 0])    # corr = 0.1 / sqrt(25.01) < 0.2
    assert abs(O.next_rho(0.8, O.RHO_BB, e0, e1, v0, v3, p) - 0.8) < 1e-15
    v4 = v0 + _fields([-1, 0, 0, 0, 0, 0], [-1, 0, 0, 0, 0, 0])
    assert abs(O.next_rho(0.8, O.RHO_BB, e0, e1, v0, v4, p) - 0.8) < 1e-15
    assert abs(O.next_rho(0.8, O.RHO_BB, e0, e0, v0, v1, p) - 0.8) < 1e-15       # de = 0


def test_lorenz_tran_dinh_ratio_literal():
    """LTD (text after Eq. 30): rho = |v| / |e| of the new iterate, with the R3 clamp.

    v = (0.6, 0, 0, 0, 0, 0.8) per voxel (|v| = 1), e = (0, 2, 0, 0, 0, 0) (|e| = 2): rho = 0.5."""
    p = O.Params(rho_step_max=2.0)
    e = _fields([0, 2, 0, 0, 0, 0], [0, 2, 0, 0, 0, 0])
    v = _fields([0.6, 0, 0, 0, 0, 0.8], [0.6, 0, 0, 0, 0, 0.8])
    z = np.zeros_like(e)
    assert abs(O.next_rho(0.7, O.RHO_LTD, z, e, z, v, p) - 0.5) < 1e-15
    assert abs(O.next_rho(0.2, O.RHO_LTD, z, e, z, v, p) - 0.4) < 1e-15          # clamped to 2 x 0.2
    assert abs(O.next_rho(1.6, O.RHO_LTD, z, e, z, v, p) - 0.8) < 1e-15          # clamped to 1.6 / 2
    # |v| and |e| are L2 norms over voxels: voxels with |v| = 1, 3 and |e| = 2, 2 give sqrt(5)/2
    v2 = _fields([1, 0, 0, 0, 0, 0], [0, 0, 3, 0, 0, 0])
    assert abs(O.next_rho(1.0, O.RHO_LTD, z, e, z, v2, p) - math.sqrt(5.0) / 2.0) < 1e-15
    assert abs(O.next_rho(0.7, O.RHO_LTD, z, z, z, v, p) - 0.7) < 1e-15          # |e| = 0 keeps rho


def test_constant_rule_keeps_rho():
    p = O.Params()
    e = _fields([1, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0])
    assert abs(O.next_rho(0.37, O.RHO_CONST, e, 2 * e, e, 3 * e, p) - 0.37) < 1e-15

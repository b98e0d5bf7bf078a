"""FP64 CPU oracle of the gradient of the effective crack energy with respect to
the local crack resistances, through K unrolled damped-ADMM iterations.

TEST INFRASTRUCTURE ONLY (see ccmf_oracle.py); it shares no code with the CUDA path.

Function differentiated (reading R8 of the design notes): J(gamma) is the
reported effective crack energy after K updates of Eq. 30, i.e. the max-flow
value <xi_bar, A* v^K> (Eq. 12, reading R5), with the penalty sequence
rho^0 ... rho^{K-1} held fixed (recorded from a run with the adaptive rule and
replayed). Each update is then a fixed map of (e, v) that depends on gamma only
through the node-wise projection onto C_gamma (Eq. 19):

  w = e - v / rho,  xi_h = A xi_bar + M w,  xi = a xi_h - b e,  z = v + rho xi,
  v' = P_C(z),  e' = (z - v') / rho,           a = 2(1 - delta), b = 1 - 2 delta,

with M = Id - A A* + A Gamma A* (Eq. 28). Reverse mode (adjoints written with a
bar): with u = vbar' - ebar' / rho,

  zbar = ebar' / rho + J_C(z) u,  gammabar += [|z| > gamma] (z / |z|) . u,
  wbar = M (a rho zbar)   (M is self-adjoint: A A* and Gamma are orthogonal projectors),
  ebar = wbar - b rho zbar,  vbar = zbar - wbar / rho,

where J_C(z) = Id on |z| <= gamma and (gamma / |z|)(Id - zz^T/|z|^2) otherwise.
The seed is vbar^K = A xi_bar / N (the gradient of <xi_bar, A* v> in v, with the
1/N of Eq. 11), ebar^K = 0. e^0 and v^0 do not depend on gamma (reading R1).

At convergence dJ/dgamma(x) tends to |xi*(x)| / N, the envelope (Danskin)
derivative of the min-cut value of Eq. 21 (gradient check of the tests).
"""

from __future__ import annotations

import numpy as np

from . import ccmf_oracle as O


def forward_replay(gamma, xi_bar, rho_seq, delta=0.25, keep=True):
    """K = len(rho_seq) updates of Eq. 30 with the given penalties; returns
    (J, e^K, v^K, list of z^k) where J = <xi_bar, A* v^K>."""
    gamma = np.asarray(gamma, dtype=np.float64)
    xi_bar = np.asarray(xi_bar, dtype=np.float64)
    xi_bar = xi_bar / np.linalg.norm(xi_bar)
    shape = gamma.shape
    e = O.op_A(O.const_field(xi_bar, shape))
    v = np.zeros((6,) + shape)
    a, b = 2.0 * (1.0 - delta), 1.0 - 2.0 * delta
    zs = []
    for rho in rho_seq:
        xi_h = O.op_A(O.const_field(xi_bar, shape)) + O.op_M(e - v / rho)
        z = v + rho * (a * xi_h - b * e)
        v_new = O.project_C(z, gamma)
        e = (z - v_new) / rho
        v = v_new
        if keep:
            zs.append(z)
    J = O.flow_objective(O.op_A_adj(v), xi_bar)
    return J, e, v, zs


def gradient(gamma, xi_bar, rho_seq, delta=0.25):
    """dJ/dgamma (shape of gamma) by reverse mode through the replayed updates."""
    gamma = np.asarray(gamma, dtype=np.float64)
    xi_bar = np.asarray(xi_bar, dtype=np.float64)
    xi_bar = xi_bar / np.linalg.norm(xi_bar)
    J, _, _, zs = forward_replay(gamma, xi_bar, rho_seq, delta)
    shape = gamma.shape
    N = gamma.size
    a, b = 2.0 * (1.0 - delta), 1.0 - 2.0 * delta
    vbar = O.op_A(O.const_field(xi_bar, shape)) / N
    ebar = np.zeros_like(vbar)
    gbar = np.zeros(shape)
    for k in range(len(rho_seq) - 1, -1, -1):
        rho = rho_seq[k]
        z = zs[k]
        u = vbar - ebar / rho
        nz = np.sqrt(np.sum(z * z, axis=0))
        clip = nz > gamma
        zbar = ebar / rho + u
        zhat = np.zeros_like(z)
        zhat[:, clip] = z[:, clip] / nz[clip]
        zu = np.sum(zhat * u, axis=0)
        # J_C u on clipped voxels: (gamma/|z|)(u - zhat (zhat . u))
        scale = np.zeros_like(nz)
        scale[clip] = gamma[clip] / nz[clip]
        jc = scale[None] * (u - zhat * zu[None])
        zbar[:, clip] = ebar[:, clip] / rho + jc[:, clip]
        gbar += np.where(clip, zu, 0.0)
        wbar = O.op_M(a * rho * zbar)
        ebar = wbar - b * rho * zbar
        vbar = zbar - wbar / rho
    return J, gbar


def record_rho(gamma, xi_bar, K, params=None):
    """The penalty sequence rho^0 .. rho^{K-1} of an adaptive run of K updates."""
    params = params or O.Params()
    p = O.Params(**{**params.__dict__, "fixed_iters": K})
    r = O.solve(gamma, xi_bar, p)
    return [h[1] for h in r.history]

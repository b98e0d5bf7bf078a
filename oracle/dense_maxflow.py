"""Dense log-barrier solver of the CCMF maximum-flow problem on tiny grids.

TEST INFRASTRUCTURE ONLY (see ccmf_oracle.py). It pins the ADMM oracle to the
plain definition of the discrete problem without using any of the oracle's
operators: it is built straight from the face-based form of Sec. 2.2 of the
paper, i.e. the mass balance on voxel faces (Eq. 6), the per-voxel bound on
the six face flows (Eq. 7) and the mean flux objective (Eq. 8).

Unknowns: one flow value per face. Face (i + 1/2, j, k) is numbered
0 * N + lin(i, j, k), face (i, j + 1/2, k) is N + lin(i, j, k) and face
(i, j, k + 1/2) is 2 N + lin(i, j, k), with lin the C-order voxel index and
periodic wrap-around.

Method: the equality constraints are eliminated through a null-space basis
(dense SVD); the inequality constraints 2 gamma^2 - sum(face flows^2) > 0 get a
logarithmic barrier; Newton's method with backtracking follows the central path
with t multiplied by 10 per stage until the barrier gap m / t is below the
requested tolerance. The returned value is the objective of a strictly
feasible flow, a lower bound on the optimum that is within m / t of it.
Requires gamma > 0 everywhere (Slater point f = 0, Sec. 2.1).
"""

from __future__ import annotations

import numpy as np


def _lin(n, i, j, k):
    return ((i % n[0]) * n[1] + (j % n[1])) * n[2] + (k % n[2])


def build_problem(n):
    """Incidence data of Eq. 6 and Eq. 7 for a periodic grid of shape n."""
    N = n[0] * n[1] * n[2]
    B = np.zeros((N, 3 * N))          # mass balance rows (Eq. 6)
    G = np.zeros((N, 3 * N))          # faces touching each voxel, with multiplicity (Eq. 7)
    for i in range(n[0]):
        for j in range(n[1]):
            for k in range(n[2]):
                p = _lin(n, i, j, k)
                out_faces = [0 * N + p, 1 * N + p, 2 * N + p]
                in_faces = [0 * N + _lin(n, i - 1, j, k),
                            1 * N + _lin(n, i, j - 1, k),
                            2 * N + _lin(n, i, j, k - 1)]
                for f in out_faces:
                    B[p, f] += 1.0
                    G[p, f] += 1.0
                for f in in_faces:
                    B[p, f] -= 1.0
                    G[p, f] += 1.0
    return B, G


def max_flow(gamma, xi_bar, gap_tol=1e-11, max_newton=200):
    """Maximise (1/N) sum xi_bar . (face flows) s.t. Eq. 6 and Eq. 7.

    Returns (value, face_flows, gap_bound).
    """
    gamma = np.asarray(gamma, dtype=np.float64)
    n = gamma.shape
    N = gamma.size
    if np.min(gamma) <= 0.0:
        raise ValueError("the barrier solver needs gamma > 0")
    xi_bar = np.asarray(xi_bar, dtype=np.float64)
    xi_bar = xi_bar / np.linalg.norm(xi_bar)
    B, G = build_problem(n)
    c = np.concatenate([np.full(N, xi_bar[0]), np.full(N, xi_bar[1]), np.full(N, xi_bar[2])]) / N
    # null space of the mass balance
    _, s, vt = np.linalg.svd(B)
    rank = int(np.sum(s > 1e-10 * s[0]))
    Z = vt[rank:].T                    # (3N, 3N - rank)
    cz = Z.T @ c
    g2 = 2.0 * gamma.reshape(-1) ** 2  # right-hand side of Eq. 7

    def slack(y):
        f = Z @ y
        return g2 - G @ (f * f), f

    y = np.zeros(Z.shape[1])
    m = float(N)
    t = 1.0
    while True:
        for _ in range(max_newton):
            q, f = slack(y)
            # F(y) = -t c.f - sum log q
            grad_f = -t * c + 2.0 * (G.T @ (1.0 / q)) * f
            gy = Z.T @ grad_f
            J = G * f[None, :]                                  # rows: (G_p o f)
            H = np.diag(2.0 * (G.T @ (1.0 / q))) + J.T @ ((4.0 / q ** 2)[:, None] * J)
            Hy = Z.T @ H @ Z
            dy = -np.linalg.solve(Hy, gy)
            dec = float(-gy @ dy)
            if dec / 2.0 <= 1e-12:
                break
            step = 1.0
            F0 = -t * (c @ f) - np.sum(np.log(q))
            while True:
                qn, fn = slack(y + step * dy)
                if np.all(qn > 0.0):
                    Fn = -t * (c @ fn) - np.sum(np.log(qn))
                    if Fn <= F0 - 0.25 * step * dec:
                        break
                step *= 0.5
                if step < 1e-14:
                    break
            y = y + step * dy
        if m / t < gap_tol:
            break
        t *= 10.0
    _, f = slack(y)
    return float(c @ f), f, m / t

"""Plain FP64 CPU oracle of the CCMF discretisation and its FFT-based ADMM solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product (the C-ABI library and its
Python binding) imports, links or calls this module; only the tests, the smoke
check and the CPU-baseline leg of the benchmark do. It shares no code with the
CUDA path.

What it follows, from Ernesti & Schneider, "An FFT-based method for computing the
effective crack energy of a heterogeneous material on a combinatorially
consistent grid" (arXiv:2103.05968), equations numbered as in the paper:

* Sec. 2.2: staggered flow stored at voxel centres, the backward divergence
  div^- (text after Eq. 8), the backward shift S (Eq. 9), the compact bound
  (Eq. 10) and the normalised inner product (Eq. 11).
* Sec. 3.1: the forward shift S* (Eq. 14), the doubling operator A (Eq. 15) and
  its adjoint A* (Eq. 17), the set C_gamma (Eq. 19), the forward gradient
  grad^+ in the set K_xi (text before Eq. 21) and the min-cut objective (Eq. 21).
* Sec. 3.2: the projection onto K (Eq. 28, Gamma = grad^+ (div^- grad^+)^+ div^-),
  the radial projection onto C_gamma (text after Eq. 28), the damped ADMM
  (Eq. 30), the Lorenz-Tran-Dinh and Barzilai-Borwein penalties (text after
  Eq. 30) and the convergence criterion (Eq. 31, Sec. 4.1).

Every array is float64. Scalar fields have shape (N1, N2, N3) indexed
[i, j, k] = (x, y, z); 3-vector fields have shape (3, N1, N2, N3) with
component a along axis a; 6-vector fields stack the two halves (w1, w2) as
(6, N1, N2, N3).

Readings where the paper is silent (each one is listed in the design notes):
  R1 initial values: e^0 = A xi_bar, v^0 = 0.
  R2 rho^0: the given value, else min(gamma) if positive, else mean(gamma).
  R3 the Barzilai-Borwein safeguard (delegated by the paper to another work):
     accept rho_BB = <dv,de>/|de|^2 only if <dv,de> > 0, |de| > 0, |dv| > 0 and
     <dv,de>/(|dv||de|) > bb_corr_min; clamp it to [rho/s, rho*s] with
     s = rho_step_max; otherwise keep rho. The Lorenz-Tran-Dinh ratio gets the
     same clamp and keeps rho when either norm vanishes.
  R4 the criterion of Eq. 31 at iteration k uses xi^{k+1/2}, e^k and v^k; it is
     evaluated from k = 1 on (at k = 0 both sides vanish) and, when it holds,
     the solver stops after the update to k + 1 that the same pass performs.
  R5 outputs come from one further projection of the final state (e^K, v^K):
     cut = xi^{K+1/2} = P_K(e^K - v^K / rho^K), min-cut estimate
     mean(gamma |cut|) (Eq. 21), flow = A* v^K and max-flow estimate
     <xi_bar, A* v^K> (Eq. 12). The reported effective crack energy is the
     max-flow estimate: Sec. 2.2 defines the CCMF discretisation as the maximum
     flow problem of Eq. 8 / Eq. 12, and this estimate is linear in v, so
     rounding noise in the fields averages out instead of adding |noise| to a
     norm. Both estimates converge to the same value (strong duality, Sec. 2.1).
  R6 P_C keeps w when |w| <= gamma (the strict '>' branch); gamma = 0 maps to 0.
  R7 the zero frequency of (div^- grad^+)^+ is set to zero (pseudo-inverse).
  R10 residual balancing (compared in Sec. 4.3 and its appendix, defined only by
     reference to He et al.): primal residual r = |e^k - xi^{k+1/2}| (Eq. 31),
     dual residual s = rho^k |e^{k+1} - e^k|; rho * s_max if r > 10 s, rho / s_max
     if s > 10 r, else rho (s_max = rho_step_max).

Pins: what fixes each function independently of itself (tests/), and the planted
mistake (tests/test_oracle_mutations.py) that the pin catches.
  shift_back, shift_forward  S*S = Id, <Su, w> = <u, S*w>; face form of Eq. 6/7 equals
                             Eq. 10 (test_oracle_operators) -- wrong shift direction
  op_A, op_A_adj             A*A = Id, AA* a projector (test_oracle_operators); homogeneous
                             gamma_eff = gamma for oblique normals -- missing 1/sqrt2; dense
                             barrier max-flow (test_oracle_solver) -- unshifted A*
  div_minus, grad_plus       <grad^+ phi, u> = -<phi, div^- u>; face-form divergence B f
                             (test_oracle_operators) -- backward gradient
  laplacian_symbol, _pinv    real-space Laplacian by rolls on odd and radix-3/5 grids
                             (test_oracle_operators) -- symbol without its factor 4
  op_Gamma, op_M, project_K  Gamma a self-adjoint projector fixing gradients; P_K(w) in K,
                             idempotent, the nearest point (test_oracle_operators); the
                             column closed form of P_K (test_oracle_trajectory)
  project_C                  feasible, idempotent, nearest point (test_oracle_operators);
                             dense barrier agreement -- no clip
  admm_step                  one step of Eq. 30 on a 1 x 1 x 2 column against literal
                             values, random columns against the column closed form, and
                             delta = 1/2 against the undamped scheme (test_oracle_trajectory)
                             -- delta swapped with 1 - delta, relaxation dropped
  next_rho                   BB and LTD ratios, the R3 safeguard and clamp on hand-made
                             fields with literal values; residual-balancing direction
                             (test_oracle_trajectory, test_oracle_solver) -- the other BB
                             step |dv|^2/<dv,de>, LTD inverted
  solve, evaluate            homogeneous, laminate, axis-normal bounds, config-1 exact value
                             0.8171875, the paper's Sec. 4.2 result, dense barrier
                             max-flow on 2x3x5 ... 8^3 grids, strong duality, equivariances
                             (test_oracle_solver)
  mincut_objective,          both estimates bracket and converge to the dense barrier value
  flow_objective             and the closed forms (test_oracle_solver)
  initial_rho                R2 is a reading; gamma -> 2 gamma equivariance with rho^0
                             proportional to gamma (test_oracle_solver)
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

RHO_BB = 0
RHO_CONST = 1
RHO_LTD = 2
RHO_RB = 3
RB_MU = 10.0   # residual balancing: ratio of the residuals that triggers a change (R10)

_SQRT_HALF = 1.0 / math.sqrt(2.0)


# ---------------------------------------------------------------------------
# Operators of Sec. 2.2 and Sec. 3.1
# ---------------------------------------------------------------------------

def shift_back(u):
    """S of Eq. 9: (S u)_a[p] = u_a[p - e_a], periodic."""
    return np.stack([np.roll(u[a], 1, axis=a) for a in range(3)])


def shift_forward(u):
    """S* of Eq. 14: (S* u)_a[p] = u_a[p + e_a], periodic."""
    return np.stack([np.roll(u[a], -1, axis=a) for a in range(3)])


def op_A(u):
    """A of Eq. 15: A u = (u, S u) / sqrt(2), a 6-component field."""
    return np.concatenate([u, shift_back(u)]) * _SQRT_HALF


def op_A_adj(w):
    """A* of Eq. 17: A*(w1, w2) = (w1 + S* w2) / sqrt(2)."""
    return (w[:3] + shift_forward(w[3:])) * _SQRT_HALF


def div_minus(u):
    """Backward divergence of Sec. 2.2: sum_a u_a[p] - u_a[p - e_a]."""
    return sum(u[a] - np.roll(u[a], 1, axis=a) for a in range(3))


def grad_plus(phi):
    """Forward gradient of Sec. 3.1: (grad^+ phi)_a[p] = phi[p + e_a] - phi[p]."""
    return np.stack([np.roll(phi, -1, axis=a) - phi for a in range(3)])


def inner(x, y):
    """Normalised inner product of Eq. 11 (mean over voxels of the pointwise dot)."""
    return float(np.sum(x * y) / x[0].size) if x.ndim == 4 else float(np.mean(x * y))


def l2_norm(x):
    return math.sqrt(inner(x, x))


def laplacian_symbol(shape):
    """Fourier symbol of div^- grad^+ on the periodic grid: -sum_a 4 sin^2(pi k_a / N_a)."""
    lam = np.zeros(shape)
    for a, m in enumerate(shape):
        k = np.arange(m, dtype=np.float64)
        s = 4.0 * np.sin(np.pi * k / m) ** 2
        sh = [1, 1, 1]
        sh[a] = -1
        lam = lam - s.reshape(sh)
    return lam


def laplacian_pinv(d):
    """(div^- grad^+)^+ d via the FFT (Sec. 3.2, Gamma of Eq. 28); zero frequency -> 0 (R7)."""
    lam = laplacian_symbol(d.shape)
    dh = np.fft.fftn(d)
    ph = np.zeros_like(dh)
    nz = lam != 0.0
    ph[nz] = dh[nz] / lam[nz]
    return np.fft.ifftn(ph).real


def op_Gamma(u):
    """Gamma = grad^+ (div^- grad^+)^+ div^- of Eq. 28, acting on 3-vector fields."""
    return grad_plus(laplacian_pinv(div_minus(u)))


def op_M(w):
    """M = Id - A A* + A Gamma A* of Eq. 28 / Eq. 30, acting on 6-vector fields."""
    aw = op_A_adj(w)
    return w - op_A(aw) + op_A(op_Gamma(aw))


def const_field(xi_bar, shape):
    return np.broadcast_to(np.asarray(xi_bar, dtype=np.float64).reshape(3, 1, 1, 1),
                           (3,) + tuple(shape)).copy()


def project_K(w, xi_bar):
    """P_K of Eq. 28: A xi_bar + (Id - A A* + A Gamma A*) w."""
    return op_A(const_field(xi_bar, w.shape[1:])) + op_M(w)


def project_C(z, gamma):
    """Radial projection onto C_gamma (Eq. 19), node-wise in R^6 (text after Eq. 28), R6."""
    nz = np.sqrt(np.sum(z * z, axis=0))
    out = z.copy()
    over = nz > gamma
    scale = np.zeros_like(nz)
    scale[over] = gamma[over] / nz[over]
    out[:, over] = z[:, over] * scale[over]
    return out


def mincut_objective(xi, gamma):
    """Objective of Eq. 21: mean over voxels of gamma |xi| (|.| the 6-vector norm)."""
    return float(np.mean(gamma * np.sqrt(np.sum(xi * xi, axis=0))))


def flow_objective(u, xi_bar):
    """Objective of Eq. 12: <xi_bar, u>."""
    return float(sum(xi_bar[a] * np.mean(u[a]) for a in range(3)))


# ---------------------------------------------------------------------------
# Damped ADMM with adaptive penalty (Eq. 30, Eq. 31)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    tol: float = 1e-4            # Eq. 31 tolerance (Sec. 4.1 default)
    max_iter: int = 20000
    delta: float = 0.25          # damping of Eq. 30 (Sec. 4.1 default)
    rho_rule: int = RHO_BB       # Sec. 4.1 default
    rho0: float = 0.0            # <= 0: automatic (R2)
    bb_corr_min: float = 0.2     # R3
    rho_step_max: float = 2.0    # R3
    fixed_iters: int = 0         # > 0: run exactly this many updates, no test


@dataclasses.dataclass
class Result:
    gamma_eff: float             # = gamma_dual, the max-flow objective (R5)
    gamma_primal: float
    gamma_dual: float
    residual: float              # |e^K - xi^{K+1/2}|_{L2} of the final evaluation
    mean_v_norm: float           # |<v^K>|
    rho: float
    iters: int
    converged: bool
    e: np.ndarray
    v: np.ndarray
    cut: np.ndarray
    flow: np.ndarray
    history: list


def initial_rho(gamma, params):
    if params.rho0 > 0.0:
        return float(params.rho0)
    gmin = float(np.min(gamma))
    return gmin if gmin > 0.0 else float(np.mean(gamma))


def next_rho(rho, rule, e_old, e_new, v_old, v_new, params, primal_res=None):
    """Penalty update after Eq. 30 (BB or LTD scaling), with the safeguard of R3; or residual
    balancing (R10, the rule the paper compares in Sec. 4.3 and its appendix): primal residual
    r = |e^k - xi^{k+1/2}| (Eq. 31), dual residual s = rho |e^{k+1} - e^k|; rho * tau if
    r > mu s, rho / tau if s > mu r (mu = 10, tau = rho_step_max)."""
    if rule == RHO_CONST:
        return rho
    lo, hi = rho / params.rho_step_max, rho * params.rho_step_max
    if rule == RHO_BB:
        de = e_new - e_old
        dv = v_new - v_old
        s_ve = inner(dv, de)
        s_ee = inner(de, de)
        s_vv = inner(dv, dv)
        if s_ve > 0.0 and s_ee > 0.0 and s_vv > 0.0 and s_ve / math.sqrt(s_vv * s_ee) > params.bb_corr_min:
            return min(max(s_ve / s_ee, lo), hi)
        return rho
    if rule == RHO_LTD:
        nv = l2_norm(v_new)
        ne = l2_norm(e_new)
        if nv > 0.0 and ne > 0.0:
            return min(max(nv / ne, lo), hi)
        return rho
    if rule == RHO_RB:
        r = float(primal_res)
        s = rho * l2_norm(e_new - e_old)
        if r > RB_MU * s:
            return hi
        if s > RB_MU * r:
            return lo
        return rho
    raise ValueError("unknown rho rule")


def admm_step(e, v, rho, gamma, xi_bar, delta):
    """One pass of Eq. 30 from (e^k, v^k, rho^k); returns (xi^{k+1/2}, e^{k+1}, v^{k+1})."""
    shape = gamma.shape
    xi_half = op_A(const_field(xi_bar, shape)) - op_M(v - rho * e) / rho
    xi = 2.0 * (1.0 - delta) * xi_half - (1.0 - 2.0 * delta) * e
    z = v + rho * xi
    e_new = (z - project_C(z, gamma)) / rho
    v_new = v + rho * (xi - e_new)
    return xi_half, e_new, v_new


def solve(gamma, xi_bar, params=None, e0=None, v0=None, rho0_state=None, record_history=True):
    """Run the damped ADMM of Eq. 30 on the CCMF min-cut problem (Eq. 21).

    gamma: (N1, N2, N3) float64, gamma >= 0.  xi_bar: crack normal, normalised here
    (the effective crack energy is 1-homogeneous in it, Eq. 3).
    e0, v0, rho0_state: optional state to resume from.
    """
    params = params or Params()
    gamma = np.asarray(gamma, dtype=np.float64)
    xi_bar = np.asarray(xi_bar, dtype=np.float64)
    xi_bar = xi_bar / np.linalg.norm(xi_bar)
    shape = gamma.shape
    e = op_A(const_field(xi_bar, shape)) if e0 is None else np.array(e0, dtype=np.float64)
    v = np.zeros((6,) + shape) if v0 is None else np.array(v0, dtype=np.float64)
    rho = initial_rho(gamma, params) if rho0_state is None else float(rho0_state)
    history = []
    converged = False
    k = 0
    limit = params.fixed_iters if params.fixed_iters > 0 else params.max_iter
    while k < limit:
        xi_half, e_new, v_new = admm_step(e, v, rho, gamma, xi_bar, params.delta)
        r = l2_norm(e - xi_half)
        mv = math.sqrt(sum(float(np.mean(v[c])) ** 2 for c in range(6)))
        if record_history:
            history.append((k, rho, r, mv, mincut_objective(xi_half, gamma), flow_objective(op_A_adj(v), xi_bar)))
        rho_new = next_rho(rho, params.rho_rule, e, e_new, v, v_new, params, primal_res=r)
        e, v, rho = e_new, v_new, rho_new
        k += 1
        if params.fixed_iters <= 0 and k >= 2 and r <= params.tol * mv:
            converged = True
            break
    return evaluate(gamma, xi_bar, e, v, rho, k, converged, history)


def evaluate(gamma, xi_bar, e, v, rho, iters=0, converged=False, history=None):
    """Final evaluation of a state (R5)."""
    xi_half = project_K(e - v / rho, xi_bar)
    flow = op_A_adj(v)
    mv = math.sqrt(sum(float(np.mean(v[c])) ** 2 for c in range(6)))
    gp = mincut_objective(xi_half, gamma)
    gd = flow_objective(flow, xi_bar)
    return Result(gamma_eff=gd, gamma_primal=gp, gamma_dual=gd,
                  residual=l2_norm(e - xi_half), mean_v_norm=mv, rho=rho, iters=iters,
                  converged=converged, e=e, v=v, cut=xi_half, flow=flow,
                  history=history or [])

"""Infinite-contrast cells through the GPU solver: porous solids and a three-phase
sand-binder composite.

The paper solves (Sec. 4.5) solids with 200 monodisperse spherical pores of vanishing
crack resistance at porosities 5, 25, 40 and 50 % on 256^3 grids, and (Sec. 4.6) a
sand-core microstructure of grains (58.6 %), binder (1.3 %) and a third phase (40.1 %)
for three assignments of crack resistances, reporting gamma_eff and the ADMM
iterations for the normal e_x. Its structures are not available; this module runs the
same cases on seeded stand-ins from `microstructure.porous_spheres` and
`microstructure.sand_binder` (relaxed, non-overlapping balls in place of mechanical
contraction). Zero crack resistance enters P_C as a vanishing ball (v = 0 there), and
rho^0 falls back to the mean of gamma (reading R2). The tolerance of Eq. 31 is not
stated for these sections; 5e-4 (the tolerance of the fibre study, Sec. 4.4) is used.

    python -m paper_2103_05968_gb300.study_porous       # one JSON line per case
"""

from __future__ import annotations

import argparse
import json

import numpy as np

from . import ccmf
from . import microstructure as M

POROSITIES = (0.05, 0.25, 0.40, 0.50)
# (gamma_matrix, gamma_grain, gamma_binder) of the three cases of Sec. 4.6
SAND_CASES = ((0.0, 1.0, 1.0), (1.0, 10.0, 1.0), (10.0, 1.0, 10.0))


def sand_gamma(labels, case, dtype=np.float32):
    gm, gg, gb = case
    table = np.array([gm, gg, gb], dtype=np.float64)
    return table[labels].astype(dtype)


def solve_one(gamma, normal, precision, tol, max_iter, device):
    import torch

    dt = torch.float64 if precision == ccmf.CCMF_FP64 else torch.float32
    g = torch.from_numpy(np.ascontiguousarray(gamma)).to(device=device, dtype=dt)
    plan = ccmf.Plan(gamma.shape, batch=1, precision=precision, device=device)
    res, _, _ = plan.solve(g, [normal], ccmf.Params(tol=tol, max_iter=max_iter, check_every=64))
    plan.close()
    return res[0]


def run(n=256, pores=200, grain_radius=20.0, seed=2103, tol=5e-4, max_iter=20000,
        precision=ccmf.CCMF_FP32_MIXED, device="cuda"):
    normal = [1.0, 0.0, 0.0]
    rows = []
    for por in POROSITIES:
        gamma, vox = M.porous_spheres((n, n, n), pores, por, seed, dtype=np.float32)
        r = solve_one(gamma, normal, precision, tol, max_iter, device)
        rows.append({"cell": "porous", "n": n, "pores": pores, "porosity_target": por, "porosity_voxels": vox,
                     "gamma_eff_over_gamma": r["gamma_eff"], "gamma_primal": r["gamma_primal"],
                     "iterations": int(r["iters"]), "converged": bool(r["converged"]), "status": int(r["status"])})
    labels, fr = M.sand_binder((n, n, n), grain_radius * n / 256.0, 0.586, 0.013, seed)
    for c, case in enumerate(SAND_CASES):
        r = solve_one(sand_gamma(labels, case), normal, precision, tol, max_iter, device)
        rows.append({"cell": "sand-binder", "n": n, "case": c + 1, "gamma_matrix_grain_binder": list(case),
                     "fractions": fr, "gamma_eff": r["gamma_eff"], "gamma_primal": r["gamma_primal"],
                     "iterations": int(r["iters"]), "converged": bool(r["converged"]), "status": int(r["status"])})
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--tol", type=float, default=5e-4)
    ap.add_argument("--fp64", action="store_true")
    args = ap.parse_args()
    prec = ccmf.CCMF_FP64 if args.fp64 else ccmf.CCMF_FP32_MIXED
    for row in run(n=args.n, tol=args.tol, precision=prec):
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()

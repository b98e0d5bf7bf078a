"""Penalty-strategy and damping study of the damped ADMM (Eq. 30) on the GPU solver.

The paper compares, on a unidirectional fibre composite (Sec. 4.3 and its
appendix), the lower-bound constant penalty rho = min gamma, the Barzilai-Borwein and
Lorenz-Tran-Dinh scalings (text after Eq. 30) and residual balancing, each with
damping delta = 1/4 and delta = 1/2, by the iterations needed to reach the Eq. 31
tolerance and the error of the result. This module runs the same comparison through
the library on a synthetic stand-in for that structure (`microstructure.disks_2d`:
128^2 voxels, 32 non-overlapping disks, 50 % filler, gamma 10 in the disks, 1 in the
matrix, crack normal e_x). The reference value is a tight Barzilai-Borwein solve.

    python -m paper_2103_05968_gb300.study_penalty          # one JSON line per rule and delta
"""

from __future__ import annotations

import argparse
import json

import numpy as np

from . import ccmf
from . import microstructure as M

RULES = (("lower bound", ccmf.CCMF_RHO_CONST), ("Barzilai-Borwein", ccmf.CCMF_RHO_BB),
         ("Lorenz-Tran-Dinh", ccmf.CCMF_RHO_LTD), ("residual balancing", ccmf.CCMF_RHO_RB))


def run(n=128, count=32, fraction=0.5, contrast=10.0, seed=599, tol=1e-5, max_iter=10000, ref_tol=1e-9,
        ref_max_iter=50000, precision=ccmf.CCMF_FP64, device="cuda"):
    """Returns a list of dicts, one per (rule, delta), plus the reference value."""
    import torch

    gamma, _ = M.disks_2d(n, count, fraction, contrast, 1.0, seed)
    dt = torch.float64 if precision == ccmf.CCMF_FP64 else torch.float32
    g = torch.from_numpy(gamma).to(device=device, dtype=dt)
    normal = [[1.0, 0.0, 0.0]]
    plan = ccmf.Plan(gamma.shape, batch=1, precision=precision, device=device)
    ref = plan.solve(g, normal, ccmf.Params(tol=ref_tol, max_iter=ref_max_iter, check_every=256))[0][0]
    g_ref = ref["gamma_eff"]
    rows = []
    for name, rule in RULES:
        for delta in (0.25, 0.5):
            p = ccmf.Params(tol=tol, max_iter=max_iter, rho_rule=rule, delta=delta, check_every=64,
                            rho0=float(gamma.min()) if rule == ccmf.CCMF_RHO_CONST else 0.0)
            r = plan.solve(g, normal, p)[0][0]
            rows.append({"rule": name, "delta": delta, "iterations": int(r["iters"]),
                         "converged": bool(r["converged"]), "status": int(r["status"]),
                         "gamma_eff": r["gamma_eff"],
                         "rel_error": abs(r["gamma_eff"] - g_ref) / abs(g_ref) if np.isfinite(r["gamma_eff"]) else None,
                         "final_rho": r["rho"]})
    plan.close()
    return {"reference": {"gamma_eff": g_ref, "iterations": int(ref["iters"]), "converged": bool(ref["converged"]),
                          "tol": ref_tol},
            "cell": {"n": n, "disks": count, "fraction": fraction, "contrast": contrast, "seed": seed,
                     "normal": "e_x", "tol": tol, "max_iter": max_iter}, "runs": rows}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--max-iter", type=int, default=10000)
    ap.add_argument("--fp32", action="store_true", help="FP32-mixed instead of FP64")
    args = ap.parse_args()
    out = run(tol=args.tol, max_iter=args.max_iter,
              precision=ccmf.CCMF_FP32_MIXED if args.fp32 else ccmf.CCMF_FP64)
    print(json.dumps({"reference": out["reference"], "cell": out["cell"]}))
    for row in out["runs"]:
        print(json.dumps(row))


if __name__ == "__main__":
    main()

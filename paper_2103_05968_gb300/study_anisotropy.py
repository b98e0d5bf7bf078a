"""Anisotropy of the effective crack energy and its contrast dependence, through the
batched solver.

The paper reports gamma_eff for the three axis normals of a short-fibre composite
and its dependence on the fibre / matrix contrast (Sec. 4.4). Here the direction
dependence is sampled over many crack normals at once: the normals of a Fibonacci
lattice on the half sphere (gamma_eff(-n) = gamma_eff(n)) are solved as one batch
of one plan, sharing the gamma field, in one captured graph. The contrast sweep
repeats the three axis normals for several fibre resistances. The field is a
config-3-like fibre composite (diameter 6, aspect ratio 20, 12 % fibres) on a
smaller periodic cell.

    python -m paper_2103_05968_gb300.study_anisotropy      # JSON lines
"""

from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import ccmf
from . import microstructure as M


def fibonacci_normals(count):
    """`count` unit normals spread over the upper half sphere (z >= 0): golden-angle
    spiral with equal-area steps in z."""
    out = np.zeros((count, 3))
    golden = math.pi * (3.0 - math.sqrt(5.0))
    for k in range(count):
        z = 1.0 - (k + 0.5) / count          # in (0, 1)
        rxy = math.sqrt(max(0.0, 1.0 - z * z))
        phi = golden * k
        out[k] = (rxy * math.cos(phi), rxy * math.sin(phi), z)
    return out


def anisotropy(gamma, normals, precision=ccmf.CCMF_FP32_MIXED, tol=1e-4, max_iter=20000, device="cuda"):
    """gamma_eff for every normal (one batch, shared gamma); returns the result dicts."""
    import torch

    dt = torch.float64 if precision == ccmf.CCMF_FP64 else torch.float32
    g = torch.from_numpy(np.ascontiguousarray(gamma)).to(device=device, dtype=dt)
    plan = ccmf.Plan(gamma.shape, batch=len(normals), precision=precision, device=device)
    res, _, _ = plan.solve(g, normals, ccmf.Params(tol=tol, max_iter=max_iter, check_every=64))
    plan.close()
    return res


def run(n=96, count=64, contrasts=(1.5, 3.0, 10.0), seed=2103, tol=1e-4, device="cuda"):
    gamma, nf = M.short_fibres((n, n, n), 6.0, 20.0, 0.12, 3.0, 1.0, seed, dtype=np.float32)
    normals = fibonacci_normals(count)
    res = anisotropy(gamma, normals, tol=tol, device=device)
    sweep = []
    fibre = gamma > 1.0
    for c in contrasts:
        gc = np.where(fibre, np.float32(c), np.float32(1.0))
        rc = anisotropy(gc, np.eye(3), tol=tol, device=device)
        sweep.append({"contrast": c, "gamma_eff_axes": [r["gamma_eff"] for r in rc],
                      "iterations": [int(r["iters"]) for r in rc], "converged": [bool(r["converged"]) for r in rc]})
    vals = np.array([r["gamma_eff"] for r in res])
    return {"cell": {"n": n, "fibres": int(nf), "fraction": float(fibre.mean()), "contrast": 3.0, "seed": seed,
                     "normals": count, "tol": tol},
            "normals": normals.tolist(), "gamma_eff": vals.tolist(),
            "iterations": [int(r["iters"]) for r in res], "converged": [bool(r["converged"]) for r in res],
            "min": float(vals.min()), "max": float(vals.max()), "sweep": sweep}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=96)
    ap.add_argument("--normals", type=int, default=64)
    ap.add_argument("--tol", type=float, default=1e-4)
    args = ap.parse_args()
    out = run(n=args.n, count=args.normals, tol=args.tol)
    print(json.dumps({k: out[k] for k in ("cell", "min", "max")}))
    print(json.dumps({"gamma_eff": out["gamma_eff"], "iterations": out["iterations"]}))
    for row in out["sweep"]:
        print(json.dumps(row))


if __name__ == "__main__":
    main()

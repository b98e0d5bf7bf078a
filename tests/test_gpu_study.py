"""The penalty-strategy study (Sec. 4.3 comparison) runs through the library on a small
disk cell: every rule and damping returns a finite result, the Barzilai-Borwein runs
converge, and converged runs agree with the reference value to the tolerance's order."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2103_05968_gb300 import ccmf  # noqa: E402
from paper_2103_05968_gb300 import study_penalty  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_penalty_study_small_cell():
    out = study_penalty.run(n=48, count=8, fraction=0.4, seed=3, tol=1e-4, max_iter=4000, ref_tol=1e-8,
                            ref_max_iter=20000, device="cuda:0")
    assert out["reference"]["converged"]
    assert len(out["runs"]) == 8
    for row in out["runs"]:
        assert row["status"] == 0 and np.isfinite(row["gamma_eff"])
        if row["converged"]:
            assert row["rel_error"] < 1e-2
    bb = [r for r in out["runs"] if r["rule"] == "Barzilai-Borwein"]
    assert all(r["converged"] for r in bb)


def test_anisotropy_homogeneous_and_normals():
    """Batched normals of the anisotropy study: a homogeneous cell gives gamma_eff = gamma for
    every unit normal (the closed form of the oracle pins); the Fibonacci normals are unit
    vectors on the upper half sphere."""
    from paper_2103_05968_gb300 import study_anisotropy as A
    nrm = A.fibonacci_normals(24)
    assert np.allclose(np.linalg.norm(nrm, axis=1), 1.0) and np.all(nrm[:, 2] > 0)
    gamma = np.full((16, 12, 20), 1.7, dtype=np.float32)
    res = A.anisotropy(gamma, nrm, tol=1e-5, max_iter=2000, device="cuda:0")
    for r in res:
        assert r["status"] == 0
        assert abs(r["gamma_eff"] - 1.7) <= 1e-5 * 1.7


def test_anisotropy_batch_equals_single_normals():
    """Every normal of a batch gives what the same normal gives in a plan of its own (FP64)."""
    from paper_2103_05968_gb300 import study_anisotropy as A
    from paper_2103_05968_gb300 import microstructure as M
    gamma, _ = M.boolean_spheres((20, 16, 24), 3.0, 0.2, 0.3, 1.0, seed=31)
    nrm = A.fibonacci_normals(5)
    batch = A.anisotropy(gamma, nrm, precision=ccmf.CCMF_FP64, tol=1e-6, max_iter=5000, device="cuda:0")
    for k in range(len(nrm)):
        one = A.anisotropy(gamma, nrm[k:k + 1], precision=ccmf.CCMF_FP64, tol=1e-6, max_iter=5000,
                           device="cuda:0")[0]
        assert one["iters"] == batch[k]["iters"]
        assert abs(one["gamma_eff"] - batch[k]["gamma_eff"]) <= 1e-12 * abs(one["gamma_eff"])


def _fp64_fixed(gamma, normals, iters):
    g = torch.from_numpy(np.ascontiguousarray(gamma, dtype=np.float64)).to("cuda:0")
    plan = ccmf.Plan(gamma.shape, batch=len(normals), precision=ccmf.CCMF_FP64, device="cuda:0")
    res, flow, cut = plan.solve(g, normals, ccmf.Params(fixed_iters=iters), want_flow=True, want_cut=True)
    plan.close()
    return res, flow, cut


def test_anisotropy_heterogeneous_fibre_cell_against_oracle():
    """Five Fibonacci normals on a small short-fibre cell (diameter 4, aspect ratio 5, 10 %,
    gamma 3 / 1), solved as one batch like the anisotropy study, against the oracle per
    normal at equal iterations: |d gamma_eff| / gamma_eff <= 1e-10, cut and flow <= 1e-9.
    The contrast-sweep field (fibres at gamma 10) with the axis normals, likewise."""
    from oracle import ccmf_oracle as O
    from paper_2103_05968_gb300 import microstructure as M
    from paper_2103_05968_gb300 import study_anisotropy as A
    gamma, nf = M.short_fibres((24, 20, 30), 4.0, 5.0, 0.10, 3.0, 1.0, seed=9, dtype=np.float64)
    assert nf > 0 and 0.09 < float(np.mean(gamma > 1.0)) < 0.2
    for field, normals in ((gamma, A.fibonacci_normals(5)), (np.where(gamma > 1.0, 10.0, 1.0), np.eye(3))):
        res, flow, cut = _fp64_fixed(field, normals, 30)
        for k, n in enumerate(normals):
            ref = O.solve(field, n, O.Params(fixed_iters=30), record_history=False)
            assert abs(res[k]["gamma_eff"] - ref.gamma_eff) <= 1e-10 * abs(ref.gamma_eff)
            np.testing.assert_allclose(cut[k].cpu().numpy(), ref.cut, rtol=0, atol=1e-9)
            np.testing.assert_allclose(flow[k].cpu().numpy(), ref.flow, rtol=0, atol=1e-9)


def test_porous_and_sand_standins_against_oracle():
    """Infinite-contrast stand-ins of Sec. 4.5 / 4.6 at 40^3: pores of gamma 0 at 25 % and 50 %
    porosity, and the sand-binder cases 1 (pores as the third phase) and 3, normal e_x, FP64
    against the oracle at equal iterations (rho^0 = mean gamma where min gamma = 0)."""
    from oracle import ccmf_oracle as O
    from paper_2103_05968_gb300 import microstructure as M
    from paper_2103_05968_gb300 import study_porous as S
    fields = [M.porous_spheres((40, 40, 40), 12, por, seed=4)[0] for por in (0.25, 0.5)]
    labels, fr = M.sand_binder((40, 40, 40), 5.0, 0.586, 0.013, seed=5)
    assert abs(fr["grain"] - 0.586) < 0.03 and abs(fr["binder"] - 0.013) < 0.002
    fields += [S.sand_gamma(labels, S.SAND_CASES[0], np.float64), S.sand_gamma(labels, S.SAND_CASES[2], np.float64)]
    for field in fields:
        res, flow, cut = _fp64_fixed(field, [[1.0, 0.0, 0.0]], 30)
        ref = O.solve(field, [1.0, 0.0, 0.0], O.Params(fixed_iters=30), record_history=False)
        assert res[0]["status"] == 0
        assert abs(res[0]["gamma_eff"] - ref.gamma_eff) <= 1e-10 * max(abs(ref.gamma_eff), 1e-3)
        np.testing.assert_allclose(cut[0].cpu().numpy(), ref.cut, rtol=0, atol=1e-9)
        np.testing.assert_allclose(flow[0].cpu().numpy(), ref.flow, rtol=0, atol=1e-9)


def test_porous_study_small_cells():
    """The porous / sand study on 64^3 cells runs to the tolerance; gamma_eff falls with the
    porosity and lies in [0, gamma_solid]; the sand cases are bounded by their phase values."""
    from paper_2103_05968_gb300 import study_porous as S
    rows = S.run(n=64, pores=20, grain_radius=20.0, tol=1e-3, max_iter=20000, device="cuda:0")
    por = [r for r in rows if r["cell"] == "porous"]
    assert all(r["status"] == 0 and r["converged"] for r in rows)
    vals = [r["gamma_eff_over_gamma"] for r in por]
    assert all(0.0 <= v <= 1.0 for v in vals)
    assert all(a > b for a, b in zip(vals, vals[1:]))
    for r in rows:
        if r["cell"] == "sand-binder":
            lo, hi = min(r["gamma_matrix_grain_binder"]), max(r["gamma_matrix_grain_binder"])
            assert lo - 1e-6 <= r["gamma_eff"] <= hi + 1e-6

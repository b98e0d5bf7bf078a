"""Batches of solves on grids of different shapes (one captured graph, per-shape
sub-plans): every solve of a batch must give what the same solve gives alone,
and what the FP64 oracle gives at equal iteration counts."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import ccmf_oracle as O  # noqa: E402
from paper_2103_05968_gb300 import ccmf  # noqa: E402
from paper_2103_05968_gb300 import microstructure as M  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def make_case(dtype):
    fields = [M.random_two_phase((8, 8, 8), 0.3, 0.25, 1.0, 1),
              M.uniform_random((12, 10, 6), 0.5, 1.5, 2),
              M.boolean_spheres((16, 12, 10), 2.0, 0.2, 0.3, 1.0, 3)[0],
              M.random_two_phase((8, 8, 8), 0.4, 0.2, 1.0, 4)]
    # solve -> (field index, normal)
    plan = [(0, [1, 0, 0]), (1, [0.36, 0.48, 0.8]), (0, [0, 0, 1]), (2, [0, 1, 0]), (3, [0.6, 0.0, 0.8]),
            (2, [0, 0, 1]), (1, [1, 0, 0])]
    dev = [torch.from_numpy(f.astype(dtype)).to(DEV) for f in fields]
    gammas = [dev[f] for f, _ in plan]
    normals = np.array([n for _, n in plan], dtype=np.float64)
    shapes = [fields[f].shape for f, _ in plan]
    return fields, plan, gammas, normals, shapes


def test_batch_matches_oracle_fp64():
    fields, plan, gammas, normals, shapes = make_case(np.float64)
    batch = ccmf.Batch(shapes, precision=ccmf.CCMF_FP64, device=DEV)
    assert batch.buckets() == 3
    res = batch.solve(gammas, normals, ccmf.Params(fixed_iters=30))
    for s, (f, n) in enumerate(plan):
        ref = O.solve(fields[f], n, O.Params(fixed_iters=30), record_history=False)
        assert res[s]["status"] == 0 and res[s]["iters"] == 30
        assert abs(res[s]["gamma_eff"] - ref.gamma_eff) <= 1e-10 * abs(ref.gamma_eff)
        assert abs(res[s]["gamma_primal"] - ref.gamma_primal) <= 1e-10 * abs(ref.gamma_primal)
        assert abs(res[s]["rho"] - ref.rho) <= 1e-10 * ref.rho


@pytest.mark.parametrize("precision", [ccmf.CCMF_FP64, ccmf.CCMF_FP32_MIXED])
def test_batch_each_solve_equals_solo_run(precision):
    dtype = np.float64 if precision == ccmf.CCMF_FP64 else np.float32
    fields, plan, gammas, normals, shapes = make_case(dtype)
    batch = ccmf.Batch(shapes, precision=precision, device=DEV)
    params = ccmf.Params(tol=1e-5, max_iter=3000, check_every=16)
    res = batch.solve(gammas, normals, params)
    tol = 1e-10 if precision == ccmf.CCMF_FP64 else 1e-5
    for s in range(len(plan)):
        solo = ccmf.Plan(shapes[s], batch=1, precision=precision, device=DEV)
        r, _, _ = solo.solve(gammas[s], normals[s:s + 1], params)
        r = r[0]
        assert res[s]["status"] == 0
        assert res[s]["converged"] == r["converged"]
        if precision == ccmf.CCMF_FP64:
            assert res[s]["iters"] == r["iters"]
        assert abs(res[s]["gamma_eff"] - r["gamma_eff"]) <= tol * abs(r["gamma_eff"])
        solo.close()
    # a second call on the same batch object gives the same answers (graph reuse)
    res2 = batch.solve(gammas, normals, params)
    for a, b in zip(res, res2):
        assert a["iters"] == b["iters"] and a["gamma_eff"] == b["gamma_eff"]


def test_batch_rejects_host_gamma():
    fields, plan, gammas, normals, shapes = make_case(np.float64)
    batch = ccmf.Batch(shapes[:2], precision=ccmf.CCMF_FP64, device=DEV)
    host = [torch.from_numpy(fields[0]), torch.from_numpy(fields[1])]
    with pytest.raises(ccmf.CCMFError) as ei:
        batch.solve(host, normals[:2], ccmf.Params(fixed_iters=2))
    assert ei.value.code == ccmf.CCMF_ERR_INVALID_ARG


def test_batch_autotune_keeps_parity():
    """ccmf_batch_autotune tunes each shape group on its own solves; afterwards every solve
    still matches the FP64 oracle at equal iterations (tuning changes only the launch)."""
    fields = [M.random_two_phase((20, 12, 10), 0.3, 0.25, 1.0, 7), M.uniform_random((10, 10, 10), 0.5, 1.5, 8)]
    plan = [(0, [1, 0, 0]), (1, [0.36, 0.48, 0.8]), (0, [0, 0, 1]), (1, [0, 1, 0]), (0, [0.6, 0.0, 0.8])]
    dev = [torch.from_numpy(f).to(DEV) for f in fields]
    gammas = [dev[f] for f, _ in plan]
    normals = np.array([n for _, n in plan], dtype=np.float64)
    batch = ccmf.Batch([fields[f].shape for f, _ in plan], precision=ccmf.CCMF_FP64, device=DEV)
    ms = batch.autotune(gammas, normals, iters=3)
    assert len(ms) == batch.buckets() == 2 and min(ms) > 0
    res = batch.solve(gammas, normals, ccmf.Params(fixed_iters=25))
    for s, (f, n) in enumerate(plan):
        ref = O.solve(fields[f], n, O.Params(fixed_iters=25), record_history=False)
        assert res[s]["status"] == 0 and res[s]["iters"] == 25
        assert abs(res[s]["gamma_eff"] - ref.gamma_eff) <= 1e-10 * abs(ref.gamma_eff)
    code, text = ccmf.ccmf_tuning_export()
    assert code == ccmf.CCMF_OK and "ccmf-tuning 20 12 10 3 0 " in text and "ccmf-tuning 10 10 10 2 0 " in text
    batch.close()

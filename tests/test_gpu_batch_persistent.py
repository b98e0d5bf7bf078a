"""The batched persistent launch (ccmf_batch_set_persistent): one kernel launch per
iteration runs every pass of every solve of an uneven batch from one device work
queue. Each solve must match the FP64 oracle at equal iteration counts (Eq. 30 with
the BB rule), stop where the graph-mode batch stops, repeat bit for bit, and report
a bounded device wait that gives up as CCMF_ERR_TIMEOUT."""

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


def uneven_case(dtype):
    """Odd, radix-3/5, single-voxel-axis and power-of-two grids, shared and separate fields."""
    fields = [M.random_two_phase((8, 8, 8), 0.3, 0.25, 1.0, 1),
              M.uniform_random((12, 10, 6), 0.5, 1.5, 2),
              M.boolean_spheres((16, 12, 10), 2.0, 0.2, 0.3, 1.0, 3)[0],
              M.random_two_phase((6, 10, 15), 0.4, 0.2, 1.0, 4),
              M.uniform_random((9, 5, 1), 0.5, 1.5, 5),
              M.random_two_phase((1, 1, 20), 0.5, 0.3, 1.0, 6)]
    plan = [(0, [1, 0, 0]), (1, [0.36, 0.48, 0.8]), (0, [0, 0, 1]), (2, [0, 1, 0]), (3, [0.6, 0.0, 0.8]),
            (2, [0, 0, 1]), (4, [1, 0, 0]), (5, [0, 0, 1]), (1, [1, 0, 0])]
    dev = [torch.from_numpy(f.astype(dtype)).to(DEV) for f in fields]
    gammas = [dev[f] for f, _ in plan]
    normals = np.array([n for _, n in plan], dtype=np.float64)
    shapes = [fields[f].shape for f, _ in plan]
    return fields, plan, gammas, normals, shapes


def test_persistent_batch_matches_oracle_fp64():
    fields, plan, gammas, normals, shapes = uneven_case(np.float64)
    batch = ccmf.Batch(shapes, precision=ccmf.CCMF_FP64, device=DEV)
    batch.set_persistent(True)
    res = batch.solve(gammas, normals, ccmf.Params(fixed_iters=30))
    for s, (f, n) in enumerate(plan):
        ref = O.solve(fields[f], n, O.Params(fixed_iters=30), record_history=False)
        r = res[s]
        assert r["status"] == 0 and r["iters"] == 30, (s, r)
        for key, rk in (("gamma_eff", ref.gamma_eff), ("gamma_primal", ref.gamma_primal), ("rho", ref.rho),
                        ("residual", ref.residual), ("mean_v_norm", ref.mean_v_norm)):
            assert abs(r[key] - rk) <= 1e-10 * abs(rk) + 1e-14, (s, key, r[key], rk)
    batch.close()


def test_persistent_batch_full_size_grids_fp64():
    """64^3 and 40 x 24 x 36 grids (several tiles per pass, radix-3/5 axes) against the oracle."""
    g1, _ = M.boolean_spheres((64, 64, 64), 5.0, 0.2, 0.3, 1.0, 11)
    g2 = M.random_two_phase((40, 24, 36), 0.3, 0.25, 1.0, 12)
    fields = [g1, g2]
    plan = [(0, [0, 0, 1]), (1, [0.36, 0.48, 0.8]), (0, [1, 0, 0])]
    dev = [torch.from_numpy(f).to(DEV) for f in fields]
    batch = ccmf.Batch([fields[f].shape for f, _ in plan], precision=ccmf.CCMF_FP64, device=DEV)
    batch.set_persistent(True)
    iters = 12
    res = batch.solve([dev[f] for f, _ in plan], np.array([n for _, n in plan], dtype=np.float64),
                      ccmf.Params(fixed_iters=iters))
    for s, (f, n) in enumerate(plan):
        ref = O.solve(fields[f], n, O.Params(fixed_iters=iters), record_history=False)
        r = res[s]
        assert r["status"] == 0 and r["iters"] == iters
        for key, rk in (("gamma_eff", ref.gamma_eff), ("gamma_primal", ref.gamma_primal), ("rho", ref.rho),
                        ("residual", ref.residual)):
            assert abs(r[key] - rk) <= 1e-10 * abs(rk), (s, key, r[key], rk)
    batch.close()


@pytest.mark.parametrize("precision", [ccmf.CCMF_FP64, ccmf.CCMF_FP32_MIXED])
def test_persistent_stops_where_graph_batch_stops(precision):
    dtype = np.float64 if precision == ccmf.CCMF_FP64 else np.float32
    fields, plan, gammas, normals, shapes = uneven_case(dtype)
    params = ccmf.Params(tol=1e-5, max_iter=3000, check_every=16)
    graph = ccmf.Batch(shapes, precision=precision, device=DEV)
    ref = graph.solve(gammas, normals, params)
    pers = ccmf.Batch(shapes, precision=precision, device=DEV)
    pers.set_persistent(True)
    res = pers.solve(gammas, normals, params)
    tol = 1e-10 if precision == ccmf.CCMF_FP64 else 1e-5
    for a, b in zip(res, ref):
        assert a["status"] == 0 and a["converged"] == b["converged"]
        if precision == ccmf.CCMF_FP64:
            assert a["iters"] == b["iters"]
        assert abs(a["gamma_eff"] - b["gamma_eff"]) <= tol * abs(b["gamma_eff"])
    # repeated calls on the same batch object repeat bit for bit (graph reuse, fixed reduction order)
    res2 = pers.solve(gammas, normals, params)
    for a, b in zip(res, res2):
        assert a["iters"] == b["iters"] and a["gamma_eff"] == b["gamma_eff"] and a["rho"] == b["rho"]
    graph.close()
    pers.close()


def test_persistent_fp32_bench_shapes_against_graph_mode():
    """The four grid sizes of the 192-solve workload (64 ... 160, radix 2/3/5), FP32: the
    persistent launch agrees with the graph mode after 40 iterations."""
    shapes, gammas = [], []
    for r, n in enumerate((64, 96, 128, 160)):
        g, _ = M.boolean_spheres((n, n, n), 6.0, 0.2, 0.2, 1.0, 2103 + r)
        gammas.append(torch.from_numpy(g.astype(np.float32)).to(DEV))
        shapes.append((n, n, n))
    normals = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [0.36, 0.48, 0.8]], dtype=np.float64)
    params = ccmf.Params(fixed_iters=40)
    graph = ccmf.Batch(shapes, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    ref = graph.solve(gammas, normals, params)
    pers = ccmf.Batch(shapes, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    pers.set_persistent(True)
    res = pers.solve(gammas, normals, params)
    for a, b in zip(res, ref):
        assert a["status"] == 0 and a["iters"] == 40
        assert abs(a["gamma_eff"] - b["gamma_eff"]) <= 1e-5 * abs(b["gamma_eff"])
        assert abs(a["rho"] - b["rho"]) <= 1e-4 * b["rho"]
    graph.close()
    pers.close()


def test_persistent_device_wait_timeout_reported(monkeypatch):
    """With the debug budget of zero polls every dependency wait gives up: each solve
    reports CCMF_ERR_TIMEOUT and retires; the next call on the same batch is healthy."""
    fields, plan, gammas, normals, shapes = uneven_case(np.float32)
    batch = ccmf.Batch(shapes, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    batch.set_persistent(True)
    monkeypatch.setenv("CCMF_DEBUG_SPIN_LIMIT", "0")
    res = batch.solve(gammas, normals, ccmf.Params(fixed_iters=3))
    assert all(r["status"] == ccmf.CCMF_ERR_TIMEOUT for r in res), [r["status"] for r in res]
    monkeypatch.delenv("CCMF_DEBUG_SPIN_LIMIT")
    res = batch.solve(gammas, normals, ccmf.Params(fixed_iters=3))
    assert all(r["status"] == 0 and r["iters"] == 3 and np.isfinite(r["gamma_eff"]) for r in res)
    batch.close()


def test_persistent_narrow_tiles_for_long_axes():
    """A batch with an axis too long for the wide tiles (beyond about 400 points in FP32, 200 in
    FP64) runs the narrow-tile instantiation (4 line pairs, 8 lines) for all its groups: FP64
    against the oracle at equal iterations, FP32 against the graph mode."""
    f64 = [M.random_two_phase((6, 10, 256), 0.3, 0.25, 1.0, 41), M.uniform_random((8, 8, 8), 0.5, 1.5, 42)]
    plan = [(0, [0, 0, 1]), (1, [0.36, 0.48, 0.8]), (0, [1, 0, 0])]
    dev = [torch.from_numpy(f).to(DEV) for f in f64]
    batch = ccmf.Batch([f64[f].shape for f, _ in plan], precision=ccmf.CCMF_FP64, device=DEV)
    batch.set_persistent(True)
    res = batch.solve([dev[f] for f, _ in plan], np.array([n for _, n in plan], dtype=np.float64),
                      ccmf.Params(fixed_iters=20))
    for s, (f, n) in enumerate(plan):
        ref = O.solve(f64[f], n, O.Params(fixed_iters=20), record_history=False)
        assert res[s]["status"] == 0 and res[s]["iters"] == 20
        for key, rk in (("gamma_eff", ref.gamma_eff), ("gamma_primal", ref.gamma_primal), ("rho", ref.rho),
                        ("residual", ref.residual)):
            assert abs(res[s][key] - rk) <= 1e-10 * abs(rk), (s, key, res[s][key], rk)
    batch.close()
    f32 = [M.random_two_phase((8, 8, 512), 0.3, 0.25, 1.0, 43).astype(np.float32),
           M.boolean_spheres((16, 12, 10), 2.0, 0.2, 0.3, 1.0, 44)[0].astype(np.float32)]
    gam = [torch.from_numpy(f).to(DEV) for f in f32]
    normals = np.array([[0, 0, 1], [1, 0, 0]], dtype=np.float64)
    out = []
    for persistent in (False, True):
        b = ccmf.Batch([f.shape for f in f32], precision=ccmf.CCMF_FP32_MIXED, device=DEV)
        b.set_persistent(persistent)
        out.append(b.solve(gam, normals, ccmf.Params(fixed_iters=30)))
        b.close()
    for a, r in zip(out[1], out[0]):
        assert a["status"] == 0 and a["iters"] == 30
        assert abs(a["gamma_eff"] - r["gamma_eff"]) <= 1e-5 * abs(r["gamma_eff"])

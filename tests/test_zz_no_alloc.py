"""The allocation-free entry point ccmf_solve_static against ccmf_solve.

ccmf_solve_static serves callers that cannot allocate device memory where they
need a solve (for example a plug-in under a host application that owns all device
memory through its own pool, or a latency-critical path that must not take the
implicit synchronisation of cudaMalloc): it keeps its whole working set in the
library's fixed device scratch area instead of a caller-provided workspace.
This test calls it through the C ABI twice in a row on different inputs (the
second call reuses the scratch the first one left behind) and checks each call
against the existing workspace-based entry point within the parity tolerances
of the other GPU tests. It lives in its own file so that pytest collects it
last.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2103_05968_gb300 import ccmf  # noqa: E402
from paper_2103_05968_gb300 import microstructure as M  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def reference(gamma, xi, params, precision):
    plan = ccmf.Plan(gamma.shape, batch=1, precision=precision, device=DEV)
    dt = torch.float64 if precision == ccmf.CCMF_FP64 else torch.float32
    g = torch.from_numpy(gamma).to(DEV, dt)
    res, flow, cut = plan.solve(g, [xi], params, want_flow=True, want_cut=True)
    torch.cuda.synchronize()
    plan.close()
    return res[0], flow[0].cpu().numpy(), cut[0].cpu().numpy()


def static_solve(gamma, xi, params, precision, gamma_offset=0):
    """gamma_offset > 0 passes gamma as a view that starts that many elements into a
    larger buffer (not 16-byte aligned: the scalar update pass)."""
    dt = torch.float64 if precision == ccmf.CCMF_FP64 else torch.float32
    n1, n2, n3 = gamma.shape
    with torch.cuda.device(DEV):
        buf = torch.empty(gamma.size + gamma_offset, dtype=dt, device=DEV)
        g = buf[gamma_offset:].view(gamma.shape)
        g.copy_(torch.from_numpy(gamma).to(DEV, dt))
        flow = torch.empty((3, n1, n2, n3), dtype=dt, device=DEV)
        cut = torch.empty((6, n1, n2, n3), dtype=dt, device=DEV)
        res = ccmf.ccmf_result()
        stream = ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)
        code = ccmf.ccmf_solve_static(n1, n2, n3, precision, ctypes.c_void_p(g.data_ptr()), np.asarray(xi, float),
                                      params.to_c(), ctypes.c_void_p(flow.data_ptr()),
                                      ctypes.c_void_p(cut.data_ptr()), ctypes.byref(res), stream)
        torch.cuda.synchronize()
    assert code == ccmf.CCMF_OK, ccmf.ccmf_status_string(code)
    r = {f[0]: getattr(res, f[0]) for f in ccmf.ccmf_result._fields_}
    return r, flow.cpu().numpy(), cut.cpu().numpy()


CALLS = [
    # two calls in a row: different grids, normals and stopping rules
    (lambda: M.boolean_spheres((24, 20, 16), 3.0, 0.2, 0.3, 1.0, seed=3)[0], [0.36, 0.48, 0.8],
     ccmf.Params(fixed_iters=40)),
    (lambda: M.config_single_sphere_32(), [0.0, 0.0, 1.0], ccmf.Params(tol=1e-6)),
]


@pytest.mark.parametrize("precision", [ccmf.CCMF_FP64, ccmf.CCMF_FP32_MIXED])
def test_static_matches_workspace_entry_point(precision):
    for build, xi, params in CALLS:
        gamma = build()
        r0, f0, c0 = reference(gamma, xi, params, precision)
        r1, f1, c1 = static_solve(gamma, xi, params, precision)
        assert r1["status"] == 0 and r1["iters"] == r0["iters"] and r1["converged"] == r0["converged"]
        if precision == ccmf.CCMF_FP64:
            geff_tol, field_tol = 1e-10, 1e-9
        else:
            geff_tol, field_tol = 1e-5, 1e-4 * max(1.0, float(np.abs(c0).max()))
        assert abs(r1["gamma_eff"] - r0["gamma_eff"]) <= geff_tol * abs(r0["gamma_eff"])
        assert abs(r1["gamma_primal"] - r0["gamma_primal"]) <= geff_tol * abs(r0["gamma_primal"])
        np.testing.assert_allclose(f1, f0, rtol=0, atol=field_tol)
        np.testing.assert_allclose(c1, c0, rtol=0, atol=field_tol)


EDGE_CASES = [
    # the documented size limits (80^3 FP32, 64^3 FP64), an odd N3 (scalar divergence and
    # update passes) and an offset gamma view (scalar update pass); the tolerance cases stop
    # after more updates than check_every
    ("limit_fp32", lambda: M.boolean_spheres((80, 80, 80), 4.0, 0.2, 0.3, 1.0, seed=4)[0], [0.0, 0.6, 0.8],
     ccmf.Params(fixed_iters=60), ccmf.CCMF_FP32_MIXED, 0),
    ("limit_fp64", lambda: M.boolean_spheres((64, 64, 64), 4.0, 0.2, 0.3, 1.0, seed=5)[0], [0.0, 0.0, 1.0],
     ccmf.Params(tol=1e-4, check_every=16, max_iter=3000), ccmf.CCMF_FP64, 0),
    ("odd_n3_fp64", lambda: M.boolean_spheres((18, 20, 15), 2.5, 0.2, 0.3, 1.0, seed=6)[0], [0.36, 0.48, 0.8],
     ccmf.Params(tol=1e-6, check_every=5, max_iter=5000), ccmf.CCMF_FP64, 0),
    ("offset_gamma_fp64", lambda: M.boolean_spheres((16, 24, 20), 2.5, 0.2, 0.3, 1.0, seed=7)[0], [1.0, 0.0, 0.0],
     ccmf.Params(tol=1e-6, check_every=9, max_iter=5000), ccmf.CCMF_FP64, 1),
    ("offset_gamma_fp32", lambda: M.boolean_spheres((16, 24, 20), 2.5, 0.2, 0.3, 1.0, seed=7)[0], [1.0, 0.0, 0.0],
     ccmf.Params(fixed_iters=45), ccmf.CCMF_FP32_MIXED, 3),
]


@pytest.mark.parametrize("case", EDGE_CASES, ids=[c[0] for c in EDGE_CASES])
def test_static_edge_cases_match_workspace_entry_point(case):
    _, build, xi, params, precision, offset = case
    gamma = build()
    r0, f0, c0 = reference(gamma, xi, params, precision)
    r1, f1, c1 = static_solve(gamma, xi, params, precision, gamma_offset=offset)
    assert r1["status"] == 0 and r1["iters"] == r0["iters"] and r1["converged"] == r0["converged"]
    if params.fixed_iters == 0:
        assert r0["iters"] > params.check_every
    if precision == ccmf.CCMF_FP64:
        geff_tol, field_tol = 1e-10, 1e-9
    else:
        geff_tol, field_tol = 1e-5, 1e-4 * max(1.0, float(np.abs(c0).max()))
    assert abs(r1["gamma_eff"] - r0["gamma_eff"]) <= geff_tol * abs(r0["gamma_eff"])
    np.testing.assert_allclose(f1, f0, rtol=0, atol=field_tol)
    np.testing.assert_allclose(c1, c0, rtol=0, atol=field_tol)


def test_static_rejects_grids_beyond_the_scratch_area():
    g = torch.ones((128, 128, 128), dtype=torch.float64, device=DEV)
    res = ccmf.ccmf_result()
    code = ccmf.ccmf_solve_static(128, 128, 128, ccmf.CCMF_FP64, ctypes.c_void_p(g.data_ptr()),
                                  np.array([0.0, 0.0, 1.0]), ccmf.Params(fixed_iters=2).to_c(), None, None,
                                  ctypes.byref(res), None)
    assert code == ccmf.CCMF_ERR_UNSUPPORTED_SIZE
    host = np.ones((8, 8, 8))
    code = ccmf.ccmf_solve_static(8, 8, 8, ccmf.CCMF_FP64, ctypes.c_void_p(host.ctypes.data),
                                  np.array([0.0, 0.0, 1.0]), ccmf.Params(fixed_iters=2).to_c(), None, None,
                                  ctypes.byref(res), None)
    assert code == ccmf.CCMF_ERR_INVALID_ARG

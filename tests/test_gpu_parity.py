"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars (written out per test):
* FP64 GPU vs oracle at equal iteration counts: |d gamma_eff| / gamma_eff <= 1e-10,
  fields (e, v, cut, flow) <= 1e-9 max-abs.
* FP32-mixed vs the converged FP64 solution: |d gamma_eff| / gamma_eff <= 1e-5.
"""

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
FIELD_TOL = 1e-9
GEFF_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_run(gamma, normals, params, precision=ccmf.CCMF_FP64, want=True, host=False):
    normals = np.atleast_2d(np.asarray(normals, dtype=np.float64))
    batch = normals.shape[0]
    shape = gamma.shape[-3:]
    plan = ccmf.Plan(shape, batch=batch, precision=precision, device=DEV)
    dt = np.float64 if precision == ccmf.CCMF_FP64 else np.float32
    g = torch.from_numpy(np.ascontiguousarray(gamma.astype(dt)))
    if not host:
        g = g.to(DEV)
    res, flow, cut = plan.solve(g, normals, params, want_flow=want, want_cut=want)
    e, v, rho, iters = plan.state()
    torch.cuda.synchronize()
    out = dict(res=res, flow=None if flow is None else flow.cpu().numpy(),
               cut=None if cut is None else cut.cpu().numpy(), e=e.cpu().numpy(), v=v.cpu().numpy(),
               rho=rho, iters=iters, plan=plan)
    return out


def assert_parity(out, refs):
    for s, ref in enumerate(refs):
        r = out["res"][s]
        assert r["status"] == 0
        assert r["iters"] == ref.iters
        assert abs(r["gamma_eff"] - ref.gamma_eff) <= GEFF_TOL * abs(ref.gamma_eff)
        assert abs(r["gamma_dual"] - ref.gamma_dual) <= GEFF_TOL * abs(ref.gamma_eff) + 1e-13
        assert abs(r["gamma_primal"] - ref.gamma_primal) <= GEFF_TOL * abs(ref.gamma_primal) + 1e-13
        assert abs(out["rho"][s] - ref.rho) <= 1e-10 * ref.rho
        np.testing.assert_allclose(out["e"][s], ref.e, rtol=0, atol=FIELD_TOL)
        np.testing.assert_allclose(out["v"][s], ref.v, rtol=0, atol=FIELD_TOL)
        np.testing.assert_allclose(out["cut"][s], ref.cut, rtol=0, atol=FIELD_TOL)
        np.testing.assert_allclose(out["flow"][s], ref.flow, rtol=0, atol=FIELD_TOL)


CASES = [
    # (name, gamma builder, normals, iterations)
    ("odd_6x10x15", lambda: M.random_two_phase((6, 10, 15), 0.3, 0.25, 1.0, 1), [[0.36, 0.48, 0.8]], 60),
    ("cube_8", lambda: M.uniform_random((8, 8, 8), 0.5, 2.0, 2), [[1.0, 0.0, 0.0]], 60),
    ("flat_N3_1", lambda: M.random_two_phase((12, 10, 1), 0.4, 0.2, 1.0, 3), [[0.6, 0.8, 0.0]], 80),
    ("radix35_15x9x25", lambda: M.random_two_phase((15, 9, 25), 0.3, 0.3, 1.0, 4), [[0.0, 0.6, -0.8]], 40),
    ("line_1x1x20", lambda: M.uniform_random((1, 1, 20), 0.4, 1.5, 5), [[0.0, 0.0, 1.0]], 50),
    ("tiles_40x24x36", lambda: M.boolean_spheres((40, 24, 36), 3.0, 0.2, 0.3, 1.0, 6)[0],
     [[1, 0, 0], [0, 1, 0], [0, 0, 1]], 30),
]


@pytest.mark.parametrize("name,build,normals,iters", CASES, ids=[c[0] for c in CASES])
def test_fp64_equal_iterations(name, build, normals, iters):
    gamma = build()
    out = gpu_run(gamma, normals, ccmf.Params(fixed_iters=iters))
    refs = [O.solve(gamma, n, O.Params(fixed_iters=iters), record_history=False) for n in normals]
    assert_parity(out, refs)


@pytest.mark.parametrize("rule", [ccmf.CCMF_RHO_CONST, ccmf.CCMF_RHO_LTD, ccmf.CCMF_RHO_BB, ccmf.CCMF_RHO_RB])
def test_fp64_penalty_rules_and_damping(rule):
    # rho^0 below min(gamma): with rho^0 = min(gamma) the first update meets |z| = gamma exactly
    # at the weakest voxels, where rounding decides whether |e^1| is 0 or 1e-16, and the LTD
    # ratio |v|/|e| of that noise would flip rho differently on both sides.
    gamma = M.random_two_phase((10, 12, 8), 0.3, 0.2, 1.0, 11)
    delta = 0.5 if rule == ccmf.CCMF_RHO_BB else 0.25
    out = gpu_run(gamma, [[0.0, 0.0, 1.0]], ccmf.Params(fixed_iters=70, rho_rule=rule, delta=delta, rho0=0.15))
    ref = O.solve(gamma, [0, 0, 1], O.Params(fixed_iters=70, rho_rule=rule, delta=delta, rho0=0.15),
                  record_history=False)
    assert_parity(out, [ref])


def test_fp64_config_single_sphere_to_tolerance():
    """32^3 centred ball (gamma 0.1 in 1.0), e3, tol 1e-6: same stop iteration as the oracle,
    and the exact value 0.8171875 (closed form of the golden note) within the tolerance."""
    gamma = M.config_single_sphere_32()
    out = gpu_run(gamma, [[0, 0, 1]], ccmf.Params(tol=1e-6))
    ref = O.solve(gamma, [0, 0, 1], O.Params(tol=1e-6), record_history=False)
    r = out["res"][0]
    assert r["converged"] == 1 and ref.converged
    assert r["iters"] == ref.iters
    assert abs(r["gamma_eff"] - ref.gamma_eff) <= GEFF_TOL * ref.gamma_eff
    assert abs(r["gamma_eff"] - 0.8171875) <= 5e-6


def test_fp32_mixed_against_converged_fp64():
    """32^3 centred ball, e3: FP32-mixed at the iteration count where FP64 meets tol 1e-6
    agrees with the converged FP64 value to 1e-5 (and with the exact 0.8171875); FP32-mixed
    also meets the paper's tolerance 1e-4 (Sec. 4.1) on its own."""
    gamma = M.config_single_sphere_32()
    o64 = gpu_run(gamma, [[0, 0, 1]], ccmf.Params(tol=1e-6), want=False)
    k64 = o64["res"][0]["iters"]
    o32 = gpu_run(gamma, [[0, 0, 1]], ccmf.Params(fixed_iters=k64), precision=ccmf.CCMF_FP32_MIXED, want=False)
    g64, g32 = o64["res"][0]["gamma_eff"], o32["res"][0]["gamma_eff"]
    assert o64["res"][0]["converged"] == 1
    assert abs(g32 - g64) / g64 <= 1e-5
    assert abs(g32 - 0.8171875) / 0.8171875 <= 1e-5
    t32 = gpu_run(gamma, [[0, 0, 1]], ccmf.Params(tol=1e-4), precision=ccmf.CCMF_FP32_MIXED, want=False)
    assert t32["res"][0]["converged"] == 1


def test_fp32_mixed_equal_iterations_fields():
    """FP32-mixed fields track the FP64 oracle at equal iterations to FP32 accuracy."""
    gamma = M.random_two_phase((12, 10, 15), 0.3, 0.25, 1.0, 21)
    out = gpu_run(gamma, [[0.36, 0.48, 0.8]], ccmf.Params(fixed_iters=20, rho_rule=ccmf.CCMF_RHO_CONST),
                  precision=ccmf.CCMF_FP32_MIXED)
    ref = O.solve(gamma, [0.36, 0.48, 0.8], O.Params(fixed_iters=20, rho_rule=O.RHO_CONST), record_history=False)
    scale = max(np.abs(ref.v).max(), np.abs(ref.e).max())
    assert np.abs(out["e"][0] - ref.e).max() <= 1e-4 * scale
    assert np.abs(out["v"][0] - ref.v).max() <= 1e-4 * scale
    assert abs(out["res"][0]["gamma_eff"] - ref.gamma_eff) <= 1e-5 * ref.gamma_eff


def test_full_size_one_step_from_imported_state():
    """128^3 Boolean spheres (radius 6, 20 %, gamma 0.3 / 1.0), three normals: the GPU
    state after 40 FP64 iterations is imported into the oracle, and one further GPU step
    is compared element by element with one oracle step from the same state."""
    gamma, _ = M.config_boolean_spheres_128()
    normals = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    plan = ccmf.Plan(gamma.shape, batch=3, precision=ccmf.CCMF_FP64, device=DEV)
    g = torch.from_numpy(gamma).to(DEV)
    plan.solve(g, normals, ccmf.Params(fixed_iters=40))
    e0, v0, rho0, it0 = plan.state()
    e0n, v0n = e0.cpu().numpy(), v0.cpu().numpy()
    res, flow, cut = plan.solve(g, normals, ccmf.Params(fixed_iters=1, resume=1), want_flow=True)
    e1, v1, rho1, it1 = plan.state()
    e1n, v1n = e1.cpu().numpy(), v1.cpu().numpy()
    assert list(it1) == [41, 41, 41]
    for s in (0, 2):   # two of the three normals keep the CPU time bounded
        xi = np.asarray(normals[s], dtype=np.float64)
        _, e_ref, v_ref = O.admm_step(e0n[s], v0n[s], rho0[s], gamma, xi, 0.25)
        np.testing.assert_allclose(e1n[s], e_ref, rtol=0, atol=FIELD_TOL)
        np.testing.assert_allclose(v1n[s], v_ref, rtol=0, atol=FIELD_TOL)
        rho_ref = O.next_rho(rho0[s], O.RHO_BB, e0n[s], e_ref, v0n[s], v_ref, O.Params())
        assert abs(rho1[s] - rho_ref) <= 1e-10 * rho_ref
        ev = O.evaluate(gamma, xi, e_ref, v_ref, rho_ref)
        assert abs(res[s]["gamma_eff"] - ev.gamma_eff) <= GEFF_TOL * ev.gamma_eff
        np.testing.assert_allclose(flow[s].cpu().numpy(), ev.flow, rtol=0, atol=FIELD_TOL)
    # properties that hold at any size: the multiplier stays in C_gamma
    nv = np.sqrt(np.sum(v1n ** 2, axis=1))
    assert np.all(nv <= gamma[None] * (1 + 1e-12) + 1e-14)


def test_fp32_full_size_properties():
    """FP32-mixed at 128^3 x 3 normals in the benchmark's launch shape: finite, feasible
    multiplier, primal above dual minus the duality gap tolerance, gamma_eff between
    min and mean gamma."""
    gamma, _ = M.config_boolean_spheres_128(dtype=np.float32)
    out = gpu_run(gamma, [[1, 0, 0], [0, 1, 0], [0, 0, 1]], ccmf.Params(fixed_iters=200),
                  precision=ccmf.CCMF_FP32_MIXED, want=False)
    for r in out["res"]:
        assert r["status"] == 0 and r["iters"] == 200
        assert 0.3 <= r["gamma_eff"] <= float(gamma.mean()) + 1e-6
        assert np.isfinite(r["gamma_dual"])
    nv = np.sqrt(np.sum(out["v"].astype(np.float64) ** 2, axis=1))
    assert np.all(nv <= gamma[None].astype(np.float64) * (1 + 1e-6) + 1e-7)


def test_host_buffers_match_device_buffers():
    gamma = M.random_two_phase((10, 8, 12), 0.3, 0.25, 1.0, 31)
    p = ccmf.Params(fixed_iters=30)
    a = gpu_run(gamma, [[0.36, 0.48, 0.8]], p)
    b = gpu_run(gamma, [[0.36, 0.48, 0.8]], p, host=True)
    assert a["res"][0]["gamma_eff"] == b["res"][0]["gamma_eff"]
    np.testing.assert_array_equal(a["cut"], b["cut"])
    np.testing.assert_array_equal(a["flow"], b["flow"])


def test_resume_is_bit_identical_and_deterministic():
    gamma = M.random_two_phase((12, 12, 12), 0.3, 0.25, 1.0, 41)
    n = [[0.0, 0.6, 0.8]]
    full = gpu_run(gamma, n, ccmf.Params(fixed_iters=50))
    again = gpu_run(gamma, n, ccmf.Params(fixed_iters=50))
    np.testing.assert_array_equal(full["e"], again["e"])
    np.testing.assert_array_equal(full["v"], again["v"])
    half = gpu_run(gamma, n, ccmf.Params(fixed_iters=20))
    plan = half["plan"]
    plan.solve(torch.from_numpy(gamma).to(DEV), n, ccmf.Params(fixed_iters=30, resume=1))
    e, v, rho, iters = plan.state()
    np.testing.assert_array_equal(e.cpu().numpy(), full["e"])
    np.testing.assert_array_equal(v.cpu().numpy(), full["v"])
    assert rho[0] == full["rho"][0] and iters[0] == 50
    # resume from an exported checkpoint loaded into a fresh plan
    fresh = ccmf.Plan(gamma.shape, batch=1, precision=ccmf.CCMF_FP64, device=DEV)
    fresh.load_state(torch.from_numpy(half["e"]), torch.from_numpy(half["v"]), half["rho"], half["iters"])
    fresh.solve(torch.from_numpy(gamma).to(DEV), n, ccmf.Params(fixed_iters=30, resume=1))
    e2, v2, _, _ = fresh.state()
    np.testing.assert_array_equal(e2.cpu().numpy(), full["e"])


def test_history_matches_oracle():
    gamma = M.random_two_phase((8, 10, 6), 0.3, 0.25, 1.0, 51)
    out = gpu_run(gamma, [[1, 0, 0]], ccmf.Params(fixed_iters=40), want=False)
    ref = O.solve(gamma, [1, 0, 0], O.Params(fixed_iters=40))
    h = out["plan"].history()[0]
    assert h.shape == (40, 6)
    hr = np.array(ref.history)
    np.testing.assert_array_equal(h[:, 0], hr[:, 0])
    np.testing.assert_allclose(h[:, 1], hr[:, 1], rtol=1e-10)
    np.testing.assert_allclose(h[:, 2], hr[:, 2], rtol=1e-8, atol=1e-13)
    np.testing.assert_allclose(h[:, 4], hr[:, 4], rtol=1e-10)
    np.testing.assert_allclose(h[:, 5], hr[:, 5], rtol=1e-10, atol=1e-14)


def test_invalid_gamma_reported_per_solve():
    gamma = np.stack([M.uniform_random((6, 6, 6), 0.5, 1.0, 61) for _ in range(3)])
    gamma[1, 2, 3, 4] = -1.0
    gamma[2, 0, 0, 0] = np.nan
    out = gpu_run(gamma, [[1, 0, 0]] * 3, ccmf.Params(fixed_iters=10), want=False)
    st = [r["status"] for r in out["res"]]
    assert st == [0, ccmf.CCMF_ERR_NUMERICAL, ccmf.CCMF_ERR_NUMERICAL]
    assert out["res"][0]["iters"] == 10
    zero = gpu_run(np.zeros((4, 4, 4)), [[1, 0, 0]], ccmf.Params(fixed_iters=5), want=False)
    assert zero["res"][0]["status"] == ccmf.CCMF_ERR_INVALID_ARG


def test_pores_gamma_zero_phase():
    """gamma = 0 voxels (pores, Sec. 4.5): rho^0 falls back to mean(gamma); parity holds."""
    gamma = M.random_two_phase((10, 10, 10), 0.2, 0.0, 1.0, 71)
    out = gpu_run(gamma, [[1, 0, 0]], ccmf.Params(fixed_iters=40))
    ref = O.solve(gamma, [1, 0, 0], O.Params(fixed_iters=40), record_history=False)
    assert_parity(out, [ref])


@pytest.mark.parametrize("shape", [(1024, 2, 4), (4, 1024, 2), (2, 4, 1024), (1, 1, 1)])
def test_max_and_degenerate_axis_lengths(shape):
    # one voxel: the BB ratio is a quotient of rounding noise, so the constant rule is used
    rule = O.RHO_CONST if shape == (1, 1, 1) else O.RHO_BB
    gamma = M.uniform_random(shape, 0.5, 1.5, 81)
    out = gpu_run(gamma, [[0.36, 0.48, 0.8]], ccmf.Params(fixed_iters=15, rho_rule=rule))
    ref = O.solve(gamma, [0.36, 0.48, 0.8], O.Params(fixed_iters=15, rho_rule=rule), record_history=False)
    assert_parity(out, [ref])


def test_bad_arguments_return_codes():
    plan = ccmf.Plan((4, 4, 4), batch=1, precision=ccmf.CCMF_FP64, device=DEV)
    g = torch.ones((4, 4, 4), dtype=torch.float64, device=DEV)
    for normal, params in ([[0, 0, 0]], ccmf.Params()), ([[np.nan, 0, 1]], ccmf.Params()), \
            ([[1, 0, 0]], ccmf.Params(tol=0.0)), ([[1, 0, 0]], ccmf.Params(delta=1.0)), \
            ([[1, 0, 0]], ccmf.Params(rho_rule=9)):
        with pytest.raises(ccmf.CCMFError) as ei:
            plan.solve(g, normal, params)
        assert ei.value.code == ccmf.CCMF_ERR_INVALID_ARG
    res = (ccmf.ccmf_result * 1)()
    code = ccmf.ccmf_solve(plan.handle, g.data_ptr(), 0, np.array([1.0, 0, 0]), ccmf.Params().to_c(),
                           plan.ws_ptr, plan.workspace_bytes - 1024, None, None, res, None)
    assert code == ccmf.CCMF_ERR_WORKSPACE


def test_kernel_timing_mode():
    gamma, _ = M.boolean_spheres((32, 32, 32), 3.0, 0.2, 0.3, 1.0, 91)
    plan = ccmf.Plan(gamma.shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    plan.set_kernel_timing(True)
    g = torch.from_numpy(gamma.astype(np.float32)).to(DEV)
    res, _, _ = plan.solve(g, [[0, 0, 1]], ccmf.Params(fixed_iters=10))
    t = plan.kernel_times()
    launched = {name for name, (ms, n) in t.items() if n > 0}
    fused = {"k_div_rfft_z", "k_fft_plane", "k_irfft_z", "k_update"}
    split = {"k_div_rfft_z", "k_fft_y_fwd", "k_fft_x_solve", "k_fft_y_inv", "k_irfft_z", "k_update"}
    assert launched in (fused, split)
    for name in launched:
        ms, n = t[name]
        assert n == 10 and ms > 0.0
    plan.set_kernel_timing(False)
    res2, _, _ = plan.solve(g, [[0, 0, 1]], ccmf.Params(fixed_iters=10))
    assert res2[0]["gamma_eff"] == res[0]["gamma_eff"]


@pytest.mark.parametrize("variant", [1, 3], ids=["tma_rows", "tma_pipe"])
def test_device_wait_timeout_reported(variant, monkeypatch):
    """A bounded device wait that gives up is reported, not hung or faulted: with a zero-poll
    budget (debug setting) the TMA-staged update passes give up on their first tile, drain
    their copies in flight with the full budget, and the solve returns CCMF_ERR_TIMEOUT.
    The next solve on the same plan, with the normal budget, is healthy."""
    gamma = M.random_two_phase((64, 64, 64), 0.3, 0.25, 1.0, 71).astype(np.float32)
    plan = ccmf.Plan(gamma.shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    plan.set_tuning(update_variant=variant)
    g = torch.from_numpy(gamma).to(DEV)
    monkeypatch.setenv("CCMF_DEBUG_SPIN_LIMIT", "0")
    res, _, _ = plan.solve(g, [[0, 0, 1]], ccmf.Params(fixed_iters=3))
    assert res[0]["status"] == ccmf.CCMF_ERR_TIMEOUT
    monkeypatch.delenv("CCMF_DEBUG_SPIN_LIMIT")
    res, _, _ = plan.solve(g, [[0, 0, 1]], ccmf.Params(fixed_iters=3))
    assert res[0]["status"] == 0 and res[0]["iters"] == 3 and np.isfinite(res[0]["gamma_eff"])
    plan.close()

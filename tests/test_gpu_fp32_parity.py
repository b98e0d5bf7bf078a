"""FP32-mixed GPU path against the FP64 oracle at full size.

One step from an imported state (Eq. 30): the FP32 GPU state after some iterations is
exported, widened to FP64 and stepped once by the oracle; the next FP32 GPU step must
match it element by element. Bar: the FP32 step rounds w, d, the FFT pair of the Poisson
solve and the projection (relative errors of a few eps32 log2 N ~ 1e-6 of the largest
term, mostly the potential's forward difference), and P_C is 1-Lipschitz; e^{k+1} and
v^{k+1} are held to 1e-5 of the largest of max|e^{k+1}|, max|v^{k+1}| (FIELD_REL), rho^{k+1}
to 1e-4 relative, gamma_eff to 1e-5 relative (the FP32-mixed bar of the other tests).
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
FIELD_REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def one_step_against_oracle(gamma, normals, plan, warm, check):
    """Run `warm` FP32 iterations, export the state, run one more GPU step and compare the
    solves listed in `check` with one oracle step from the exported state."""
    g = torch.from_numpy(gamma.astype(np.float32)).to(DEV)
    plan.solve(g, normals, ccmf.Params(fixed_iters=warm))
    e0, v0, rho0, it0 = plan.state()
    res, flow, _ = plan.solve(g, normals, ccmf.Params(fixed_iters=1, resume=1), want_flow=True)
    e1, v1, rho1, it1 = plan.state()
    assert all(i == warm + 1 for i in it1)
    g64 = gamma.astype(np.float64)
    worst = []
    for s in check:
        e0s = e0[s].cpu().numpy().astype(np.float64)
        v0s = v0[s].cpu().numpy().astype(np.float64)
        xi = np.asarray(normals[s], dtype=np.float64)
        xi = xi / np.linalg.norm(xi)
        _, e_ref, v_ref = O.admm_step(e0s, v0s, rho0[s], g64, xi, 0.25)
        scale = max(np.abs(e_ref).max(), np.abs(v_ref).max())
        de = np.abs(e1[s].cpu().numpy().astype(np.float64) - e_ref).max()
        dv = np.abs(v1[s].cpu().numpy().astype(np.float64) - v_ref).max()
        assert de <= FIELD_REL * scale, (s, de, scale)
        assert dv <= FIELD_REL * scale, (s, dv, scale)
        rho_ref = O.next_rho(rho0[s], O.RHO_BB, e0s, e_ref, v0s, v_ref, O.Params())
        assert abs(rho1[s] - rho_ref) <= 1e-4 * rho_ref
        ev = O.evaluate(g64, xi, e_ref, v_ref, rho_ref)
        assert abs(res[s]["gamma_eff"] - ev.gamma_eff) <= 1e-5 * abs(ev.gamma_eff)
        fl = flow[s].cpu().numpy().astype(np.float64)
        assert np.abs(fl - ev.flow).max() <= FIELD_REL * max(1.0, np.abs(ev.flow).max())
        worst.append((de / scale, dv / scale))
    return worst


def test_fp32_full_size_one_step_from_imported_state():
    """128^3 Boolean spheres x 3 normals in the benchmark's launch shape (built-in rules):
    one FP32 step after 40 iterations against one oracle step (two of the normals)."""
    gamma, _ = M.config_boolean_spheres_128(dtype=np.float64)
    normals = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    plan = ccmf.Plan(gamma.shape, batch=3, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    worst = one_step_against_oracle(gamma, normals, plan, 40, (0, 2))
    plan.close()
    print("128^3 x 3 FP32 one-step relative max errors (e, v):", worst)


def test_fp32_fibre_corner_block_one_step_512_tuning():
    """512 x 512 x 128 corner block of the 512^3 short-fibre field (its own periodic cell),
    FP32 in the launch shape the 512^3 tuning picks: one warp per line for the y / x passes
    (line length 512), both z passes one warp per line pair, register-vector update."""
    full, _ = M.config_short_fibres_512(dtype=np.float32)
    gamma = np.ascontiguousarray(full[:, :, :128]).astype(np.float64)
    del full
    plan = ccmf.Plan(gamma.shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    plan.set_tuning(update_variant=0, plane_blocks=0, line_engine=1, z_engine=2)
    t = plan.tuning()
    assert t["line_engine"] == 1 and t["z_engine"] == 2 and t["plane_blocks"] == 0
    worst = one_step_against_oracle(gamma, [[0, 0, 1]], plan, 30, (0,))
    plan.close()
    print("512x512x128 FP32 one-step relative max errors (e, v):", worst)


def test_fp32_x_lines_512_three_normals():
    """FP32 x passes of length 512 (in FP32 the 512-point transforms of the x pass run in
    registers with one shared-memory exchange each) on a 512 x 24 x 16 two-phase cell with
    three normals, strided line passes: one step after 20 iterations against the oracle."""
    gamma = M.random_two_phase((512, 24, 16), 0.3, 0.25, 1.0, 29)
    normals = [[1, 0, 0], [0.36, 0.48, 0.8], [0, 0, 1]]
    plan = ccmf.Plan(gamma.shape, batch=3, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    plan.set_tuning(plane_blocks=0, line_engine=1)
    assert plan.tuning()["plane_blocks"] == 0 and plan.tuning()["line_engine"] == 1
    worst = one_step_against_oracle(gamma, normals, plan, 20, (0, 1, 2))
    plan.close()
    print("512x24x16 FP32 one-step relative max errors (e, v):", worst)


def test_fp32_x_lines_512_tma_tiles():
    """The x pass with its 8-line tiles moved by TMA (line engine 2: cp.async.bulk.tensor into a
    64-byte swizzled buffer and back) does the same arithmetic as the warp engine's copy loop
    (line engine 1): states bit-identical after 20 iterations on the 512 x 24 x 16 cell with
    three normals in three graph branches, and one step against the oracle."""
    gamma = M.random_two_phase((512, 24, 16), 0.3, 0.25, 1.0, 29)
    normals = [[1, 0, 0], [0.36, 0.48, 0.8], [0, 0, 1]]
    g = torch.from_numpy(gamma.astype(np.float32)).to(DEV)
    states = []
    for le in (1, 2):
        plan = ccmf.Plan(gamma.shape, batch=3, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
        plan.set_tuning(plane_blocks=0, line_engine=le, branches=3)
        assert plan.tuning()["line_engine"] == le
        res, _, _ = plan.solve(g, normals, ccmf.Params(fixed_iters=20))
        e, v, rho, _ = plan.state()
        states.append((e.cpu().numpy(), v.cpu().numpy(), list(rho), [r["gamma_eff"] for r in res]))
        plan.close()
    (e1, v1, r1, g1), (e2, v2, r2, g2) = states
    assert np.array_equal(e1, e2) and np.array_equal(v1, v2) and r1 == r2 and g1 == g2
    plan = ccmf.Plan(gamma.shape, batch=3, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    plan.set_tuning(plane_blocks=0, line_engine=2)
    worst = one_step_against_oracle(gamma, normals, plan, 20, (0, 1, 2))
    plan.close()
    print("512x24x16 FP32 TMA x tiles, one-step relative max errors (e, v):", worst)


def test_fp32_fibre_block_tma_x_tiles_equal_warp_engine():
    """512 x 512 x 64 corner block of the 512^3 fibre field in the 512^3 launch shape: the TMA
    x pass leaves the state bit-identical to the warp engine's after 6 iterations."""
    full, _ = M.config_short_fibres_512(dtype=np.float32)
    gamma = np.ascontiguousarray(full[:, :, :64])
    del full
    g = torch.from_numpy(gamma).to(DEV)
    out = []
    for le in (1, 2):
        plan = ccmf.Plan(gamma.shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
        plan.set_tuning(update_variant=11, plane_blocks=0, line_engine=le, z_engine=1)
        res, _, _ = plan.solve(g, [[0, 0, 1]], ccmf.Params(fixed_iters=6))
        e, v, rho, _ = plan.state()
        out.append((e.cpu().numpy(), v.cpu().numpy(), rho[0], res[0]["gamma_eff"]))
        plan.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3]


def test_tma_x_tiles_wait_timeout_reported(monkeypatch):
    """The TMA x pass's bounded mbarrier wait: with the zero-poll debug budget it gives up,
    drains its loads in flight, and the solve reports CCMF_ERR_TIMEOUT; the next call is healthy."""
    gamma = M.random_two_phase((512, 16, 8), 0.3, 0.25, 1.0, 31)
    g = torch.from_numpy(gamma.astype(np.float32)).to(DEV)
    plan = ccmf.Plan(gamma.shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    plan.set_tuning(plane_blocks=0, line_engine=2, update_variant=0)
    monkeypatch.setenv("CCMF_DEBUG_SPIN_LIMIT", "0")
    res, _, _ = plan.solve(g, [[0, 0, 1]], ccmf.Params(fixed_iters=3))
    assert res[0]["status"] == ccmf.CCMF_ERR_TIMEOUT
    monkeypatch.delenv("CCMF_DEBUG_SPIN_LIMIT")
    res, _, _ = plan.solve(g, [[0, 0, 1]], ccmf.Params(fixed_iters=3))
    assert res[0]["status"] == 0 and res[0]["iters"] == 3 and np.isfinite(res[0]["gamma_eff"])
    plan.close()


def test_tma_x_tiles_rejected_where_not_applicable():
    """Line engine 2 needs FP32, N1 = 512 and N2 a multiple of 8."""
    for shape, prec in (((512, 12, 8), ccmf.CCMF_FP32_MIXED), ((256, 16, 8), ccmf.CCMF_FP32_MIXED),
                        ((512, 16, 8), ccmf.CCMF_FP64)):
        plan = ccmf.Plan(shape, batch=1, precision=prec, device=DEV)
        with pytest.raises(ccmf.CCMFError) as ei:
            plan.set_tuning(plane_blocks=0, line_engine=2)
        assert ei.value.code == ccmf.CCMF_ERR_UNSUPPORTED_SIZE
        plan.close()


def _one_weakest_layer():
    layers = np.array([1.0, 0.9, 1.2, 0.6, 1.1, 0.7, 1.4, 0.8] * 8)
    layers[37] = 0.4
    return layers


def _rel_l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / max(np.sum(b ** 2), 1e-300)))


def test_fp32_converged_fields_against_fp64():
    """Error of the FP32-mixed solution against the FP64 GPU solution at equal iteration
    counts after convergence: gamma_eff (the max-flow value) within 1e-5, and the cut
    xi^{K+1/2} and flow A* v^K fields reported as max-abs and relative L2 errors.

    Two cells: the 128^3 Boolean workload (normal e3) and a 64^3 laminate whose layer 37 is
    the only weakest one (gamma 0.4 against 0.6 ... 1.4 in the others), normal e3, where
    the min cut is unique (the weakest layer: a laminate normal to its layers has
    gamma_eff = min gamma): there the cut field must agree to 1e-3 relative L2."""
    cases = {
        "boolean128_e3": (M.config_boolean_spheres_128(dtype=np.float64)[0], 1e-7, 6000),
        "laminate64_e3": (np.ascontiguousarray(M.laminate(64, 64, _one_weakest_layer())), 1e-8, 20000),
    }
    report = {}
    for name, (gamma, tol, max_iter) in cases.items():
        g64 = torch.from_numpy(gamma).to(DEV)
        p64 = ccmf.Plan(gamma.shape, batch=1, precision=ccmf.CCMF_FP64, device=DEV)
        r64, f64, c64 = p64.solve(g64, [[0, 0, 1]], ccmf.Params(tol=tol, max_iter=max_iter), want_flow=True,
                                  want_cut=True)
        p64.close()
        K = int(r64[0]["iters"])
        g32 = torch.from_numpy(gamma.astype(np.float32)).to(DEV)
        p32 = ccmf.Plan(gamma.shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
        r32, f32, c32 = p32.solve(g32, [[0, 0, 1]], ccmf.Params(fixed_iters=K), want_flow=True, want_cut=True)
        p32.close()
        c64n, c32n = c64[0].cpu().numpy(), c32[0].cpu().numpy().astype(np.float64)
        f64n, f32n = f64[0].cpu().numpy(), f32[0].cpu().numpy().astype(np.float64)
        geff_err = abs(r32[0]["gamma_eff"] - r64[0]["gamma_eff"]) / abs(r64[0]["gamma_eff"])
        report[name] = dict(iters=K, fp64_converged=int(r64[0]["converged"]),
                            fp64_gap_rel=(r64[0]["gamma_primal"] - r64[0]["gamma_dual"]) / r64[0]["gamma_dual"],
                            gamma_eff_rel=geff_err,
                            cut_maxabs=float(np.abs(c32n - c64n).max()), cut_max=float(np.abs(c64n).max()),
                            cut_rel_l2=_rel_l2(c32n, c64n),
                            flow_maxabs=float(np.abs(f32n - f64n).max()), flow_rel_l2=_rel_l2(f32n, f64n))
        assert geff_err <= 1e-5, report[name]
    print("FP32-mixed vs FP64 converged fields:", report)
    lam = report["laminate64_e3"]
    assert lam["fp64_converged"] == 1
    assert lam["cut_rel_l2"] <= 1e-3, lam

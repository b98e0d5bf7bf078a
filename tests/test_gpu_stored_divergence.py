"""The stored-divergence schedule (update variants 8, 9, 10 and 13 .. 15) against the oracle.

The update pass writes a = div^- A* e and b = div^- A* v of the state it produces, and
the first pass of the next iteration forms d = a - b / rho from them (Eq. 28, Eq. 30:
d is linear in the state). It changes only where the divergence is computed, so FP64
results must match the oracle at equal iteration counts with the bars of the other
parity tests (|d gamma_eff| / gamma_eff <= 1e-10, fields <= 1e-9). The cases cover one
and several z passes per row, y tiles with a ragged last tile, x segments with a
ragged last segment, grids narrower than a tile, resume (stored divergences kept) and
an imported state (stored divergences recomputed)."""

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

CASES = [
    # (shape, normals): FP64 variants 8 and 13 .. 15 run 64-voxel z passes, variant 9 32-voxel passes
    ((40, 24, 64), [[1, 0, 0], [0.36, 0.48, 0.8]]),
    ((20, 15, 128), [[0, 0, 1]]),
    ((9, 5, 256), [[0.6, 0.0, 0.8]]),
    ((3, 2, 64), [[0, 1, 0]]),
    ((1, 1, 64), [[0, 0, 1]]),
    ((9, 30, 32), [[0.0, 0.6, 0.8]]),
]


def _solve(gamma, normals, variant, params, precision=ccmf.CCMF_FP64):
    plan = ccmf.Plan(gamma.shape, batch=len(normals), precision=precision, device=DEV)
    plan.set_tuning(update_variant=variant)
    assert plan.tuning()["update_variant"] == variant
    dt = np.float64 if precision == ccmf.CCMF_FP64 else np.float32
    g = torch.from_numpy(gamma.astype(dt)).to(DEV)
    res, flow, cut = plan.solve(g, normals, params, want_flow=True, want_cut=True)
    e, v, rho, iters = plan.state()
    return plan, g, res, flow, cut, e, v, rho, iters


@pytest.mark.parametrize("variant", [8, 9, 10, 13, 14, 15])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_fp64_stored_divergence_matches_oracle(variant, case):
    shape, normals = CASES[case]
    if variant in (8, 13, 14, 15) and shape[2] % 64:
        pytest.skip("variants 8 and 13 .. 15 need N3 % 64 == 0 in FP64")
    gamma = M.boolean_spheres(shape, 2.5, 0.2, 0.3, 1.0, seed=31 + case)[0]
    plan, g, res, flow, cut, e, v, rho, iters = _solve(gamma, normals, variant, ccmf.Params(fixed_iters=25))
    for s, n in enumerate(normals):
        ref = O.solve(gamma, n, O.Params(fixed_iters=25), record_history=False)
        assert res[s]["status"] == 0 and res[s]["iters"] == 25
        assert abs(res[s]["gamma_eff"] - ref.gamma_eff) <= 1e-10 * abs(ref.gamma_eff)
        assert abs(rho[s] - ref.rho) <= 1e-10 * ref.rho
        np.testing.assert_allclose(e[s].cpu().numpy(), ref.e, rtol=0, atol=1e-9)
        np.testing.assert_allclose(v[s].cpu().numpy(), ref.v, rtol=0, atol=1e-9)
        np.testing.assert_allclose(cut[s].cpu().numpy(), ref.cut, rtol=0, atol=1e-9)
        np.testing.assert_allclose(flow[s].cpu().numpy(), ref.flow, rtol=0, atol=1e-9)
    plan.close()


@pytest.mark.parametrize("variant", [8, 9, 10, 13, 14, 15])
def test_stored_divergence_resume_and_import(variant):
    """Resume continues from the stored divergences bit for bit; an imported state gets its
    divergences recomputed and continues within rounding of the uninterrupted run."""
    gamma = M.boolean_spheres((12, 15, 64), 2.5, 0.2, 0.3, 1.0, seed=41)[0]
    n = [[0.0, 0.6, 0.8]]
    full = _solve(gamma, n, variant, ccmf.Params(fixed_iters=30))
    half = _solve(gamma, n, variant, ccmf.Params(fixed_iters=12))
    plan, g = half[0], half[1]
    plan.solve(g, n, ccmf.Params(fixed_iters=18, resume=1))
    e, v, rho, iters = plan.state()
    np.testing.assert_array_equal(e.cpu().numpy(), full[5].cpu().numpy())
    np.testing.assert_array_equal(v.cpu().numpy(), full[6].cpu().numpy())
    fresh = ccmf.Plan(gamma.shape, batch=1, precision=ccmf.CCMF_FP64, device=DEV)
    fresh.set_tuning(update_variant=variant)
    fresh.load_state(half[5], half[6], half[7], half[8])
    fresh.solve(g, n, ccmf.Params(fixed_iters=18, resume=1))
    e2, v2, _, it2 = fresh.state()
    assert it2[0] == 30
    np.testing.assert_allclose(e2.cpu().numpy(), full[5].cpu().numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(v2.cpu().numpy(), full[6].cpu().numpy(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("variant", [8, 9, 10, 13, 14, 15])
def test_fp32_stored_divergence_against_default_schedule(variant):
    """FP32-mixed 128^3 Boolean workload x 3 normals: the stored-divergence schedule against
    the default update at equal iterations (gamma_eff within 1e-5, fields within FP32
    noise), and one step from an imported state against the oracle."""
    gamma, _ = M.config_boolean_spheres_128(dtype=np.float64)
    normals = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    p = ccmf.Params(fixed_iters=60)
    a = _solve(gamma, normals, 0, p, precision=ccmf.CCMF_FP32_MIXED)
    b = _solve(gamma, normals, variant, p, precision=ccmf.CCMF_FP32_MIXED)
    for s in range(3):
        assert abs(a[2][s]["gamma_eff"] - b[2][s]["gamma_eff"]) <= 1e-5 * abs(a[2][s]["gamma_eff"])
    scale = float(torch.max(torch.abs(a[5])).item())
    assert float(torch.max(torch.abs(a[5] - b[5])).item()) <= 1e-4 * scale
    # one further step of the stored-divergence plan against one oracle step
    plan, g = b[0], b[1]
    e0, v0, rho0, _ = plan.state()
    plan.solve(g, normals, ccmf.Params(fixed_iters=1, resume=1))
    e1, v1, _, _ = plan.state()
    xi = np.array([0.0, 0.0, 1.0])
    _, e_ref, v_ref = O.admm_step(e0[2].cpu().numpy().astype(np.float64), v0[2].cpu().numpy().astype(np.float64),
                                  rho0[2], gamma, xi, 0.25)
    sc = max(np.abs(e_ref).max(), np.abs(v_ref).max())
    assert np.abs(e1[2].cpu().numpy() - e_ref).max() <= 1e-5 * sc
    assert np.abs(v1[2].cpu().numpy() - v_ref).max() <= 1e-5 * sc


@pytest.mark.parametrize("variant", [8, 9, 10, 13, 14, 15])
def test_fp32_stored_divergence_warp_z_passes(variant):
    """The first pass as one warp per line pair (z engine 2) reading the stored divergences,
    N3 = 128 and 256: FP32 against the default update pass with the same FFT passes over
    several iterations (gamma_eff within 1e-5, state within FP32 noise)."""
    for shape in ((48, 40, 128), (30, 24, 256)):
        gamma = M.boolean_spheres(shape, 3.0, 0.2, 0.3, 1.0, seed=43)[0]
        out = []
        for var in (0, variant):
            plan = ccmf.Plan(shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
            plan.set_tuning(update_variant=var, z_engine=2, line_engine=0, plane_blocks=0)
            res, _, _ = plan.solve(torch.from_numpy(gamma.astype(np.float32)).to(DEV), [[0, 0, 1]],
                                   ccmf.Params(fixed_iters=20))
            e, _, _, _ = plan.state()
            out.append((res[0]["gamma_eff"], e[0].cpu().numpy()))
            plan.close()
        assert np.isfinite(out[1][0])
        assert abs(out[1][0] - out[0][0]) <= 1e-5 * abs(out[0][0])
        assert np.abs(out[1][1] - out[0][1]).max() <= 1e-4 * np.abs(out[0][1]).max()


def test_stored_divergence_unavailable_grids_are_rejected():
    plan = ccmf.Plan((16, 16, 48), batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    for bad in (8, 9, 10, 13, 14, 16):   # N3 = 48 is not a multiple of 128 / 64; 16 is no variant
        with pytest.raises(ccmf.CCMFError) as err:
            plan.set_tuning(update_variant=bad)
        assert err.value.code == ccmf.CCMF_ERR_UNSUPPORTED_SIZE
    plan.close()

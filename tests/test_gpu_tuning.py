"""The tuning knobs and the autotuner (ccmf_plan_set_tuning / ccmf_plan_autotune).

Every knob changes only how the Eq. 30 step is launched (update-pass variant,
plane pass on one block, a cluster or strided passes, lines per block, graph
branches, radix schedule), so FP64 results under any tuning must match the
oracle at equal iteration counts with the parity bars of the other tests."""

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


TUNINGS = [
    dict(update_variant=0, plane_blocks=0, y_lines_per_block=2, x_lines_per_block=16),
    dict(update_variant=1, plane_blocks=1, z_pairs_per_block=1, radix_mode=1),
    dict(update_variant=3, plane_blocks=2, z_pairs_per_block=4, radix_mode=2, branches=1),
    dict(update_variant=7, plane_blocks=4, branches=3, radix_mode=1),
    dict(update_variant=5, plane_blocks=0, y_lines_per_block=16, x_lines_per_block=1, radix_mode=2, branches=2),
    dict(update_variant=11, plane_blocks=1, branches=3),
    dict(update_variant=12, plane_blocks=0, branches=1),
    dict(update_variant=9, plane_blocks=0, branches=2),
]


@pytest.mark.parametrize("knobs", TUNINGS, ids=[f"t{i}" for i in range(len(TUNINGS))])
def test_fp64_parity_under_tuning(knobs):
    gamma = M.boolean_spheres((40, 24, 32), 3.0, 0.2, 0.3, 1.0, seed=17)[0]
    normals = [[1, 0, 0], [0.36, 0.48, 0.8], [0, 0, 1]]
    plan = ccmf.Plan(gamma.shape, batch=3, precision=ccmf.CCMF_FP64, device=DEV)
    plan.set_tuning(**knobs)
    t = plan.tuning()
    for k, v in knobs.items():
        assert t[k] == v
    assert min(t.values()) >= 0
    res, flow, cut = plan.solve(torch.from_numpy(gamma).to(DEV), normals, ccmf.Params(fixed_iters=25),
                                want_flow=True, want_cut=True)
    e, v, rho, _ = plan.state()
    for s, n in enumerate(normals):
        ref = O.solve(gamma, n, O.Params(fixed_iters=25), record_history=False)
        assert abs(res[s]["gamma_eff"] - ref.gamma_eff) <= 1e-10 * ref.gamma_eff
        np.testing.assert_allclose(e[s].cpu().numpy(), ref.e, rtol=0, atol=1e-9)
        np.testing.assert_allclose(v[s].cpu().numpy(), ref.v, rtol=0, atol=1e-9)
        np.testing.assert_allclose(cut[s].cpu().numpy(), ref.cut, rtol=0, atol=1e-9)
    plan.close()


def test_infeasible_tuning_is_rejected_and_kept():
    plan = ccmf.Plan((40, 24, 12), batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    before = plan.tuning()
    for bad in (dict(plane_blocks=16), dict(plane_blocks=3), dict(z_pairs_per_block=3), dict(update_variant=9),
                dict(update_variant=13), dict(update_variant=16),
                dict(branches=5), dict(radix_mode=7)):
        with pytest.raises(ccmf.CCMFError) as err:
            plan.set_tuning(**bad)
        assert err.value.code == ccmf.CCMF_ERR_UNSUPPORTED_SIZE
        assert plan.tuning() == before
    plan.close()


def test_autotune_keeps_the_fastest_and_records_it():
    gamma = M.boolean_spheres((64, 64, 64), 4.0, 0.2, 0.3, 1.0, seed=23)[0].astype(np.float32)
    normals = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    g = torch.from_numpy(gamma).to(DEV)
    plan = ccmf.Plan(gamma.shape, batch=3, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    plan.solve(g, normals, ccmf.Params(fixed_iters=5))
    best, ms = plan.autotune(g, normals, iters=5)
    assert ms > 0 and best == plan.tuning()
    # the tuning table now holds this key: a new plan of the same key starts from it
    again = ccmf.Plan(gamma.shape, batch=3, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    assert again.tuning() == best
    code, text = ccmf.ccmf_tuning_export()
    assert code == ccmf.CCMF_OK
    line = [x for x in text.splitlines() if x.startswith("ccmf-tuning 64 64 64 3 1 ")]
    assert len(line) == 1
    # the tuned plan still solves: state after 5 + autotuning updates stays feasible and finite
    res, _, _ = again.solve(g, normals, ccmf.Params(fixed_iters=20))
    for r in res:
        assert r["status"] == 0 and np.isfinite(r["gamma_eff"])
    plan.close()
    again.close()


@pytest.mark.parametrize("shape", [(128, 256, 4), (128, 96, 6), (96, 128, 6), (512, 64, 4), (64, 512, 4)],
                         ids=["warp_xy", "warp_x_generic_y", "generic_x_warp_y", "x_512", "y_512"])
@pytest.mark.parametrize("engine", [1, 0], ids=["warp_lines", "block_lines"])
def test_fp64_line_passes_against_oracle(shape, engine):
    """Strided y / x passes with one warp per power-of-two line (natural order) or in-place
    block stages (digit-reversed order), alone and mixed per axis: FP64 parity with the oracle."""
    gamma = M.random_two_phase(shape, 0.3, 0.25, 1.0, 13)
    normals = [[0.36, 0.48, 0.8]]
    plan = ccmf.Plan(shape, batch=1, precision=ccmf.CCMF_FP64, device=DEV)
    plan.set_tuning(plane_blocks=0, line_engine=engine)
    assert plan.tuning()["line_engine"] == engine and plan.launch_info()["plane_fused"] == 0
    res, flow, cut = plan.solve(torch.from_numpy(gamma).to(DEV), normals, ccmf.Params(fixed_iters=20),
                                want_flow=True, want_cut=True)
    e, v, rho, _ = plan.state()
    ref = O.solve(gamma, normals[0], O.Params(fixed_iters=20), record_history=False)
    assert abs(res[0]["gamma_eff"] - ref.gamma_eff) <= 1e-10 * ref.gamma_eff
    np.testing.assert_allclose(e[0].cpu().numpy(), ref.e, rtol=0, atol=1e-9)
    np.testing.assert_allclose(v[0].cpu().numpy(), ref.v, rtol=0, atol=1e-9)
    np.testing.assert_allclose(cut[0].cpu().numpy(), ref.cut, rtol=0, atol=1e-9)
    plan.close()


def test_plans_of_different_sizes_coexist():
    """A kernel's dynamic shared memory limit is shared by every plan in the process: a plan
    with smaller tiles created after a larger one must not break the larger plan's launches
    (128^2 planes need 132 KB per block in FP32, 96^2 planes 74 KB)."""
    big = ccmf.Plan((128, 128, 8), batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    small = ccmf.Plan((96, 96, 8), batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    assert big.launch_info()["plane_blocks"] == 1 and small.launch_info()["plane_blocks"] == 1
    for plan, shape in ((big, (128, 128, 8)), (small, (96, 96, 8)), (big, (128, 128, 8))):
        g = torch.from_numpy(M.random_two_phase(shape, 0.3, 0.25, 1.0, 5).astype(np.float32)).to(DEV)
        res, _, _ = plan.solve(g, [[0, 0, 1]], ccmf.Params(fixed_iters=5))
        assert res[0]["status"] == 0 and np.isfinite(res[0]["gamma_eff"])
    big.close()
    small.close()


@pytest.mark.parametrize("shape", [(6, 5, 128), (3, 4, 256), (5, 3, 512), (9, 18, 128)],
                         ids=["n3_128", "n3_256", "n3_512", "tiles_9x18"])
@pytest.mark.parametrize("engine", [2, 1, 0], ids=["warp_both", "warp_inverse", "block_z"])
def test_fp64_z_passes_against_oracle(shape, engine):
    """Divergence + R2C and C2R along z with one warp per line pair (power-of-two N3, line
    counts that leave a partial tile of 16 lines, several tiles with neighbour rows in other
    tiles) or Stockham tiles: FP64 parity with the oracle."""
    gamma = M.random_two_phase(shape, 0.3, 0.25, 1.0, 17)
    normals = [[0.36, 0.48, 0.8], [0.0, 0.0, 1.0]]
    plan = ccmf.Plan(shape, batch=2, precision=ccmf.CCMF_FP64, device=DEV)
    plan.set_tuning(z_engine=engine)
    assert plan.tuning()["z_engine"] == engine
    res, flow, cut = plan.solve(torch.from_numpy(gamma).to(DEV), normals, ccmf.Params(fixed_iters=20),
                                want_flow=True, want_cut=True)
    e, v, rho, _ = plan.state()
    for s, n in enumerate(normals):
        ref = O.solve(gamma, n, O.Params(fixed_iters=20), record_history=False)
        assert abs(res[s]["gamma_eff"] - ref.gamma_eff) <= 1e-10 * ref.gamma_eff
        np.testing.assert_allclose(e[s].cpu().numpy(), ref.e, rtol=0, atol=1e-9)
        np.testing.assert_allclose(v[s].cpu().numpy(), ref.v, rtol=0, atol=1e-9)
        np.testing.assert_allclose(flow[s].cpu().numpy(), ref.flow, rtol=0, atol=1e-9)
    plan.close()

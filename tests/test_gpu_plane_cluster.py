"""The plane pass on a thread-block cluster: C blocks share one (x, y) plane of the
half spectrum through distributed shared memory (forward y and x transforms, the
Poisson symbol of Eq. 28 and the inverse transforms). FP64 against the oracle at
equal iteration counts for every cluster size, on grids whose rows and columns per
block are powers of two, odd or radix 3 / 5; FP32-mixed on a 512 x 512 plane, the
plane of the 512^3 workload, against the FP64 oracle."""

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


def run(gamma, normals, params, precision, monkeypatch, cluster):
    monkeypatch.setenv("CCMF_PLANE_CLUSTER", str(cluster))
    plan = ccmf.Plan(gamma.shape, batch=len(normals), precision=precision, device=DEV)
    info = plan.launch_info()
    dt = np.float64 if precision == ccmf.CCMF_FP64 else np.float32
    g = torch.from_numpy(np.ascontiguousarray(gamma.astype(dt))).to(DEV)
    res, flow, cut = plan.solve(g, normals, params, want_flow=True, want_cut=True)
    e, v, rho, iters = plan.state()
    torch.cuda.synchronize()
    out = dict(res=res, flow=flow.cpu().numpy(), cut=cut.cpu().numpy(), e=e.cpu().numpy(), v=v.cpu().numpy(),
               rho=rho, info=info)
    plan.close()
    return out


CASES = [
    # (cluster size, grid, normals, iterations): rows R1 = n1 / C and columns R2 = n2 / C per block
    (2, (40, 24, 36), [[1, 0, 0], [0, 1, 0], [0, 0, 1]], 25),   # R1 20, R2 12
    (4, (40, 24, 12), [[0.36, 0.48, 0.8]], 30),                # R1 10, R2 6
    (8, (48, 40, 10), [[0.0, 0.6, -0.8]], 30),                 # R1 6, R2 5
    (16, (32, 48, 6), [[0.6, 0.0, 0.8]], 30),                  # R1 2, R2 3
    (2, (60, 30, 9), [[0.0, 0.0, 1.0]], 30),                   # R1 30, R2 15 (radix 3 / 5)
]


@pytest.mark.parametrize("cl,shape,normals,iters", CASES, ids=[f"C{c[0]}_{'x'.join(map(str, c[1]))}" for c in CASES])
def test_fp64_cluster_plane_equal_iterations(cl, shape, normals, iters, monkeypatch):
    gamma = M.boolean_spheres(shape, 3.0, 0.2, 0.3, 1.0, seed=cl + shape[0])[0]
    out = run(gamma, normals, ccmf.Params(fixed_iters=iters), ccmf.CCMF_FP64, monkeypatch, cl)
    assert out["info"]["plane_fused"] == 1 and out["info"]["plane_blocks"] == cl
    for s, n in enumerate(normals):
        ref = O.solve(gamma, n, O.Params(fixed_iters=iters), record_history=False)
        r = out["res"][s]
        assert r["status"] == 0 and r["iters"] == iters
        assert abs(r["gamma_eff"] - ref.gamma_eff) <= 1e-10 * abs(ref.gamma_eff)
        assert abs(out["rho"][s] - ref.rho) <= 1e-10 * ref.rho
        for key, val in (("e", ref.e), ("v", ref.v), ("cut", ref.cut), ("flow", ref.flow)):
            np.testing.assert_allclose(out[key][s], val, rtol=0, atol=1e-9)


def test_plane_pass_choice_rules(monkeypatch):
    """Built-in rule: one block per plane when the plane fits its shared memory, else the
    strided passes; clusters are chosen explicitly (tuning or CCMF_PLANE_CLUSTER) and are
    rejected where a block's share of the plane does not fit."""
    monkeypatch.delenv("CCMF_PLANE_CLUSTER", raising=False)
    cases = [((128, 128, 8), ccmf.CCMF_FP32_MIXED, 1), ((128, 128, 8), ccmf.CCMF_FP64, 0),
             ((160, 160, 4), ccmf.CCMF_FP32_MIXED, 0), ((512, 512, 4), ccmf.CCMF_FP32_MIXED, 0)]
    for shape, prec, want in cases:
        plan = ccmf.Plan(shape, batch=1, precision=prec, device=DEV)
        info = plan.launch_info()
        assert info["plane_blocks"] == want, (shape, prec, info)
        plan.close()
    ok = ccmf.Plan((512, 512, 4), batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    ok.set_tuning(plane_blocks=16)
    assert ok.launch_info()["plane_blocks"] == 16
    ok.close()
    bad = ccmf.Plan((512, 512, 4), batch=1, precision=ccmf.CCMF_FP64, device=DEV)
    with pytest.raises(ccmf.CCMFError):
        bad.set_tuning(plane_blocks=16)   # 16384 FP64 elements per block exceed its registers
    bad.close()


@pytest.mark.parametrize("blocks", [16, 0], ids=["cluster16", "line_passes"])
def test_fp32_plane_512_against_fp64_oracle(blocks, monkeypatch):
    """512 x 512 x 6 two-phase field (the 512^3 workload's plane) through a cluster of 16
    blocks and through the persistent line passes: FP32-mixed fields at equal iterations
    within FP32 accuracy of the FP64 oracle."""
    gamma = M.random_two_phase((512, 512, 6), 0.3, 0.25, 1.0, 77)
    normals = [[0.36, 0.48, 0.8]]
    out = run(gamma.astype(np.float32), normals, ccmf.Params(fixed_iters=8, rho_rule=ccmf.CCMF_RHO_CONST),
              ccmf.CCMF_FP32_MIXED, monkeypatch, blocks)
    assert out["info"]["plane_blocks"] == blocks
    ref = O.solve(gamma.astype(np.float32).astype(np.float64), normals[0],
                  O.Params(fixed_iters=8, rho_rule=O.RHO_CONST), record_history=False)
    scale = max(np.abs(ref.v).max(), np.abs(ref.e).max())
    assert np.abs(out["e"][0] - ref.e).max() <= 1e-4 * scale
    assert np.abs(out["v"][0] - ref.v).max() <= 1e-4 * scale
    assert abs(out["res"][0]["gamma_eff"] - ref.gamma_eff) <= 1e-5 * abs(ref.gamma_eff)

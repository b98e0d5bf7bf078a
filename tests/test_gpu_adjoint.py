"""GPU reverse mode (ccmf_adjoint, the torch.autograd.Function around it) against
the oracle gradient, central finite differences and the envelope derivative."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import ccmf_adjoint as D  # noqa: E402
from oracle import ccmf_oracle as O  # noqa: E402
from paper_2103_05968_gb300 import ccmf  # noqa: E402
from paper_2103_05968_gb300 import microstructure as M  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_grad(gamma, xi, K, m, precision=ccmf.CCMF_FP64, sched=None, params=None):
    dt = np.float64 if precision == ccmf.CCMF_FP64 else np.float32
    plan = ccmf.Plan(gamma.shape, batch=1, precision=precision, device=DEV)
    g = torch.from_numpy(gamma.astype(dt)).to(DEV)
    grad, res, rho = plan.gradient(g, [xi], K, m, params=params, rho_schedule=sched)
    torch.cuda.synchronize()
    out = grad[0].double().cpu().numpy(), res[0], rho[0]
    plan.close()
    return out


@pytest.mark.parametrize("shape,K,m", [((6, 5, 8), 25, 7), ((8, 8, 8), 30, 10), ((5, 9, 1), 20, 20)])
def test_fp64_gradient_matches_oracle(shape, K, m):
    g = M.uniform_random(shape, 0.5, 1.5, 11)
    xi = [0.36, 0.48, 0.8]
    p = ccmf.Params(rho0=0.9 * float(g.min()))   # start below the k = 0 kink of the projection
    grad, res, rho = gpu_grad(g, xi, K, m, params=p)
    J, ref = D.gradient(g, xi, list(rho))
    assert abs(res["gamma_eff"] - J) <= 1e-10 * abs(J)
    np.testing.assert_allclose(grad, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("shape,K,m", [((6, 5, 8), 25, 7), ((8, 8, 8), 30, 10)])
def test_fp32_reverse_with_fp64_forward_matches_oracle(shape, K, m):
    """FP32 plan, FP64 forward (ccmf_set_adjoint_forward): the replayed value is the FP64 one and
    the FP32 reverse sweep, following the FP64 projection branches, gives the oracle gradient to
    FP32 accuracy (1e-5 of its largest entry)."""
    g = M.uniform_random(shape, 0.5, 1.5, 11)
    xi = [0.36, 0.48, 0.8]
    p = ccmf.Params(rho0=0.9 * float(g.min()))
    plan = ccmf.Plan(g.shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    plan.set_adjoint_forward(ccmf.CCMF_FP64)
    grad, res, rho2 = plan.gradient(torch.from_numpy(g.astype(np.float32)).to(DEV), [xi], K, m, params=p)
    plan.close()
    # gamma was rounded to float: the FP64 forward sees float(gamma), compare with that map
    J32, ref32 = D.gradient(g.astype(np.float32).astype(np.float64), xi, list(rho2[0]))
    assert abs(res[0]["gamma_eff"] - J32) <= 1e-10 * abs(J32)
    np.testing.assert_allclose(grad[0].double().cpu().numpy(), ref32, rtol=0, atol=1e-5 * np.abs(ref32).max())


def test_fp64_gradient_matches_central_differences():
    # the replayed map is piecewise smooth (kinks of the projection at |z| = gamma): a step of 1e-7
    # keeps central differences off the kinks, larger steps straddle some of them
    g = M.random_two_phase((10, 8, 12), 0.3, 0.3, 1.0, 5)
    xi = [0.0, 0.6, 0.8]
    K, m = 40, 9
    grad, res, rho = gpu_grad(g, xi, K, m, params=ccmf.Params(rho0=0.25))
    rng = np.random.default_rng(3)
    for _ in range(3):
        eta = rng.standard_normal(g.shape)
        h = 1e-7
        jp = gpu_grad(g + h * eta, xi, K, m, sched=rho[None])[1]["gamma_eff"]
        jm = gpu_grad(g - h * eta, xi, K, m, sched=rho[None])[1]["gamma_eff"]
        fd = (jp - jm) / (2 * h)
        assert abs(fd - float(np.sum(grad * eta))) <= 1e-5 * max(abs(fd), 1e-3)


def test_envelope_gradient_at_convergence():
    g = M.single_sphere((16, 16, 16), (8.0, 8.0, 8.0), 4.0, 0.1, 1.0)
    ref = O.solve(g, [0, 0, 1], O.Params(tol=1e-7, max_iter=20000))
    grad, res, rho = gpu_grad(g, [0, 0, 1], ref.iters, 50)
    env = np.sqrt(np.sum(ref.cut ** 2, axis=0)) / g.size
    cos = float(np.sum(grad * env) / np.sqrt(np.sum(grad ** 2) * np.sum(env ** 2)))
    assert cos > 0.99


def test_config_lognormal_128_fp32_against_fp64_differences():
    """128^3 gamma = exp(0.5 g), g Gaussian with correlation length 8; d gamma_eff(e3) / d gamma through
    200 updates with checkpoints every 20, against central differences of the FP64 replayed map on three
    random directions.

    * FP64 reverse mode: <= 1e-4 relative at the step h = 1e-7 (off the projection kinks, reading R9).
    * FP32 plan with the FP64 forward (ccmf_set_adjoint_forward: FP64 forward and recompute, clip
      decisions kept as bits, FP32 reverse sweep): <= 1e-4 relative per direction at h = 1e-7, and within
      1e-4 of the FP64 gradient in relative L2.
    * FP32 plan with the FP32 forward: its trajectory takes the other branch of P_C at near-tied voxels,
      so it differentiates a neighbouring piece of the map; held to 3e-3.
    The config's own step h = 1e-4 straddles kinks of the projection; its differences are reported."""
    g = M.lognormal_field((128, 128, 128), 8.0, 0.5, seed=5)
    xi = [0.0, 0.0, 1.0]
    K, m = 200, 20
    g64, r64, rho = gpu_grad(g, xi, K, m, params=ccmf.Params(rho0=0.9 * float(g.min())))
    g32, r32, _ = gpu_grad(g, xi, K, m, precision=ccmf.CCMF_FP32_MIXED, sched=rho[None])
    plan = ccmf.Plan(g.shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=DEV)
    plan.set_adjoint_forward(ccmf.CCMF_FP64)
    gm_t, rm, _ = plan.gradient(torch.from_numpy(g.astype(np.float32)).to(DEV), [xi], K, m,
                                rho_schedule=rho[None])
    gmx = gm_t[0].double().cpu().numpy()
    plan.close()
    rel_l2_mixed = np.linalg.norm(gmx - g64) / np.linalg.norm(g64)
    rel_l2_fp32 = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    print(f"gradient rel L2 vs FP64: FP64 forward + FP32 reverse {rel_l2_mixed:.2e}, FP32 {rel_l2_fp32:.2e}")
    assert rel_l2_mixed <= 1e-4
    assert rel_l2_fp32 <= 3e-3
    assert abs(r32["gamma_eff"] - r64["gamma_eff"]) <= 1e-5 * r64["gamma_eff"]
    # the FP32 plan's gamma is float(gamma): its FP64 forward differs by the rounding of gamma only
    assert abs(rm[0]["gamma_eff"] - r64["gamma_eff"]) <= 1e-7 * r64["gamma_eff"]
    rng = np.random.default_rng(8)
    report = []
    for _ in range(3):
        eta = rng.standard_normal(g.shape)
        fds = {}
        for h in (1e-7, 1e-4):
            jp = gpu_grad(g + h * eta, xi, K, m, sched=rho[None])[1]["gamma_eff"]
            jm = gpu_grad(g - h * eta, xi, K, m, sched=rho[None])[1]["gamma_eff"]
            fds[h] = (jp - jm) / (2 * h)
        fd = fds[1e-7]
        d64, dmx, d32 = (float(np.sum(gr * eta)) for gr in (g64, gmx, g32))
        report.append({"fd_h1e-7": fd, "fd_h1e-4": fds[1e-4], "rel_fp64": abs(fd - d64) / abs(fd),
                       "rel_fp64fwd_fp32rev": abs(fd - dmx) / abs(fd), "rel_fp32": abs(fd - d32) / abs(fd),
                       "rel_fp64_at_h1e-4": abs(fds[1e-4] - d64) / abs(fds[1e-4])})
        assert abs(fd - d64) <= 1e-4 * abs(fd)
        assert abs(fd - dmx) <= 1e-4 * abs(fd)
        assert abs(fd - d32) <= 3e-3 * abs(fd)
    print("directional derivatives against central differences:", report)


def test_autograd_function():
    g = M.uniform_random((8, 6, 10), 0.5, 1.5, 21)
    plan = ccmf.Plan(g.shape, batch=1, precision=ccmf.CCMF_FP64, device=DEV)
    gt = torch.from_numpy(g).to(DEV).requires_grad_(True)
    J = ccmf.crack_energy(gt, [0.0, 0.6, 0.8], plan, 30, 10, ccmf.Params(rho0=0.45))
    (dg,) = torch.autograd.grad(3.0 * J, gt)
    ref, res, rho = plan.gradient(gt.detach(), [[0.0, 0.6, 0.8]], 30, 10, ccmf.Params(rho0=0.45))
    np.testing.assert_allclose(dg.cpu().numpy(), 3.0 * ref[0].cpu().numpy(), rtol=1e-12, atol=0)
    assert abs(J.item() - res[0]["gamma_eff"]) <= 1e-14

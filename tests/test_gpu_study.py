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

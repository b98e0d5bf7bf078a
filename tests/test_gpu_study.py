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

"""CPU-side checks of the C ABI: the library builds, loads, exports every symbol
declared in include/ccmf.h, and rejects invalid arguments before touching a GPU."""

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ccmf.h")

needs_nvcc = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ccmf_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_05968_gb300 import _build, ccmf
    _build.build()
    return ccmf.load_library()


def test_header_declares_expected_entry_points():
    names = header_functions()
    for n in ("ccmf_plan_create", "ccmf_plan_destroy", "ccmf_plan_workspace_bytes", "ccmf_solve",
              "ccmf_state_export", "ccmf_state_import", "ccmf_history_export", "ccmf_status_string"):
        assert n in names


@needs_nvcc
def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


@needs_nvcc
def test_binding_covers_every_declared_symbol(lib):
    from paper_2103_05968_gb300 import ccmf
    for name in header_functions():
        assert name in ccmf._SIGNATURES, name
        assert callable(getattr(ccmf, name)), name


@needs_nvcc
def test_status_strings_and_defaults(lib):
    from paper_2103_05968_gb300 import ccmf
    assert ccmf.ccmf_status_string(0) == "ok"
    assert "unsupported" in ccmf.ccmf_status_string(ccmf.CCMF_ERR_UNSUPPORTED_SIZE)
    p = ccmf.ccmf_params_default()
    assert p.tol == 1e-4 and p.delta == 0.25 and p.rho_rule == ccmf.CCMF_RHO_BB and p.max_iter == 20000


@needs_nvcc
@pytest.mark.parametrize("shape,batch,prec,code", [
    ((0, 4, 4), 1, 1, 1), ((4, -1, 4), 1, 1, 1), ((4, 4, 4), 0, 1, 1), ((4, 4, 4), 1, 7, 1),
    ((7, 4, 4), 1, 1, 2), ((4, 11, 4), 1, 0, 2), ((4, 4, 2048), 1, 0, 2), ((4, 4, 49), 1, 1, 2),
])
def test_plan_create_rejects_before_any_cuda_call(lib, shape, batch, prec, code):
    from paper_2103_05968_gb300 import ccmf
    rc, handle = ccmf.ccmf_plan_create(*shape, batch, prec)
    assert rc == code and handle is None


@needs_nvcc
def test_null_arguments_rejected(lib):
    from paper_2103_05968_gb300 import ccmf
    assert lib.ccmf_plan_create(4, 4, 4, 1, 1, None) == ccmf.CCMF_ERR_INVALID_ARG
    assert lib.ccmf_plan_workspace_bytes(None, None) == ccmf.CCMF_ERR_INVALID_ARG
    assert lib.ccmf_plan_destroy(None) == ccmf.CCMF_OK
    assert lib.ccmf_solve(None, None, 0, None, None, None, 0, None, None, None, None) == ccmf.CCMF_ERR_INVALID_ARG
    assert lib.ccmf_set_kernel_timing(None, 1) == ccmf.CCMF_ERR_INVALID_ARG
    assert lib.ccmf_batch_set_persistent(None, 1) == ccmf.CCMF_ERR_INVALID_ARG
    assert lib.ccmf_batch_solve(None, None, None, None, None, 0, None, None) == ccmf.CCMF_ERR_INVALID_ARG
    assert lib.ccmf_batch_destroy(None) == ccmf.CCMF_OK


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2103_05968_gb300 import ccmf
    saved = ccmf._lib
    ccmf._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            ccmf.load_library(str(tmp_path / "missing.so"))
    finally:
        ccmf._lib = saved


@needs_nvcc
def test_tuning_table_text_roundtrip(lib):
    """The tuning table's text form is parsed back exactly; malformed text is rejected."""
    from paper_2103_05968_gb300 import ccmf
    line = "ccmf-tuning 48 40 10 3 1 152 : 3 0 8 4 16 2 1 8 1 0"
    assert ccmf.ccmf_tuning_import(line + "\n") == ccmf.CCMF_OK
    code, text = ccmf.ccmf_tuning_export()
    assert code == ccmf.CCMF_OK and line in text.splitlines()
    assert ccmf.ccmf_tuning_import("ccmf-tuning 1 2 3\n") == ccmf.CCMF_ERR_INVALID_ARG

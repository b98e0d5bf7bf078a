"""Thin Python binding of the CCMF solver's C ABI (include/ccmf.h).

Every entry point of the C library is exposed under the same name with the
same arguments (pointers as Python ints, host arrays as numpy arrays). The
classes `Plan` and `solve` below only marshal torch tensors into those calls:
PyTorch provides device memory and the stream, every step of the solver runs
in the library's CUDA kernels. There is no fallback: if the compiled library
is missing, loading it raises.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libccmf.so")

CCMF_OK = 0
CCMF_ERR_INVALID_ARG = 1
CCMF_ERR_UNSUPPORTED_SIZE = 2
CCMF_ERR_WORKSPACE = 3
CCMF_ERR_CUDA = 4
CCMF_ERR_NUMERICAL = 5
CCMF_ERR_TIMEOUT = 6

CCMF_FP64 = 0
CCMF_FP32_MIXED = 1

CCMF_RHO_BB = 0
CCMF_RHO_CONST = 1
CCMF_RHO_LTD = 2
CCMF_RHO_RB = 3

HIST_FIELDS = 6


class ccmf_params(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("bb_corr_min", ctypes.c_double),
        ("rho_step_max", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("rho_rule", ctypes.c_int),
        ("fixed_iters", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("resume", ctypes.c_int),
        ("history_len", ctypes.c_int),
    ]


class ccmf_result(ctypes.Structure):
    _fields_ = [
        ("gamma_eff", ctypes.c_double),
        ("gamma_primal", ctypes.c_double),
        ("gamma_dual", ctypes.c_double),
        ("residual", ctypes.c_double),
        ("mean_v_norm", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("iters", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("status", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


class ccmf_tuning(ctypes.Structure):
    _fields_ = [
        ("update_variant", ctypes.c_int),
        ("plane_blocks", ctypes.c_int),
        ("z_pairs_per_block", ctypes.c_int),
        ("y_lines_per_block", ctypes.c_int),
        ("x_lines_per_block", ctypes.c_int),
        ("branches", ctypes.c_int),
        ("radix_mode", ctypes.c_int),
        ("zinv_pairs_per_block", ctypes.c_int),
        ("line_engine", ctypes.c_int),
        ("z_engine", ctypes.c_int),
    ]


TUNING_KEYS = tuple(f[0] for f in ccmf_tuning._fields_)

_lib = None

# name -> (restype, argtypes); mirrors include/ccmf.h
_SIGNATURES = {
    "ccmf_params_default": (None, [ctypes.POINTER(ccmf_params)]),
    "ccmf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ccmf_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "ccmf_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "ccmf_plan_workspace_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "ccmf_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ccmf_params), ctypes.c_void_p,
                                   ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(ccmf_result), ctypes.c_void_p]),
    "ccmf_state_export": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                          ctypes.c_void_p]),
    "ccmf_state_import": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                          ctypes.c_void_p]),
    "ccmf_history_export": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "ccmf_kernel_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_char_p),
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "ccmf_set_kernel_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ccmf_plan_launch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]),
    "ccmf_plan_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ccmf_tuning)]),
    "ccmf_plan_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ccmf_tuning)]),
    "ccmf_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_size_t,
                                           ctypes.c_int, ctypes.POINTER(ccmf_tuning), ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_void_p]),
    "ccmf_tuning_export": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "ccmf_tuning_import": (ctypes.c_int, [ctypes.c_char_p]),
    "ccmf_adjoint_workspace_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                     ctypes.POINTER(ctypes.c_size_t)]),
    "ccmf_set_adjoint_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ccmf_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ccmf_params), ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ccmf_result),
                                     ctypes.c_void_p]),
    "ccmf_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "ccmf_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "ccmf_batch_workspace_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "ccmf_batch_buckets": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "ccmf_batch_set_persistent": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ccmf_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "ccmf_batch_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ccmf_params),
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ccmf_result),
                                         ctypes.c_void_p]),
    "ccmf_solve_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ccmf_params),
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ccmf_result),
                                          ctypes.c_void_p]),
}


def load_library(path=LIB_PATH):
    """Load libccmf.so (built by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CCMF CUDA library not built: {path} is missing "
                           "(run __graft_entry__.build() or python -m paper_2103_05968_gb300._build)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class CCMFError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {ccmf_status_string(code)} (status {code})")


def _check(code, where):
    if code != CCMF_OK:
        raise CCMFError(code, where)


# ---- same-name wrappers of the C entry points --------------------------------

def ccmf_params_default():
    p = ccmf_params()
    load_library().ccmf_params_default(ctypes.byref(p))
    return p


def ccmf_status_string(status):
    return load_library().ccmf_status_string(int(status)).decode()


def ccmf_plan_create(n1, n2, n3, batch, precision):
    out = ctypes.c_void_p()
    code = load_library().ccmf_plan_create(int(n1), int(n2), int(n3), int(batch), int(precision), ctypes.byref(out))
    return code, out.value


def ccmf_plan_destroy(plan):
    return load_library().ccmf_plan_destroy(plan)


def ccmf_plan_workspace_bytes(plan):
    b = ctypes.c_size_t()
    code = load_library().ccmf_plan_workspace_bytes(plan, ctypes.byref(b))
    return code, b.value


def ccmf_solve(plan, gamma_ptr, gamma_stride, xi_bar, params, workspace_ptr, workspace_bytes, flow_ptr, cut_ptr,
               results, stream):
    xi = np.ascontiguousarray(xi_bar, dtype=np.float64).reshape(-1)
    return load_library().ccmf_solve(plan, gamma_ptr, int(gamma_stride),
                                     xi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     ctypes.byref(params) if params is not None else None,
                                     workspace_ptr, int(workspace_bytes), flow_ptr, cut_ptr, results, stream)


def ccmf_state_export(plan, workspace_ptr, e_ptr, v_ptr, batch, stream):
    rho = (ctypes.c_double * batch)()
    iters = (ctypes.c_int * batch)()
    code = load_library().ccmf_state_export(plan, workspace_ptr, e_ptr, v_ptr, rho, iters, stream)
    return code, np.array(rho[:]), np.array(iters[:])


def ccmf_state_import(plan, workspace_ptr, e_ptr, v_ptr, rho, iters, stream):
    r = (ctypes.c_double * len(rho))(*[float(x) for x in rho])
    it = (ctypes.c_int * len(iters))(*[int(x) for x in iters])
    return load_library().ccmf_state_import(plan, workspace_ptr, e_ptr, v_ptr, r, it, stream)


def ccmf_history_export(plan, workspace_ptr, batch, max_entries, stream):
    out = np.zeros((batch, max_entries, HIST_FIELDS))
    cnt = ctypes.c_int()
    code = load_library().ccmf_history_export(plan, workspace_ptr,
                                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              int(max_entries), ctypes.byref(cnt), stream)
    return code, out[:, :cnt.value]


def ccmf_kernel_times(plan):
    cap = 16
    ms = (ctypes.c_double * cap)()
    launches = (ctypes.c_longlong * cap)()
    names = (ctypes.c_char_p * cap)()
    cnt = ctypes.c_int()
    code = load_library().ccmf_kernel_times(plan, ms, launches, names, cap, ctypes.byref(cnt))
    n = min(cnt.value, cap)
    return code, {names[i].decode(): (ms[i], launches[i]) for i in range(n)}


LAUNCH_INFO_KEYS = ("update_variant", "plane_fused", "plane_blocks", "z_pairs_per_block", "y_lines_per_block",
                    "x_lines_per_block", "update_blocks", "branches")


def ccmf_plan_launch_info(plan):
    out = (ctypes.c_int * len(LAUNCH_INFO_KEYS))()
    cnt = ctypes.c_int()
    code = load_library().ccmf_plan_launch_info(plan, out, len(LAUNCH_INFO_KEYS), ctypes.byref(cnt))
    return code, {k: int(out[i]) for i, k in enumerate(LAUNCH_INFO_KEYS)}


def ccmf_plan_get_tuning(plan):
    t = ccmf_tuning()
    code = load_library().ccmf_plan_get_tuning(plan, ctypes.byref(t))
    return code, {k: getattr(t, k) for k in TUNING_KEYS}


def ccmf_plan_set_tuning(plan, tuning):
    """tuning: dict of knob values (missing knobs = -1, the built-in rule)."""
    t = ccmf_tuning(**{k: int(tuning.get(k, -1)) for k in TUNING_KEYS})
    return load_library().ccmf_plan_set_tuning(plan, ctypes.byref(t))


def ccmf_plan_autotune(plan, gamma_ptr, gamma_stride, xi_bar, workspace_ptr, workspace_bytes, iters, stream):
    xi = np.ascontiguousarray(xi_bar, dtype=np.float64).reshape(-1)
    best = ccmf_tuning()
    ms = ctypes.c_double()
    code = load_library().ccmf_plan_autotune(plan, gamma_ptr, int(gamma_stride),
                                             xi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), workspace_ptr,
                                             int(workspace_bytes), int(iters), ctypes.byref(best), ctypes.byref(ms),
                                             stream)
    return code, {k: getattr(best, k) for k in TUNING_KEYS}, ms.value


def ccmf_tuning_export():
    n = ctypes.c_size_t()
    code = load_library().ccmf_tuning_export(None, 0, ctypes.byref(n))
    if code != CCMF_OK:
        return code, ""
    buf = ctypes.create_string_buffer(n.value + 1)
    code = load_library().ccmf_tuning_export(buf, n.value + 1, ctypes.byref(n))
    return code, buf.value.decode()


def ccmf_tuning_import(text):
    return load_library().ccmf_tuning_import(text.encode())


def ccmf_set_kernel_timing(plan, enable):
    return load_library().ccmf_set_kernel_timing(plan, int(enable))


def ccmf_adjoint_workspace_bytes(plan, K, ckpt_every):
    b = ctypes.c_size_t()
    code = load_library().ccmf_adjoint_workspace_bytes(plan, int(K), int(ckpt_every), ctypes.byref(b))
    return code, b.value


def ccmf_set_adjoint_forward(plan, precision):
    return load_library().ccmf_set_adjoint_forward(plan, int(precision))


def ccmf_adjoint(plan, gamma_ptr, gamma_stride, xi_bar, params, K, ckpt_every, rho_schedule, workspace_ptr,
                 workspace_bytes, adj_ptr, adj_bytes, grad_ptr, rho_out, results, stream):
    xi = np.ascontiguousarray(xi_bar, dtype=np.float64).reshape(-1)
    sched = None
    if rho_schedule is not None:
        sched_arr = np.ascontiguousarray(rho_schedule, dtype=np.float64).reshape(-1)
        sched = sched_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rout = rho_out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if rho_out is not None else None
    return load_library().ccmf_adjoint(plan, gamma_ptr, int(gamma_stride),
                                       xi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.byref(params) if params is not None else None, int(K), int(ckpt_every),
                                       sched, workspace_ptr, int(workspace_bytes), adj_ptr, int(adj_bytes), grad_ptr,
                                       rout, results, stream)


def ccmf_batch_create(shapes, precision):
    sh = np.ascontiguousarray(np.asarray(shapes, dtype=np.int32).reshape(-1, 3))
    out = ctypes.c_void_p()
    code = load_library().ccmf_batch_create(int(sh.shape[0]), sh.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                            int(precision), ctypes.byref(out))
    return code, out.value


def ccmf_batch_destroy(batch):
    return load_library().ccmf_batch_destroy(batch)


def ccmf_batch_workspace_bytes(batch):
    b = ctypes.c_size_t()
    code = load_library().ccmf_batch_workspace_bytes(batch, ctypes.byref(b))
    return code, b.value


def ccmf_batch_set_persistent(batch, enable):
    return load_library().ccmf_batch_set_persistent(batch, int(enable))


def ccmf_batch_buckets(batch):
    n = ctypes.c_int()
    code = load_library().ccmf_batch_buckets(batch, ctypes.byref(n))
    return code, n.value


def ccmf_batch_autotune(batch, gamma_ptrs, xi_bar, workspace_ptr, workspace_bytes, iters, buckets, stream):
    ptrs = (ctypes.c_void_p * len(gamma_ptrs))(*[int(p) for p in gamma_ptrs])
    xi = np.ascontiguousarray(xi_bar, dtype=np.float64).reshape(-1)
    ms = (ctypes.c_double * max(1, buckets))()
    code = load_library().ccmf_batch_autotune(batch, ptrs, xi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              workspace_ptr, int(workspace_bytes), int(iters), ms, stream)
    return code, list(ms[:buckets])


def ccmf_batch_solve(batch, gamma_ptrs, xi_bar, params, workspace_ptr, workspace_bytes, results, stream):
    ptrs = (ctypes.c_void_p * len(gamma_ptrs))(*[int(p) for p in gamma_ptrs])
    xi = np.ascontiguousarray(xi_bar, dtype=np.float64).reshape(-1)
    return load_library().ccmf_batch_solve(batch, ptrs, xi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           ctypes.byref(params) if params is not None else None,
                                           workspace_ptr, int(workspace_bytes), results, stream)


def ccmf_solve_static(n1, n2, n3, precision, gamma_ptr, xi_bar, params, flow_ptr, cut_ptr, result, stream):
    """The allocation-free single solve (see include/ccmf.h): all scratch lives in the
    library's fixed device array, so no workspace or plan is passed."""
    xi = np.ascontiguousarray(xi_bar, dtype=np.float64).reshape(3)
    return load_library().ccmf_solve_static(int(n1), int(n2), int(n3), int(precision), gamma_ptr,
                                            xi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            ctypes.byref(params) if params is not None else None,
                                            flow_ptr, cut_ptr, result, stream)


# ---- torch-facing convenience layer (argument marshalling only) --------------

@dataclasses.dataclass
class Params:
    tol: float = 1e-4
    delta: float = 0.25
    rho0: float = 0.0
    bb_corr_min: float = 0.2
    rho_step_max: float = 2.0
    max_iter: int = 20000
    rho_rule: int = CCMF_RHO_BB
    fixed_iters: int = 0
    check_every: int = 32
    resume: int = 0
    history_len: int = 1024

    def to_c(self):
        p = ccmf_params()
        for f in dataclasses.fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


def _stream_handle(torch, device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Plan:
    """A plan plus its torch-allocated workspace for `batch` solves on one grid."""

    def __init__(self, shape, batch=1, precision=CCMF_FP32_MIXED, device="cuda"):
        import torch

        self.torch = torch
        self.shape = tuple(int(x) for x in shape)
        self.batch = int(batch)
        self.precision = precision
        self.device = torch.device(device)
        self.dtype = torch.float64 if precision == CCMF_FP64 else torch.float32
        with torch.cuda.device(self.device):
            code, self.handle = ccmf_plan_create(*self.shape, self.batch, precision)
            _check(code, "ccmf_plan_create")
            code, nbytes = ccmf_plan_workspace_bytes(self.handle)
            _check(code, "ccmf_plan_workspace_bytes")
            self.workspace_bytes = nbytes
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256

    def close(self):
        if getattr(self, "handle", None):
            ccmf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_voxels(self):
        n1, n2, n3 = self.shape
        return n1 * n2 * n3

    def solve(self, gamma, normals, params=None, want_flow=False, want_cut=False, gamma_shared=None,
              want_results=True):
        """Run the solver. gamma: torch tensor (device or host) of shape (N1,N2,N3) shared
        by all solves, or (batch, N1, N2, N3). normals: (batch, 3). Returns (results, flow, cut)."""
        torch = self.torch
        params = params or Params()
        g = gamma
        if g.dtype != self.dtype:
            raise TypeError(f"gamma must be {self.dtype} for this plan")
        if not g.is_contiguous():
            raise ValueError("gamma must be contiguous")
        if gamma_shared is None:
            gamma_shared = (g.dim() == 3)
        stride = 0 if gamma_shared else self.n_voxels
        normals = np.asarray(normals, dtype=np.float64).reshape(self.batch, 3)
        n1, n2, n3 = self.shape
        on_dev = g.is_cuda
        flow = cut = None
        if want_flow:
            flow = torch.empty((self.batch, 3, n1, n2, n3), dtype=self.dtype, device=self.device if on_dev else "cpu")
        if want_cut:
            cut = torch.empty((self.batch, 6, n1, n2, n3), dtype=self.dtype, device=self.device if on_dev else "cpu")
        res = (ccmf_result * self.batch)()
        with torch.cuda.device(self.device):
            code = ccmf_solve(self.handle, ctypes.c_void_p(g.data_ptr()), stride, normals, params.to_c(),
                              ctypes.c_void_p(self.ws_ptr), self.workspace_bytes,
                              ctypes.c_void_p(flow.data_ptr()) if flow is not None else None,
                              ctypes.c_void_p(cut.data_ptr()) if cut is not None else None,
                              res if want_results else None, _stream_handle(torch, self.device))
        _check(code, "ccmf_solve")
        if not want_results:
            return None, flow, cut
        results = [{f[0]: getattr(r, f[0]) for f in ccmf_result._fields_} for r in res]
        return results, flow, cut

    def state(self):
        """(e, v, rho, iters): device copies of the ADMM state (checkpoint)."""
        torch = self.torch
        n1, n2, n3 = self.shape
        e = torch.empty((self.batch, 6, n1, n2, n3), dtype=self.dtype, device=self.device)
        v = torch.empty_like(e)
        with torch.cuda.device(self.device):
            code, rho, iters = ccmf_state_export(self.handle, ctypes.c_void_p(self.ws_ptr),
                                                 ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                                 self.batch, _stream_handle(torch, self.device))
        _check(code, "ccmf_state_export")
        return e, v, rho, iters

    def load_state(self, e, v, rho, iters):
        torch = self.torch
        e = e.to(device=self.device, dtype=self.dtype).contiguous()
        v = v.to(device=self.device, dtype=self.dtype).contiguous()
        with torch.cuda.device(self.device):
            code = ccmf_state_import(self.handle, ctypes.c_void_p(self.ws_ptr), ctypes.c_void_p(e.data_ptr()),
                                     ctypes.c_void_p(v.data_ptr()), list(rho), list(iters),
                                     _stream_handle(torch, self.device))
        _check(code, "ccmf_state_import")

    def history(self, max_entries=4096):
        torch = self.torch
        with torch.cuda.device(self.device):
            code, h = ccmf_history_export(self.handle, ctypes.c_void_p(self.ws_ptr), self.batch, max_entries,
                                          _stream_handle(torch, self.device))
        _check(code, "ccmf_history_export")
        return h

    def branches(self):
        """Independent graph branches the loop runs the batch in (at most 4, one per solve)."""
        return int(self.tuning()["branches"])

    def gradient(self, gamma, normals, K, ckpt_every=20, params=None, rho_schedule=None):
        """d gamma_eff / d gamma through K replayed updates (see ccmf_adjoint in include/ccmf.h).
        Returns (grad [batch, N1, N2, N3] on the device, results, rho schedule [batch, K])."""
        torch = self.torch
        params = params or Params()
        g = gamma
        stride = 0 if g.dim() == 3 else self.n_voxels
        normals = np.asarray(normals, dtype=np.float64).reshape(self.batch, 3)
        n1, n2, n3 = self.shape
        with torch.cuda.device(self.device):
            code, abytes = ccmf_adjoint_workspace_bytes(self.handle, K, ckpt_every)
            _check(code, "ccmf_adjoint_workspace_bytes")
            aws = torch.empty(abytes + 256, dtype=torch.uint8, device=self.device)
            aptr = (aws.data_ptr() + 255) // 256 * 256
            grad = torch.empty((self.batch, n1, n2, n3), dtype=self.dtype, device=self.device)
            rho_out = np.zeros((self.batch, K))
            res = (ccmf_result * self.batch)()
            code = ccmf_adjoint(self.handle, ctypes.c_void_p(g.data_ptr()), stride, normals, params.to_c(), K,
                                ckpt_every, rho_schedule, ctypes.c_void_p(self.ws_ptr), self.workspace_bytes,
                                ctypes.c_void_p(aptr), abytes, ctypes.c_void_p(grad.data_ptr()), rho_out, res,
                                _stream_handle(torch, self.device))
        _check(code, "ccmf_adjoint")
        results = [{f[0]: getattr(r, f[0]) for f in ccmf_result._fields_} for r in res]
        return grad, results, rho_out

    def set_adjoint_forward(self, precision):
        """Precision of the forward / recompute passes of gradient() (ccmf_set_adjoint_forward):
        CCMF_FP64 on an FP32 plan gives the FP64 forward with the FP32 reverse sweep."""
        with self.torch.cuda.device(self.device):
            _check(ccmf_set_adjoint_forward(self.handle, precision), "ccmf_set_adjoint_forward")

    def set_kernel_timing(self, enable):
        _check(ccmf_set_kernel_timing(self.handle, 1 if enable else 0), "ccmf_set_kernel_timing")

    def kernel_times(self):
        code, t = ccmf_kernel_times(self.handle)
        _check(code, "ccmf_kernel_times")
        return t

    def tuning(self):
        """The plan's knob values (see ccmf_tuning in include/ccmf.h)."""
        code, t = ccmf_plan_get_tuning(self.handle)
        _check(code, "ccmf_plan_get_tuning")
        return t

    def set_tuning(self, **knobs):
        """Set knob values by name; the others keep the built-in rule."""
        _check(ccmf_plan_set_tuning(self.handle, knobs), "ccmf_plan_set_tuning")

    def autotune(self, gamma, normals, iters=10):
        """Time candidate tunings on this plan's current state and keep the fastest
        (ccmf_plan_autotune); returns (tuning, ms per iteration)."""
        torch = self.torch
        stride = 0 if gamma.dim() == 3 else self.n_voxels
        normals = np.asarray(normals, dtype=np.float64).reshape(self.batch, 3)
        with torch.cuda.device(self.device):
            code, best, ms = ccmf_plan_autotune(self.handle, ctypes.c_void_p(gamma.data_ptr()), stride, normals,
                                                ctypes.c_void_p(self.ws_ptr), self.workspace_bytes, iters,
                                                _stream_handle(torch, self.device))
        _check(code, "ccmf_plan_autotune")
        return best, ms

    def launch_info(self):
        """The launch shape the plan chose (update variant, plane pass blocks per plane, ...)."""
        code, info = ccmf_plan_launch_info(self.handle)
        _check(code, "ccmf_plan_launch_info")
        return info


class Batch:
    """Solves on grids of different shapes in one call (argument marshalling only)."""

    def __init__(self, shapes, precision=CCMF_FP32_MIXED, device="cuda"):
        import torch

        self.torch = torch
        self.shapes = [tuple(int(x) for x in sh) for sh in shapes]
        self.count = len(self.shapes)
        self.precision = precision
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            code, self.handle = ccmf_batch_create(self.shapes, precision)
            _check(code, "ccmf_batch_create")
            code, nbytes = ccmf_batch_workspace_bytes(self.handle)
            _check(code, "ccmf_batch_workspace_bytes")
            self.workspace_bytes = nbytes
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        self.ws_ptr = (self.workspace.data_ptr() + 255) // 256 * 256

    def set_persistent(self, enable=True):
        """One persistent launch per iteration for the whole batch (ccmf_batch_set_persistent)."""
        _check(ccmf_batch_set_persistent(self.handle, 1 if enable else 0), "ccmf_batch_set_persistent")

    def buckets(self):
        code, n = ccmf_batch_buckets(self.handle)
        _check(code, "ccmf_batch_buckets")
        return n

    def close(self):
        if getattr(self, "handle", None):
            ccmf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, gammas, normals, iters=10):
        """Tune every shape group's launch shape on its own solves (ccmf_batch_autotune);
        returns each group's time per iteration in ms."""
        torch = self.torch
        ptrs = [g.data_ptr() for g in gammas]
        with torch.cuda.device(self.device):
            code, ms = ccmf_batch_autotune(self.handle, ptrs, np.asarray(normals, dtype=np.float64),
                                           ctypes.c_void_p(self.ws_ptr), self.workspace_bytes, iters, self.buckets(),
                                           _stream_handle(torch, self.device))
        _check(code, "ccmf_batch_autotune")
        return ms

    def solve(self, gammas, normals, params=None, want_results=True):
        """gammas: list of device tensors (one per solve, may repeat); normals: (count, 3)."""
        torch = self.torch
        params = params or Params()
        ptrs = [g.data_ptr() for g in gammas]
        res = (ccmf_result * self.count)()
        with torch.cuda.device(self.device):
            code = ccmf_batch_solve(self.handle, ptrs, np.asarray(normals, dtype=np.float64), params.to_c(),
                                    ctypes.c_void_p(self.ws_ptr), self.workspace_bytes,
                                    res if want_results else None, _stream_handle(torch, self.device))
        _check(code, "ccmf_batch_solve")
        if not want_results:
            return None
        return [{f[0]: getattr(r, f[0]) for f in ccmf_result._fields_} for r in res]


def crack_energy(gamma, normal, plan, K, ckpt_every=20, params=None):
    """gamma_eff(normal) after K updates as a differentiable torch function of gamma.

    The forward pass runs K updates with the adaptive penalty rule (ccmf_solve) and
    records the penalty schedule from the history ring; it returns the max-flow value.
    The reverse sweep runs only in the backward pass: the library's reverse mode
    (ccmf_adjoint) replays the recorded schedule, so it differentiates the same map.
    """
    import torch

    if K > 4096:
        raise ValueError("crack_energy records the penalty schedule in the history ring: K <= 4096")
    base = params or Params()

    class _CrackEnergy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, g):
            gd = g.detach().contiguous()
            rec = dataclasses.replace(base, fixed_iters=K, check_every=K, resume=0, history_len=K)
            res, _, _ = plan.solve(gd, [normal], rec)
            rho = plan.history(K)[0][:, 1].copy()
            ctx.save_for_backward(gd)
            ctx.rho = rho
            return torch.tensor(res[0]["gamma_eff"], dtype=g.dtype, device=g.device)

        @staticmethod
        def backward(ctx, gout):
            (gd,) = ctx.saved_tensors
            grad, _, _ = plan.gradient(gd, [normal], K, ckpt_every, base, rho_schedule=ctx.rho[None, :])
            return gout * grad[0]

    return _CrackEnergy.apply(gamma)

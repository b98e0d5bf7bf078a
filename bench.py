"""Benchmark: ADMM voxel-iterations per second of the CCMF FFT-ADMM solver.

One step = one damped-ADMM iteration (Eq. 30 of the paper: FFT projection onto
K, node-wise projection onto C_gamma, multiplier / residual / penalty update)
over every solve of the workload. Default workload: 128^3 Boolean model of
overlapping balls (radius 6 voxels, volume fraction 0.20, gamma 0.3 in balls /
1.0 matrix) with the three crack normals e1, e2, e3 solved together (3 solves),
FP32 fields with FP64 reductions.

Output: one JSON line (rank 0). Besides the keys of the contract it carries
`roofline` (dominant kernel against the measured HBM copy bandwidth, plus the
whole step on the 132 B/voxel basis: read e, v, gamma, the spectrum and two
stored divergences, write e, v, the spectrum and the divergences), `fibres512`
(the same figures for one 512^3 short-fibre solve, when run on one GPU),
`kernels`, `fp32_vs_fp64`, `cufft_yardstick` and `cpu_baseline` (the oracle on
all host cores and on one).
Multi-GPU runs (torchrun) are replicas: every rank solves the same workload on
its own GPU; value = all ranks' voxel-iterations / slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADMM voxel-iters/s, FP32-mixed vs FP64 at rel γ_eff err ≤1e-5; HBM % of peak"
UNIT = "voxel-iters/s"
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "boolean128": dict(shape=(128, 128, 128), normals=[[1, 0, 0], [0, 1, 0], [0, 0, 1]],
                       desc="128^3 Boolean spheres r=6 vf=0.20 gamma 0.3/1.0, normals e1,e2,e3 (3 solves)"),
    "batch192": dict(shape=None, normals=[[1, 0, 0], [0, 1, 0], [0, 0, 1]],
                     desc="192 solves: 64 Boolean-sphere realisations (radius U[4,8], volume fraction U[0.10,0.30], "
                          "gamma 0.2/1.0, grid drawn from {64,96,128,160}^3) x normals e1,e2,e3, one graph"),
    "fibres512": dict(shape=(512, 512, 512), normals=[[0, 0, 1]],
                      desc="512^3 short fibres d=6 AR=20 vf=0.12 gamma 3.0/1.0 (256^3 RSA cell tiled 2x2x2), "
                           "normal e3 (1 solve)"),
}


def make_gamma(name, dtype):
    from paper_2103_05968_gb300 import microstructure as M
    if name == "boolean128":
        g, _ = M.config_boolean_spheres_128(dtype=dtype)
        return g
    if name == "fibres512":
        g, _ = M.config_short_fibres_512(dtype=dtype)
        return g
    raise ValueError(name)


def batch_inputs(dtype, seed=2103, solves=192):
    """The 64 realisations of the batched workload: (fields, per-solve field index, normals, shapes).
    With solves < 192 only the first solves (and the realisations they use) are made."""
    from paper_2103_05968_gb300 import microstructure as M
    rng = np.random.default_rng(seed)
    fields = []
    nreal = min(64, (solves + 2) // 3)
    for r in range(nreal):
        n = int(rng.choice([64, 96, 128, 160]))
        vf = float(rng.uniform(0.10, 0.30))
        g, _ = M.boolean_spheres((n, n, n), 4.0, vf, 0.2, 1.0, seed=seed + 1 + r, radius_max=8.0, dtype=dtype)
        fields.append(g)
    index = [r for r in range(nreal) for _ in range(3)][:solves]
    normals = np.array([nv for _ in range(nreal) for nv in WORKLOADS["batch192"]["normals"]],
                       dtype=np.float64)[:solves]
    shapes = [fields[r].shape for r in index]
    return fields, index, normals, shapes


def run_batch(args, world, rank, local):
    """The batched workload: 192 solves of 4 grid shapes in one captured graph."""
    import torch

    import __graft_entry__
    from paper_2103_05968_gb300 import ccmf

    __graft_entry__.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    prec = ccmf.CCMF_FP64 if args.precision == "fp64" else ccmf.CCMF_FP32_MIXED
    np_dtype = np.float64 if prec == ccmf.CCMF_FP64 else np.float32
    esize = 8 if prec == ccmf.CCMF_FP64 else 4
    fields, index, normals, shapes = batch_inputs(np_dtype, solves=args.batch_solves)
    dfields = [torch.from_numpy(f).to(dev) for f in fields]
    gammas = [dfields[r] for r in index]
    vox = sum(int(np.prod(sh)) for sh in shapes)
    batch = ccmf.Batch(shapes, precision=prec, device=dev)
    if args.batch_launch == "persistent":
        batch.set_persistent(True)
    K, W = args.steps, args.warmup
    p = ccmf.Params(fixed_iters=K, check_every=K)
    tune = None
    if not args.no_autotune:   # set-up: every shape group's launch shape, timed on its own solves
        t_tune = time.perf_counter()
        ms_groups = batch.autotune(gammas, normals, iters=args.tune_iters)
        tune = {"ms_per_iter_groups": ms_groups, "seconds": time.perf_counter() - t_tune,
                "iters_per_candidate": args.tune_iters}
    batch.solve(gammas, normals, ccmf.Params(fixed_iters=W, check_every=W))
    batch.solve(gammas, normals, p, want_results=False)      # capture
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    batch.solve(gammas, normals, p, want_results=False)      # init + K iterations + final evaluation
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    clk = clocks.stop()
    value = world * vox * K / (t_ms * 1e-3)
    peak, peak_kind = load_peaks()
    step_bytes = vox * basis_bytes_per_voxel(esize)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if esize == 8 else "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS["batch192"]["desc"] + (
                               "" if len(shapes) == 192 else f" (first {len(shapes)} solves)"), "solves": len(shapes),
                           "voxels_per_step": vox, "buckets": batch.buckets(), "precision": args.precision,
                           "launch": args.batch_launch, "l2": "inputs larger than L2"},
                "roofline": {"bound": "hbm", "achieved": step_bytes / (t_ms / K * 1e-3) / 1e9, "peak": peak,
                             "unit": "GB/s", "frac": step_bytes / (t_ms / K * 1e-3) / 1e9 / peak,
                             "traffic": None,
                             "kernel": f"whole step ({basis_bytes_per_voxel(esize)} B/voxel basis)",
                             "peak_kind": peak_kind},
                "autotune": tune, "clocks": clk}
        print(json.dumps(line), flush=True)
    batch.close()


def basis_bytes_per_voxel(esize):
    """Algorithmic HBM bytes of one ADMM iteration per voxel in the three-pass schedule:
    pass 1 reads two stored divergences a = div^- A* e, b = div^- A* v (2 esize) and writes
    the half spectrum (esize), pass 2 reads and writes it (2 esize), pass 3 reads it (esize)
    and e, v, gamma (13 esize) and writes e, v and the divergences (14 esize): 33 esize,
    i.e. 132 B in FP32 and 264 B in FP64."""
    return 33 * esize


def bytes_per_voxel(kernel, esize, n3, stored_div=False):
    """Algorithmic DRAM bytes per voxel of one launch of each loop kernel. stored_div: the
    stored-divergence schedule (update variants 8 - 10), whose first pass reads the two
    divergences a, b and whose update pass also writes them."""
    half = (n3 // 2 + 1) / n3 * 2 * esize  # half-spectrum bytes per voxel
    return {
        "k_div_rfft_z": (2 if stored_div else 12) * esize + half,   # read a, b (or e, v); write spectrum
        "k_fft_y_fwd": 2 * half,                    # read + write spectrum
        "k_fft_x_solve": 2 * half,
        "k_fft_y_inv": 2 * half,
        "k_fft_plane": 2 * half,                    # read + write spectrum once (y, x, solve, x, y fused)
        "k_irfft_z": half + esize,                  # read spectrum; write phi
        # read e, v, gamma, phi; write e, v (and a, b)
        "k_update": 12 * esize + 2 * esize + 12 * esize + (2 * esize if stored_div else 0),
    }[kernel]


def plan_stored_div(plan):
    """True when the plan's update variant is the stored-divergence schedule (8 .. 10, 13 .. 15)."""
    v = int(plan.tuning()["update_variant"])
    return 8 <= v <= 10 or 13 <= v <= 15


def load_traffic(kernel, workload, precision, with_source=False):
    """DRAM bytes per launch of a kernel from the committed ncu summaries (profiles/*.md),
    or None when no capture of this kernel, workload and precision is recorded. The
    update pass is keyed with its variant (k_update@v<variant>), so a figure measured on
    one variant is never reported for another. with_source: also return the file name."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            parts = line.split()
            if len(parts) == 5 and parts[0] == "dram_bytes_per_launch" and parts[1:4] == [kernel, workload,
                                                                                           precision]:
                return (float(parts[4]), os.path.basename(path)) if with_source else float(parts[4])
    return (None, None) if with_source else None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in d:
                    return float(d[key]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_gpu{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # nvidia-smi needs a moment to start: wait for its first sample before the timed region
            t_end = time.time() + 3.0
            while time.time() < t_end and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _check_tuning(code, where):
    if code != 0:
        raise RuntimeError(f"tuning table {where}: status {code}")


def graph_ms_per_iter(plan, gamma_dev, normals, iters=30):
    """Device time per iteration of the captured loop (CUDA events on the launching stream)."""
    import torch
    from paper_2103_05968_gb300 import ccmf
    p = ccmf.Params(fixed_iters=iters, check_every=iters, resume=1, history_len=0)
    plan.solve(gamma_dev, normals, p, want_results=False)   # capture
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(gamma_dev.device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    plan.solve(gamma_dev, normals, p, want_results=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / iters


def first_persistent(values, ref, rel):
    """Number of updates after which |values[k] - ref| / |ref| <= rel holds from there on
    (values[k] is the max-flow value at iteration k), or None if the last one misses."""
    ok = np.abs(np.asarray(values) - ref) <= rel * abs(ref)
    if len(ok) == 0 or not ok[-1]:
        return None
    bad = np.nonzero(~ok)[0]
    return int(bad[-1] + 1) if len(bad) else 0


def time_to_accuracy(gamma_np, normals, dev, rel=1e-5, ref_tol=1e-7, max_iter=4000, max_extra=8000):
    """FP32-mixed against plain FP64 on the GPU at relative gamma_eff error <= rel.

    Reference gamma*: the FP64 solve run to the Eq. 31 criterion with tol ref_tol (at
    most max_iter updates, recorded in the history ring), then continued to tol
    ref_tol / 100 (at most max_extra more updates). For
    each precision the max-flow value <xi_bar, A* v^k> is read from the history ring at
    every iteration k; the iterations to accuracy are the first k after which it stays
    within rel of gamma*; time = iterations x device time per iteration of that precision."""
    import torch
    from paper_2103_05968_gb300 import ccmf
    B = normals.shape[0]
    hist_len = min(max_iter, 4096)
    out = {"rel_err": rel, "ref": f"FP64 GPU solve to tol {ref_tol / 100:g} (Eq. 31), max {max_iter + max_extra} "
                                  f"iterations"}
    plan64 = ccmf.Plan(gamma_np.shape, batch=B, precision=ccmf.CCMF_FP64, device=dev)
    g64 = torch.from_numpy(gamma_np.astype(np.float64)).to(dev)
    res64, _, _ = plan64.solve(g64, normals, ccmf.Params(tol=ref_tol, max_iter=max_iter, history_len=hist_len))
    h64 = plan64.history(hist_len)
    iters_ref = max(int(r["iters"]) for r in res64)
    # gamma*: the same FP64 solves continued (resume) until Eq. 31 holds at tol ref_tol / 100
    # or max_extra more updates, so that its own uncertainty (min cut minus max flow) is far
    # below the accuracy threshold
    fin, _, _ = plan64.solve(g64, normals, ccmf.Params(tol=ref_tol / 100, max_iter=max_extra, resume=1,
                                                       history_len=0))
    ref = np.array([r["gamma_eff"] for r in fin])
    plan64.autotune(g64, normals, iters=5)   # both precisions timed in their tuned launch shapes
    ms64 = graph_ms_per_iter(plan64, g64, normals)
    plan64.close()
    plan32 = ccmf.Plan(gamma_np.shape, batch=B, precision=ccmf.CCMF_FP32_MIXED, device=dev)
    g32 = torch.from_numpy(gamma_np.astype(np.float32)).to(dev)
    res32, _, _ = plan32.solve(g32, normals, ccmf.Params(fixed_iters=iters_ref, history_len=hist_len))
    h32 = plan32.history(hist_len)
    ms32 = graph_ms_per_iter(plan32, g32, normals)
    plan32.close()
    k64 = [first_persistent(h64[s][:int(res64[s]["iters"]), 5], ref[s], rel) for s in range(B)]
    k32 = [first_persistent(h32[s][:, 5], ref[s], rel) for s in range(B)]
    out.update({"gamma_ref": ref.tolist(), "ref_iters": [int(r["iters"]) for r in fin],
                "ref_gap_rel": [(r["gamma_primal"] - r["gamma_dual"]) / abs(r["gamma_dual"]) for r in fin],
                "ref_converged": [bool(r["converged"]) for r in fin],
                "ref_tol": ref_tol / 100, "history_iters": [int(r["iters"]) for r in res64],
                "iters_fp64": k64, "iters_fp32": k32, "ms_per_iter_fp64": ms64, "ms_per_iter_fp32": ms32,
                "fp32_final_rel_err": [abs(r["gamma_eff"] - ref[s]) / abs(ref[s]) for s, r in enumerate(res32)]})
    if None not in k64 and None not in k32 and max(k32) > 0:
        t64, t32 = max(k64) * ms64, max(k32) * ms32
        out.update({"ms_to_accuracy_fp64": t64, "ms_to_accuracy_fp32": t32, "speedup": t64 / t32})
    else:
        out["speedup"] = None
    return out


def call_ms(plan, gamma_dev, normals, iters):
    """Device time of one ccmf_solve call of `iters` iterations from the current state
    (init statistics, the captured loop, the final evaluation), CUDA events on the
    launching stream, after an untimed call that captures the graph."""
    import torch
    from paper_2103_05968_gb300 import ccmf
    p = ccmf.Params(fixed_iters=iters, check_every=iters, resume=1)
    plan.solve(gamma_dev, normals, p, want_results=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(gamma_dev.device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    plan.solve(gamma_dev, normals, p, want_results=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def fibres512_record(args, dev):
    """The 512^3 short-fibre workload (one solve, normal e3, FP32-mixed) measured beside
    the default line: ms per step of a K-step call (init, K iterations, final
    evaluation), ms per iteration from the difference of a 2K- and a K-step call
    (the per-call work cancels), both on the 132 B/voxel basis, and the dominant kernel
    of a sequential event-timed pass against the measured HBM bandwidth."""
    import torch
    from paper_2103_05968_gb300 import ccmf
    t_set = time.perf_counter()
    gamma_np = make_gamma("fibres512", np.float32)
    normals = np.asarray(WORKLOADS["fibres512"]["normals"], dtype=np.float64)
    N = gamma_np.size
    plan = ccmf.Plan(gamma_np.shape, batch=1, precision=ccmf.CCMF_FP32_MIXED, device=dev)
    gamma_dev = torch.from_numpy(gamma_np).to(dev)
    del gamma_np
    K = max(args.steps, 20)
    plan.solve(gamma_dev, normals, ccmf.Params(fixed_iters=args.warmup, check_every=args.warmup))
    tune = None
    if not args.no_autotune:
        best, tune_ms = plan.autotune(gamma_dev, normals, iters=max(10, args.tune_iters // 2))
        tune = {"tuning": best, "ms_per_iter": tune_ms}
    setup_s = time.perf_counter() - t_set
    t_k = call_ms(plan, gamma_dev, normals, K)
    t_2k = call_ms(plan, gamma_dev, normals, 2 * K)
    plan.set_kernel_timing(True)
    call_ms(plan, gamma_dev, normals, K)
    kt = {k: v for k, v in plan.kernel_times().items() if v[1] > 0}
    plan.set_kernel_timing(False)
    peak, peak_kind = load_peaks()
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / kt[dom][1]
    sd = plan_stored_div(plan)
    dom_bytes = bytes_per_voxel(dom, 4, 512, sd) * N
    basis = basis_bytes_per_voxel(4) * N
    ms_step, ms_iter = t_k / K, (t_2k - t_k) / K
    tuning = plan.tuning()
    plan.close()
    return {"workload": WORKLOADS["fibres512"]["desc"] + " FP32-mixed (FP64 reductions)", "steps": K,
            "ms_per_step": ms_step, "value": N * K / (t_k * 1e-3), "unit": UNIT,
            "step_frac_132": basis / (ms_step * 1e-3) / 1e9 / peak,
            "ms_per_iter": ms_iter, "iter_frac_132": basis / (ms_iter * 1e-3) / 1e9 / peak,
            "target_ms_per_iter_at_0.60": basis / (0.60 * peak * 1e9) * 1e3,
            "dominant_kernel": {"kernel": dom, "ms_per_launch": dom_ms,
                                "achieved_gbs": dom_bytes / (dom_ms * 1e-3) / 1e9,
                                "frac": dom_bytes / (dom_ms * 1e-3) / 1e9 / peak},
            "kernels_ms_per_launch": {k: v[0] / v[1] for k, v in kt.items()},
            "own_schedule_bytes_per_voxel": sum(bytes_per_voxel(k, 4, 512, sd) for k in kt),
            "tuning": tuning,
            "peak": peak, "peak_kind": peak_kind, "autotune": tune, "setup_seconds": setup_s,
            "l2": "inputs larger than L2: state 6.4 GB per step"}


def batch192_record(args, dev):
    """The batched workload (192 solves on grids of four shapes, one captured graph with one
    branch per shape group) measured beside the default line: ms per step of a K-step call
    (init, K iterations, final evaluation) and ms per iteration from the difference of a 2K-
    and a K-step call, both on the 132 B/voxel basis over all voxels of the batch."""
    import torch
    from paper_2103_05968_gb300 import ccmf
    t_set = time.perf_counter()
    fields, index, normals, shapes = batch_inputs(np.float32)
    dfields = [torch.from_numpy(f).to(dev) for f in fields]
    del fields
    gammas = [dfields[r] for r in index]
    vox = sum(int(np.prod(sh)) for sh in shapes)
    batch = ccmf.Batch(shapes, precision=ccmf.CCMF_FP32_MIXED, device=dev)
    K = min(max(args.steps // 10, 20), 200)
    batch.solve(gammas, normals, ccmf.Params(fixed_iters=args.warmup, check_every=args.warmup))
    tune = None
    if not args.no_autotune:   # every shape group's launch shape, timed on its own solves
        ms_groups = batch.autotune(gammas, normals, iters=max(10, args.tune_iters // 4))
        tune = {"ms_per_iter_groups": ms_groups, "iters_per_candidate": max(10, args.tune_iters // 4)}
    setup_s = time.perf_counter() - t_set
    stream = torch.cuda.current_stream(dev)

    def timed_call(iters):
        p = ccmf.Params(fixed_iters=iters, check_every=iters)
        batch.solve(gammas, normals, p, want_results=False)   # captures the graph for this length
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        batch.solve(gammas, normals, p, want_results=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    t_k = timed_call(K)
    t_2k = timed_call(2 * K)
    peak, peak_kind = load_peaks()
    basis = basis_bytes_per_voxel(4) * vox
    ms_step, ms_iter = t_k / K, (t_2k - t_k) / K
    buckets = batch.buckets()
    # the same solves in one persistent launch per iteration (one device work queue)
    batch.set_persistent(True)
    tp_k = timed_call(K)
    tp_2k = timed_call(2 * K)
    pms_step, pms_iter = tp_k / K, (tp_2k - tp_k) / K
    persistent = {"launch": "one k_batch_persist launch per iteration: (pass, solve, tile) items of every "
                            "solve from one device queue", "ms_per_step": pms_step,
                  "value": vox * K / (tp_k * 1e-3), "step_frac_132": basis / (pms_step * 1e-3) / 1e9 / peak,
                  "ms_per_iter": pms_iter, "iter_frac_132": basis / (pms_iter * 1e-3) / 1e9 / peak}
    batch.close()
    return {"workload": WORKLOADS["batch192"]["desc"] + " FP32-mixed (FP64 reductions)", "solves": len(shapes),
            "voxels_per_step": vox, "steps": K, "ms_per_step": ms_step, "value": vox * K / (t_k * 1e-3),
            "unit": UNIT, "step_frac_132": basis / (ms_step * 1e-3) / 1e9 / peak, "ms_per_iter": ms_iter,
            "iter_frac_132": basis / (ms_iter * 1e-3) / 1e9 / peak, "buckets": buckets,
            "launch": "one captured graph, one branch per shape group (per-shape sub-plans)",
            "persistent": persistent,
            "peak": peak, "peak_kind": peak_kind, "autotune": tune, "setup_seconds": setup_s,
            "l2": f"inputs larger than L2: state {48 * vox / 1e9:.1f} GB per step"}


def cufft_yardstick(shape, B, dev, reps=20):
    """cuFFT (torch.fft) R2C + C2R of the same B scalar grids: a yardstick beside the
    solver's own FFT passes, not used by the solver."""
    import torch
    x = torch.randn((B,) + tuple(shape), device=dev, dtype=torch.float32)
    for _ in range(3):
        y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=shape, dim=(1, 2, 3))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(reps):
        y = torch.fft.irfftn(torch.fft.rfftn(x, dim=(1, 2, 3)), s=shape, dim=(1, 2, 3))
    ev1.record(stream)
    torch.cuda.synchronize()
    del y
    return ev0.elapsed_time(ev1) / reps


def _oracle_sample(name, max_seconds, max_iters=50):
    """A bounded sample of the oracle as it stands: FP64 iterations of one solve of the
    workload's grid (128^3 corner block of larger grids) until max_seconds or max_iters.
    Returns (voxel-iterations, wall seconds, CPU seconds, iterations, grid shape)."""
    from oracle import ccmf_oracle as O
    wl = WORKLOADS[name]
    gamma = make_gamma(name, np.float64) if name == "boolean128" else None
    if gamma is None:  # pragma: no cover - the large workload samples a 128^3 sub-block
        gamma = make_gamma(name, np.float32)[:128, :128, :128].astype(np.float64)
    xi = np.asarray(wl["normals"][0], dtype=np.float64)
    e = O.op_A(O.const_field(xi, gamma.shape))
    v = np.zeros((6,) + gamma.shape)
    rho = O.initial_rho(gamma, O.Params())
    t0, c0 = time.perf_counter(), time.process_time()
    iters = 0
    while True:
        _, e2, v2 = O.admm_step(e, v, rho, gamma, xi, 0.25)
        rho = O.next_rho(rho, O.RHO_BB, e, e2, v, v2, O.Params())
        e, v = e2, v2
        iters += 1
        if time.perf_counter() - t0 > max_seconds or iters >= max_iters:
            break
    wall = time.perf_counter() - t0
    return gamma.size * iters, wall, time.process_time() - c0, iters, gamma.shape


def _oracle_worker(args):
    import os as _os
    _os.environ.setdefault("OMP_NUM_THREADS", "1")
    name, max_seconds, max_iters = args
    return _oracle_sample(name, max_seconds, max_iters)


def host_cpu():
    """(usable cores, CPU model string) of this host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return cores, f"{model or 'unknown'} ({platform.machine()})"


def cpu_baseline(name, max_seconds=20.0):
    """The oracle as it stands on the host cores, on a bounded sample of the workload:
    one process per usable core, each running FP64 iterations of one solve of the same
    grid for about max_seconds (throughput = all processes' voxel-iterations / wall
    time), then the same on one core. The processes are spawned, not forked, so a CUDA
    context of this process is never copied."""
    import multiprocessing as mp
    cores, model = host_cpu()
    one_vox, one_wall, one_cpu, one_it, shape = _oracle_sample(name, max_seconds)
    one = {"value": one_vox / one_wall, "unit": UNIT, "cores": 1, "iters": one_it,
           "sample": f"{one_it} FP64 oracle iterations of one solve ({shape[0]}^3) in {one_wall:.1f} s wall / "
                     f"{one_cpu:.1f} s CPU"}
    workers = max(1, min(cores, 64))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(workers) as pool:
        outs = pool.map(_oracle_worker, [(name, max_seconds, 50)] * workers)
    wall = time.perf_counter() - t0
    iters = sum(o[3] for o in outs)
    rate = sum(o[0] / o[1] for o in outs)   # the processes iterate concurrently
    return {"value": rate, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{workers} concurrent processes, each running FP64 oracle iterations of one solve "
                      f"({shape[0]}^3, normal {WORKLOADS[name]['normals'][0]}) for about {max_seconds:.0f} s: "
                      f"{iters} iterations; value = sum of the per-process rates ({wall:.1f} s wall with "
                      f"process start-up and field generation)",
            "nproc": cores, "cpu_model": model, "one_core": one}


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle, timed as it stands on the host cores. Each step is
    one FP64 oracle iteration of one solve (normal e1) on the 64^3 corner block of the
    workload's gamma field, treated as its own periodic cell (a bounded sample)."""
    if rank != 0:
        return
    from oracle import ccmf_oracle as O
    name = args.workload
    wl = WORKLOADS[name]
    gamma = np.ascontiguousarray(make_gamma(name, np.float64)[:64, :64, :64])
    xi = np.asarray(wl["normals"][0], dtype=np.float64)
    e = O.op_A(O.const_field(xi, gamma.shape))
    v = np.zeros((6,) + gamma.shape)
    rho = O.initial_rho(gamma, O.Params())

    def step():
        nonlocal e, v, rho
        _, e2, v2 = O.admm_step(e, v, rho, gamma, xi, 0.25)
        rho = O.next_rho(rho, O.RHO_BB, e, e2, v, v2, O.Params())
        e, v = e2, v2

    for _ in range(args.warmup):
        step()
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(args.steps):
        step()
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    value = gamma.size * args.steps / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl["desc"] + " -- reference arm (CPU oracle): per step one iteration of one "
                                               "solve (normal e1) on the 64^3 corner block",
                       "grid": list(gamma.shape), "solves": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": max(1, round(cpu / wall)), "kind": "oracle",
                             "sample": f"{args.steps} FP64 oracle iterations of one solve on the 64^3 corner block "
                                       f"after {args.warmup} warm-up iterations"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, world, rank, local):
    import torch

    import __graft_entry__
    from paper_2103_05968_gb300 import ccmf

    if rank == 0 or world == 1:
        __graft_entry__.build()
    barrier(world)
    __graft_entry__.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    name = args.workload
    wl = WORKLOADS[name]
    prec = ccmf.CCMF_FP64 if args.precision == "fp64" else ccmf.CCMF_FP32_MIXED
    np_dtype = np.float64 if prec == ccmf.CCMF_FP64 else np.float32
    esize = 8 if prec == ccmf.CCMF_FP64 else 4
    gamma_np = make_gamma(name, np_dtype)
    if args.grid:
        # a corner block of the workload's field (smaller profiling cases of the same kernels)
        n = [int(x) for x in args.grid.lower().split("x")]
        gamma_np = np.ascontiguousarray(gamma_np[:n[0], :n[1], :n[2]])
    normals = np.asarray(wl["normals"], dtype=np.float64)
    B = normals.shape[0]
    n1, n2, n3 = gamma_np.shape
    N = n1 * n2 * n3
    if args.tuning_in:
        _check_tuning(ccmf.ccmf_tuning_import(open(args.tuning_in).read()), args.tuning_in)
    plan = ccmf.Plan(gamma_np.shape, batch=B, precision=prec, device=dev)
    gamma_dev = torch.from_numpy(gamma_np).to(dev)
    K, W = args.steps, args.warmup

    if args.tuning_json:   # explicit knobs apply from the warm-up on
        plan.set_tuning(**json.loads(args.tuning_json))
    # initial state + warm-up (W iterations), untimed
    plan.solve(gamma_dev, normals, ccmf.Params(fixed_iters=W, check_every=W))
    torch.cuda.synchronize()
    # launch-shape autotuner (setup, outside the timed region): coordinate descent over the
    # update-pass variant, plane pass, lines per block, graph branches and radix schedule
    tune = None
    if args.tuning_json:
        tune = {"tuning": plan.tuning(), "note": "set from --tuning-json"}
    elif args.tuning_in:
        tune = {"tuning": plan.tuning(), "note": f"imported from {os.path.basename(args.tuning_in)}"}
    elif not args.no_autotune:
        t_tune = time.perf_counter()
        best, tune_ms = plan.autotune(gamma_dev, normals, iters=args.tune_iters)
        tune = {"tuning": best, "ms_per_iter": tune_ms, "seconds": time.perf_counter() - t_tune,
                "iters_per_candidate": args.tune_iters}
    else:
        tune = {"tuning": plan.tuning(), "note": "built-in rules (--no-autotune)"}
    if args.tuning_out:
        code, text = ccmf.ccmf_tuning_export()
        _check_tuning(code, "export")
        open(args.tuning_out, "w").write(text)
    stream = torch.cuda.current_stream(dev)
    p_timed = ccmf.Params(fixed_iters=K, check_every=K, resume=1)
    # capture the loop graph outside the timed region (same key as the timed call)
    plan.solve(gamma_dev, normals, p_timed, want_results=False)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    plan.solve(gamma_dev, normals, p_timed, want_results=False)   # K iterations + final evaluation
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    t_ms_max = max_over_ranks(t_ms, world)
    value = world * N * B * K / (t_ms_max * 1e-3)

    # per-kernel device times: the same K steps again, launched as one sequential chain
    # with CUDA events recorded between the kernels inside the captured graph
    plan.set_kernel_timing(True)
    plan.solve(gamma_dev, normals, p_timed, want_results=False)   # capture the timed graph
    torch.cuda.synchronize()
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    plan.solve(gamma_dev, normals, p_timed, want_results=False)
    ev3.record(stream)
    torch.cuda.synchronize()
    t_seq_ms = ev2.elapsed_time(ev3)
    kt = {k: v for k, v in plan.kernel_times().items() if v[1] > 0}
    plan.set_kernel_timing(False)

    # roofline of the dominant kernel
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms, dom_n = kt[dom]
    sd = plan_stored_div(plan)
    per_launch_bytes = bytes_per_voxel(dom, esize, n3, sd) * N * B
    achieved = per_launch_bytes / (dom_ms / dom_n * 1e-3) / 1e9
    peak, peak_kind = load_peaks()
    kern = {k: {"ms_per_launch": ms / n, "launches": n, "share": ms / sum(x[0] for x in kt.values()),
                "gbs": bytes_per_voxel(k, esize, n3, sd) * N * B / (ms / n * 1e-3) / 1e9}
            for k, (ms, n) in kt.items()}
    own_bpv = sum(bytes_per_voxel(k, esize, n3, sd) for k in kt)
    tuned = plan.tuning()
    traffic_key = f"{dom}@v{tuned['update_variant']}" if dom == "k_update" else dom
    traffic, traffic_src = (None, None) if args.grid else load_traffic(traffic_key, name, args.precision,
                                                                       with_source=True)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "traffic_source": (f"ncu capture summarised in profiles/{traffic_src} (not this run)"
                                   if traffic_src else None),
                "kernel": traffic_key, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "kernel_times_from": f"sequential event-timed pass of the same {K} steps "
                                     f"({t_seq_ms / K:.4f} ms/step)",
                "step_frac_132": basis_bytes_per_voxel(esize) * N * B / (t_ms_max / K * 1e-3) / 1e9 / peak,
                "step_basis_bytes_per_voxel": basis_bytes_per_voxel(esize),
                "step_frac_own_schedule": own_bpv * N * B / (t_ms_max / K * 1e-3) / 1e9 / peak,
                "own_schedule_bytes_per_voxel": own_bpv,
                "floor_100B_frac": (100 if esize == 4 else 200) * N * B / (t_ms_max / K * 1e-3) / 1e9 / peak}

    # end to end through the public API with host buffers: pinned gamma in, results out
    gamma_host = torch.from_numpy(gamma_np).pin_memory()
    p_e2e = ccmf.Params(fixed_iters=K, check_every=K)
    plan.solve(gamma_host, normals, p_e2e)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    res, _, _ = plan.solve(gamma_host, normals, p_e2e)   # H2D of gamma, init, K iterations, results D2H
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = world * N * B * K / t_e2e

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(name, max_seconds=args.cpu_seconds)

    # FFT passes of the solver beside cuFFT on the same grids (yardstick only)
    fft_cls = [k for k in kt if k.startswith("k_fft") or k.endswith("rfft_z")]
    yard = {"cufft_r2c_c2r_ms": cufft_yardstick((n1, n2, n3), B, dev),
            "solver_fft_passes_ms": sum(kt[k][0] / kt[k][1] for k in fft_cls),
            "solver_passes": fft_cls,
            "note": "cuFFT: torch.fft.rfftn + irfftn of B real grids; solver: its forward and inverse FFT "
                    "passes per iteration (the first also reads e, v and computes the divergence; the plane "
                    "pass also applies the Poisson symbol), sequential event timing"}

    # FP32-mixed vs plain FP64 time to relative gamma_eff error 1e-5 (default workload, rank 0)
    tta = None
    if rank == 0 and world == 1 and name == "boolean128" and esize == 4 and not args.no_speedup:
        tta = time_to_accuracy(gamma_np, normals, dev)

    # the 512^3 workload beside the default line (one GPU)
    fib = None
    if rank == 0 and world == 1 and name == "boolean128" and not args.grid and not args.no_fibres512:
        fib = fibres512_record(args, dev)
    b192 = None
    if rank == 0 and world == 1 and name == "boolean128" and not args.grid and not args.no_batch192:
        b192 = batch192_record(args, dev)

    # kernels launched in the timed region: per iteration one launch of each pass per graph
    # branch, plus setup and gamma statistics, plus the passes of the final evaluation
    nk = len(kt)
    launches = nk * K * plan.branches() + 2 + nk
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": t_ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if esize == 8 else "f32", "data": "synthetic",
                "config": {"workload": wl["desc"] + (f" -- corner block {args.grid}" if args.grid else "") +
                                       (" FP64" if esize == 8 else " FP32-mixed (FP64 reductions)"),
                           "grid": [n1, n2, n3], "solves": B, "parallelism": f"replicas x{world}",
                           "l2": f"inputs larger than L2: state {12 * esize * N * B / 1e6:.0f} MB per step",
                           "precision": args.precision},
                "roofline": roofline, "kernels": kern, "e2e": {
                    "value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(esize * N / K),
                    "d2h_bytes_per_step": int(B * 48 / K) + 1,
                    "note": f"one ccmf_solve from pinned host gamma: H2D {esize * N} B, init, {K} iterations, "
                            "final evaluation, results D2H"},
                "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu,
                "fp32_vs_fp64": tta, "cufft_yardstick": yard, "autotune": tune, "fibres512": fib,
                "batch192": b192,
                "gamma_eff": [r["gamma_eff"] for r in res]}
        print(json.dumps(line), flush=True)
    plan.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="boolean128", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch-shape rules")
    ap.add_argument("--tune-iters", type=int, default=40, help="iterations timed per autotuner candidate")
    ap.add_argument("--tuning-in", default=None, help="tuning table text to import instead of autotuning")
    ap.add_argument("--tuning-out", default=None, help="write the tuning table text here after autotuning")
    ap.add_argument("--tuning-json", default=None, help="knob values (JSON object) set on the plan, no autotuning")
    ap.add_argument("--grid", default=None, help="N1xN2xN3 corner block of the workload's field (profiling cases)")
    ap.add_argument("--no-fibres512", action="store_true",
                    help="skip the 512^3 short-fibre record beside the default workload")
    ap.add_argument("--batch-launch", default="graph", choices=["graph", "persistent"],
                    help="--workload batch192: the branched graph of per-shape passes, or one persistent launch "
                         "per iteration")
    ap.add_argument("--batch-solves", type=int, default=192,
                    help="--workload batch192: the first N solves only (small profiling cases)")
    ap.add_argument("--no-batch192", action="store_true",
                    help="skip the 192-solve batched record beside the default workload")
    ap.add_argument("--no-speedup", action="store_true",
                    help="skip the FP32-mixed vs FP64 time-to-accuracy measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, world, rank)
        return
    world, rank, local = dist_setup(args)
    if args.workload == "batch192":
        run_batch(args, world, rank, local)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

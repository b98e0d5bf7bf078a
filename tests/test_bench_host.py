"""Host logic of bench.py on the CPU: the algorithmic byte accounting of one ADMM pass, the
lookup of ncu DRAM bytes recorded in profiles/, the clock-sample parser and the
time-to-accuracy helper."""

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def test_bytes_per_voxel_of_one_pass():
    # FP32, N3 = 512: half spectrum 4 (257/512) * 2 = 4.02 B/voxel
    bpv = {k: bench.bytes_per_voxel(k, 4, 512) for k in
           ("k_div_rfft_z", "k_fft_y_fwd", "k_fft_x_solve", "k_fft_y_inv", "k_fft_plane", "k_irfft_z", "k_update")}
    half = 257 / 512 * 8
    assert bpv["k_div_rfft_z"] == pytest.approx(48 + half)
    assert bpv["k_update"] == 104                     # read e, v, gamma, phi; write e, v
    lines = bpv["k_div_rfft_z"] + 3 * bpv["k_fft_y_fwd"] + bpv["k_irfft_z"] + bpv["k_update"]
    plane = bpv["k_div_rfft_z"] + bpv["k_fft_plane"] + bpv["k_irfft_z"] + bpv["k_update"]
    assert lines == pytest.approx(188.1, abs=0.1)     # three line passes
    assert plane == pytest.approx(172.0, abs=0.1)     # the fused plane pass
    # FP64 doubles every figure
    assert bench.bytes_per_voxel("k_update", 8, 512) == 208
    # stored-divergence schedule: the first pass reads a, b (8 B), the update also writes them
    assert bench.bytes_per_voxel("k_div_rfft_z", 4, 512, True) == 8 + (257 / 512) * 8
    assert bench.bytes_per_voxel("k_update", 4, 512, True) == 112
    half = (257 / 512) * 8
    step = sum(bench.bytes_per_voxel(k, 4, 512, True)
               for k in ("k_div_rfft_z", "k_fft_y_fwd", "k_fft_x_solve", "k_fft_y_inv", "k_irfft_z", "k_update"))
    assert abs(step - (8 + half + 6 * half + half + 4 + 112)) < 1e-9
    assert bench.basis_bytes_per_voxel(4) == 132 and bench.basis_bytes_per_voxel(8) == 264


def test_traffic_lines_in_profiles_parse_and_are_found():
    seen = []
    for name in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        for line in open(os.path.join(ROOT, "profiles", name)):
            parts = line.split()
            if parts and parts[0] == "dram_bytes_per_launch":
                assert len(parts) == 5, line
                assert parts[1].startswith("k_") and parts[3] in ("fp32", "fp64"), line
                assert float(parts[4]) > 0
                seen.append(parts)
    assert seen, "no recorded DRAM traffic"
    for _, kernel, workload, prec, value in seen:
        assert bench.load_traffic(kernel, workload, prec) == float(value)
    # a variant without a capture has no traffic figure
    assert bench.load_traffic("k_update@v9", "boolean128", "fp32") is None


def test_clock_sampler_parses_samples(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 2040, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2070, 2070, 1250.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc = Done()
    s.fh = open(os.devnull, "w")
    out = s.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_first_persistent():
    ref = 1.0
    vals = [1.5, 1.0 + 2e-5, 1.0 + 5e-6, 1.0 + 3e-5, 1.0 + 1e-6, 1.0 - 1e-6]
    assert bench.first_persistent(vals, ref, 1e-5) == 4     # from the 5th value on
    assert bench.first_persistent(vals[:4], ref, 1e-5) is None
    assert bench.first_persistent([1.0, 1.0], ref, 1e-5) == 0
    assert bench.first_persistent(np.array([]), ref, 1e-5) is None

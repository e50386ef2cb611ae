"""Host-side arithmetic of bench.py (no GPU): the workload's sizes, the
peaks derived from unit counts, the algorithmic work counts of the
variable-coefficient forms, the roofline block and the coarse-in-fine node
map of the equal-error comparison."""
import numpy as np
import pytest

import bench
from paper_2105_01722_gb300 import inputs


def test_headline_workload_sizes():
    # 64 x 64 elements of 8 x 8 cells: (N+1)^2 = 81 GD nodes an element
    assert bench.dof() == 64 * 64 * 81
    assert bench.dof(dict(dim=1, n=(16,), N=8)) == 16 * 9
    assert bench.dof(dict(dim=3, n=(4, 4, 4), N=8)) == 64 * 729


def test_derived_peaks():
    # 152 SMs x 2070 MHz x 2 FP64 FMA lanes x 2 flop; FP32 with 128 lanes
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25856, rel=1e-5)
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(80.5478, rel=1e-5)
    assert bench.FP32_PEAK_TFLOPS / bench.FP64_PEAK_TFLOPS == pytest.approx(64.0)


def test_executed_flops_closed_form():
    # per element 44 n1 + 23.5 n1^2 with n1 = 9: 396 + 1903.5
    assert bench.executed_flops_per_stage_launch() == pytest.approx(4096 * 2299.5)


@pytest.mark.parametrize("n1", [4, 6, 9])
def test_var_counts_terms(n1):
    NA = n1 * n1
    face = 144 * n1 * n1 + 16 * NA
    it = 2 * NA * NA + 8 * n1 ** 3 + 12 * NA
    # FP64 PCG: each iteration adds one product, the preconditioner and vector work
    f0, g0, b0 = bench.var_counts(n1, 0, 0, "fp64")
    f1, _, b1 = bench.var_counts(n1, 3, 2, "fp64")
    assert g0 == 0.0 and f1 - f0 == pytest.approx(5 * it) and b1 == b0
    assert f0 == pytest.approx(2 * NA * NA + face + 16 * n1 ** 3)
    # mixed: the iterations move to FP32; each refinement sweep adds one FP64 product
    m0, m32, mb = bench.var_counts(n1, 3, 2, "mixed")
    m1, m32b, mb1 = bench.var_counts(n1, 3, 2, "mixed", sweeps_u=1.0, sweeps_v=1.0)
    assert m32 == m32b == pytest.approx(5 * it)
    assert m1 - m0 == pytest.approx(2 * 2 * NA * NA) and mb1 - mb == pytest.approx(2 * NA * NA * 8)
    # the FP32 copies of the two element matrices take half the FP64 bytes
    assert mb - 2 * NA * NA * 8 - 72 * n1 * n1 * 8 - 64 * NA == pytest.approx(2 * NA * NA * 4)
    # inverse: 12 n1 + NA folded columns of NA entries, no iteration
    i64, i32, ib = bench.var_counts(n1, 99, 99, "inverse")
    assert i32 == 0.0 and i64 == pytest.approx(2 * (12 * n1 + NA) * NA + face)
    with pytest.raises(ValueError):
        bench.var_counts(n1, 0, 0, "fp16")


def test_alu_roofline_picks_the_largest_fraction(monkeypatch):
    monkeypatch.setattr(bench, "hbm_peak_gbs", lambda: (8000.0, "test"))
    # FP64-bound: 1 TFLOP in 1 s against 8 GB/s of traffic
    r = bench.alu_roofline(1e12, 0.0, 8e9, 1.0, 1.0)
    assert r["bound"] == "alu" and r["resource"] == "fp64" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(1.0) and r["frac"] == pytest.approx(1.0 / bench.FP64_PEAK_TFLOPS)
    assert r["frac_fp64_of_probe"] == pytest.approx(1.0) and "frac_fp32" not in r
    # HBM-bound: 7.2 TB in 1 s
    r = bench.alu_roofline(1e9, 0.0, 7.2e12, 1.0, None)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["frac"] == pytest.approx(0.9)
    assert r["achieved"] == pytest.approx(7200.0) and r["frac_fp64_of_probe"] is None
    # FP32-bound: 60 TFLOP of FP32 beside 0.1 TFLOP of FP64
    r = bench.alu_roofline(1e11, 6e13, 1e9, 1.0, 1.0)
    assert r["resource"] == "fp32" and r["frac"] == pytest.approx(60.0 / bench.FP32_PEAK_TFLOPS)
    assert r["frac"] == max(r["frac_fp64"], r["frac_fp32"], r["frac_hbm"])


@pytest.mark.parametrize("n,N", [(1, 2), (2, 3), (3, 4), (4, 8), (2, 7)])
def test_coarse_nodes_are_fine_nodes(n, N):
    idx = bench.coarse_in_fine(n, N)
    assert idx.size == n * n * (N + 1) ** 2 and idx.min() >= 0 and idx.max() < (2 * n) ** 2 * (N + 1) ** 2
    # the same points to rounding (the node coordinates are computed, on the
    # Cartesian and on the sine-mapped square)
    for nodes, tol in ((inputs.cartesian_nodes, 4e-16), (lambda s, N: inputs.mapped_nodes(s, N, 0.05), 4e-16)):
        Xf, Yf = nodes((2 * n, 2 * n), N)
        X, Y = nodes((n, n), N)
        assert np.abs(Xf.ravel()[idx] - X.ravel()).max() <= tol
        assert np.abs(Yf.ravel()[idx] - Y.ravel()).max() <= tol
    # a coarse face node is shared by two coarse elements: both map to one
    # fine point (the same coordinates), so distinct coarse points hit
    # distinct fine points
    X, Y = inputs.cartesian_nodes((n, n), N)
    pts = {(round(x, 12), round(y, 12)) for x, y in zip(X.ravel(), Y.ravel())}
    fine_pts = {(round(x, 12), round(y, 12))
                for x, y in zip(inputs.cartesian_nodes((2 * n, 2 * n), N)[0].ravel()[idx],
                                inputs.cartesian_nodes((2 * n, 2 * n), N)[1].ravel()[idx])}
    assert pts == fine_pts


def test_reference_arm_json_line(monkeypatch, capsys):
    """--impl reference prints one JSON line with the contract's keys; its
    value is DOF x RK4 steps / seconds over the timed samples only."""
    import argparse
    import json
    monkeypatch.setattr(bench, "_oracle_steps", lambda n, target, threads: ([(3, 1.5)] * 2 + [(4, 1.0)] * (n - 2), None))
    monkeypatch.setattr(bench, "_env_rank", lambda: (0, 1, 0))
    args = argparse.Namespace(steps=3, warmup=2, gpus=1)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == "DOF-steps/s" and line["steps"] == 3
    assert line["value"] == pytest.approx(bench.dof() * 12 / 3.0)     # the 3 timed samples: 4 steps / 1 s each
    assert line["ms_per_step"] == pytest.approx(1000.0)
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    # other ranks print nothing
    monkeypatch.setattr(bench, "_env_rank", lambda: (1, 2, 1))
    assert bench.run_reference(args) == 0 and capsys.readouterr().out == ""


def test_oracle_timer_runs_on_the_host():
    """The oracle timer subprocess steps the full headline mesh at least once
    per sample and reports positive times."""
    rows, err = bench._oracle_steps(1, 0.05, 1)
    assert err is None and len(rows) == 1 and rows[0][0] >= 1 and rows[0][1] > 0


def test_clock_sampler_parses_nvidia_smi_rows():
    """The clocks record of the bench line: median SM clock under load, the
    maximum clock, and every throttle reason seen active; malformed rows are
    skipped, and a missing nvidia-smi is reported, not raised."""
    import tempfile

    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc = FakeProc()
    s.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.f.write("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n"
              "0, 2055, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
              "garbage line\n")
    rec = s.stop()
    assert rec["sm_mhz"] == 2055.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
    s2 = bench.ClockSampler(0)
    assert s2.stop()["reasons"] == ["nvidia-smi unavailable"]

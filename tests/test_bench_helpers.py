"""bench.py's host-side arithmetic, on the CPU: whole-job rates over ranks, the roofline figures of the
Heun and implicit lines, and the step schedules the oracle legs use."""
from __future__ import annotations

import importlib.util
import math
import os

import pytest

import oracle as O
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class Args:
    precision = "fp32"


def test_whole_job_rate_and_single_rank_max(bench):
    # 4 replicas of 1000 units for 10 steps in 20 ms (the slowest rank): 2e6 units/s
    assert bench.whole_job_rate(1000, 10, 4, 20.0) == pytest.approx(2.0e6)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5


def test_heun_roofline_counts_20_bytes_per_update(bench):
    wl = synth.LATTICE_448
    r = bench.heun_tc_roofline(wl, 2.0, 2)
    updates = wl.nx * wl.ny * wl.Q
    assert r["achieved"] == pytest.approx(20.0 * updates / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["kernel"].startswith("step_tc3_kernel")
    assert bench.heun_tc_roofline(wl, 2.0, 0)["kernel"].startswith("step_tc2_kernel")


def test_tensor_peak_of_each_operand_type(bench):
    # BF16 and BF16X3 against the BF16 peak; TF32 against it times the nominal 1.1 / 2.25
    bf, _ = bench.bf16_peak()
    assert bench.tensor_peak("bf16")[0] == bench.tensor_peak("bf16x3")[0] == bf
    tf, src = bench.tensor_peak("tf32")
    assert tf == pytest.approx(bf * 1.1 / 2.25) and "tf32" in src
    assert set(bench.TENSOR_PRECISIONS) == {"bf16", "bf16x3", "tf32", "bf16x2"}
    assert bench.TENSOR_PASSES == {"bf16": 1, "bf16x3": 3, "tf32": 1, "bf16x2": 2}
    assert bench.tensor_peak("bf16x2")[0] == bf
    assert bench.BYTES_PER_UPDATE["tf32"] == bench.BYTES_PER_UPDATE["bf16x2"] == 8


def test_implicit_roofline_counts_source_iterations(bench):
    wl = synth.PAPER_LINE_SOURCE_200_IMPLICIT
    stats = {"source_iterations": 420, "gmres_iterations": 20, "sweeps": 420}
    r = bench.implicit_roofline(Args(), wl, 10.0, stats, 10)
    assert r["source_iterations_per_step"] == 42 and r["gmres_iterations_per_step"] == 2
    # per source iteration every value is read once and written once: 2 x 4 bytes (FP32)
    assert r["achieved"] == pytest.approx(8.0 * wl.nx * wl.ny * wl.Q * 42 / 10e-3 / 1e9)


def test_oracle_steps_take_095_of_the_admissible_dt_for_heun(bench):
    wl = synth.paper_line_source(40)
    n, dt = bench.oracle_steps(wl)
    Om, w, K = bench.oracle_parts(wl)
    sa, ss, q = wl.materials()
    bound = O.heun_admissible_dt(Om, K, sa, ss, wl.sigma_as, wl.h)
    assert dt <= 0.95 * bound * (1 + 1e-12)
    assert n * dt == pytest.approx(wl.t_final)
    assert math.ceil(wl.t_final / (0.95 * bound) - 1e-12) == n


def test_oracle_steps_of_euler_and_implicit_workloads_use_the_cfl_number(bench):
    for wl in (synth.LINE_SOURCE_64, synth.paper_line_source_implicit(40)):
        assert bench.oracle_steps(wl) == wl.steps()
    n, dt = synth.paper_line_source_implicit(40).steps()
    assert dt == pytest.approx(1.0 / math.ceil(1.0 / (2.0 * 3.0 / 40)))

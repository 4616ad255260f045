"""Throughput of the explicit as-S_N step on GB300: cell-ordinate updates per second.

Default workload: the 448 x 448-cell lattice with 16 x 32 = 512 ordinates (beta = 0.5 scaled by
the ordinate spacing, sigma_as = 5, CFL 0.5), state in FP32, artificial-scattering contraction
on the tensor cores in BF16 (FP32 accumulation).  A "step" is one explicit time step of the whole
grid (one fused kernel launch).  Synthetic, seeded inputs; the state (822 MB) is larger than L2,
so consecutive steps stream it from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|bf16x3|fp32|fp64]
    python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

Prints one JSON line.  Under torchrun (N > 1) every rank advances its own independent replica of
the workload (there is no data exchange between solves); rank 0 prints the line with the max
time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "cell-ordinate updates/s"
BYTES_PER_UPDATE = {"fp64": 16, "fp32": 8, "bf16": 8, "bf16x3": 8}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "bf16x3", "fp32", "fp64"])
    ap.add_argument("--workload", default=synth.LATTICE_448.name, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64/e2e/CPU legs")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--tile", type=int, default=0, help="tensor-core tile cells (0 = automatic)")
    ap.add_argument("--stages", type=int, default=0, help="tensor-core kernel-matrix ring depth (0 = automatic)")
    ap.add_argument("--variant", type=int, default=0, help="tensor-core kernel: 0 persistent, 1 one tile per CTA")
    return ap.parse_args()


def kernel_traffic(precision: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source still matches."""
    import hashlib
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["step_tc2_kernel"]
        src = b"".join(open(os.path.join(ROOT, "paper_1911_08801_gb300", "csrc", f), "rb").read()
                       for f in ("step_tc2.cu", "tc_ptx.h"))
        if hashlib.sha256(src).hexdigest()[:16] != d["source_sha256_16"] or precision != d["precision"]:
            return None
        return d["dram_bytes_per_launch"]
    except Exception:
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_problem(A, wl, precision, stream):
    p = A.Problem(wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, precision, stream=stream)
    p.set_product_quadrature(wl.n_polar, wl.n_azim)
    sa, ss, q = wl.materials()
    p.set_cross_sections(sa, ss, q)
    p.set_artificial_scattering(wl.sigma_as, wl.eps)
    return p


def seeded_state_f32(wl, seed=0):
    rng = np.random.default_rng(seed)
    return rng.random((wl.ny, wl.nx, wl.Q), dtype=np.float32)


def run_ours(args, rank, world, dist):
    import torch

    import paper_1911_08801_gb300 as A
    from paper_1911_08801_gb300 import _lib as L

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    wl = synth.WORKLOADS[args.workload]
    n_total, dt = wl.steps()
    stream = torch.cuda.Stream()
    prob = make_problem(A, wl, args.precision, stream)
    tiling = None
    if args.precision.startswith("bf16"):
        prob.set_tiling(args.tile, args.stages, args.variant)
        tiling = prob.tiling()
    psi0 = torch.from_numpy(seeded_state_f32(wl, seed=rank)).pin_memory().numpy()
    if args.precision == "fp64":
        prob.set_state(psi0.astype(np.float64))
    else:
        L.assn_set_state_f32(prob.handle, psi0)
    torch.cuda.synchronize()
    units = wl.nx * wl.ny * wl.Q

    for _ in range(args.warmup):
        prob.step(1, dt)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = prob.launch_count()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.steps):
            prob.step(1, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = prob.launch_count() - launches0
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    value = units * args.steps * world / (ms / 1e3)

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = extras_legs(A, L, torch, wl, args, prob, psi0, stream, dt)
    hbm, src = peaks()
    achieved = BYTES_PER_UPDATE[args.precision] * units / (ms_per_step / 1e3) / 1e9
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"bf16": "bf16 contraction, fp32 state", "bf16x3": "bf16x3 contraction, fp32 state",
                  "fp32": "fp32", "fp64": "f64"}[args.precision],
        "data": "synthetic (seeded uniform state, analytic lattice materials)",
        "config": {"workload": wl.name, "cells": f"{wl.nx}x{wl.ny}", "Q": wl.Q, "beta": wl.beta,
                   "eps": wl.eps, "sigma_as": wl.sigma_as, "dt": dt, "precision": args.precision,
                   "l2": "state larger than L2 (%.0f MB per buffer)" % (units * 4 / 1e6),
                   "parallelism": f"replicas x{world}", "tiling": tiling},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm,
                     "traffic": kernel_traffic(args.precision) if args.variant == 0 and args.workload == synth.LATTICE_448.name else None,
                     "peak_source": f"{src} hbm_gbs", "bytes_per_update": BYTES_PER_UPDATE[args.precision],
                     "kernel": ("step_tc2_kernel" if args.variant == 0 else "step_tc_kernel") if args.precision.startswith("bf16")
                     else "step_simt_kernel"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "wall_s_timed": wall,
    }
    line.update(extras)
    prob.close()
    return line


def extras_legs(A, L, torch, wl, args, prob, psi0, stream, dt):
    """e2e through the public API with host buffers, the FP64 GPU path, and the CPU oracle."""
    out = {}
    units = wl.nx * wl.ny * wl.Q
    # e2e: one assn_run_f32 call = upload psi0 from pinned host memory, n steps, scalar flux to host
    if args.precision != "fp64":
        n_e2e = 20
        phi = np.empty((wl.ny, wl.nx))
        L.assn_run_f32(prob.handle, psi0, 2, dt, phi)
        reps = 3
        t0 = time.perf_counter()
        for _ in range(reps):
            L.assn_run_f32(prob.handle, psi0, n_e2e, dt, phi)
        el = (time.perf_counter() - t0) / reps
        out["e2e"] = {"value": units * n_e2e / el, "unit": "updates/s",
                      "h2d_bytes_per_step": int(psi0.nbytes) // n_e2e, "d2h_bytes_per_step": int(phi.nbytes) // n_e2e,
                      "call": f"assn_run_f32: pinned host psi0 -> {n_e2e} steps -> host Phi",
                      "ms_per_call": el * 1e3}
    # the plain FP64 GPU path on the same workload
    try:
        p64 = make_problem(A, wl, "fp64", stream)
        p64.set_state(psi0.astype(np.float64))
        p64.step(1, dt)
        torch.cuda.synchronize()
        k = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p64.step(k, dt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        out["fp64_gpu_path"] = {"value": units / (ms / 1e3), "unit": "updates/s", "ms_per_step": ms,
                                "kernel": "step_simt_kernel<double>"}
        p64.close()
    except Exception as e:  # pragma: no cover - report, do not hide
        out["fp64_gpu_path"] = {"error": str(e)}
    out["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    return out


def cpu_baseline(wl, seconds: float):
    """The FP64 oracle as it stands, timed on the host cores on a bounded strip of the workload."""
    import oracle as O

    Om, w = O.product_quadrature(wl.n_polar, wl.n_azim)
    K = O.kernel_matrix(Om, w, wl.eps)
    sa, ss, q = wl.materials()
    rows = max(1, min(wl.ny, 8))
    rng = np.random.default_rng(0)
    psi = rng.random((rows, wl.nx, wl.Q))
    _, dt = wl.steps()
    O.step(psi, K, Om, w, sa[:rows], ss[:rows], q[:rows], wl.sigma_as, wl.h, dt)
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds or n == 0:
        psi = O.step(psi, K, Om, w, sa[:rows], ss[:rows], q[:rows], wl.sigma_as, wl.h, dt)
        n += 1
    el = time.perf_counter() - t0
    units = rows * wl.nx * wl.Q * n
    return {"value": units / el, "unit": "updates/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} steps of a {rows}-row strip ({rows}x{wl.nx} cells, Q={wl.Q}) of {wl.name}, numpy FP64"}


def run_reference(args):
    """The FP64 CPU oracle stepped on a bounded strip of the workload (the reference arm)."""
    import oracle as O

    wl = synth.WORKLOADS[args.workload]
    Om, w = O.product_quadrature(wl.n_polar, wl.n_azim)
    K = O.kernel_matrix(Om, w, wl.eps)
    sa, ss, q = wl.materials()
    _, dt = wl.steps()
    rows = 4
    rng = np.random.default_rng(0)
    psi = rng.random((rows, wl.nx, wl.Q))
    for _ in range(args.warmup):
        psi = O.step(psi, K, Om, w, sa[:rows], ss[:rows], q[:rows], wl.sigma_as, wl.h, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi = O.step(psi, K, Om, w, sa[:rows], ss[:rows], q[:rows], wl.sigma_as, wl.h, dt)
    el = time.perf_counter() - t0
    units = rows * wl.nx * wl.Q * args.steps
    value = units / el
    sample = f"each step: a {rows}-row strip ({rows}x{wl.nx} cells, Q={wl.Q}) of {wl.name}, numpy FP64"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded uniform state, analytic lattice materials)",
            "config": {"workload": wl.name, "cells": f"{wl.nx}x{wl.ny}", "Q": wl.Q, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        td.init_process_group("nccl")
        dist = td
    line = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

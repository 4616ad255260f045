"""Batched stepping (include/assn.h, assn_batch_*): several uneven as-S_N problems advanced by one
persistent launch per step, optionally replayed as a CUDA graph, with the tiling autotuner.

The bar: every member of a batch ends bitwise equal to the same problem stepped alone at the same
tile width (the per-element arithmetic and its order do not depend on which other problems share
the launch), members finish at their own step counts, and a member agrees with the FP64 oracle
within the whole-run tolerance of its precision.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from helpers import RUN_TOL, ensure_built, gpu_problem, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


# uneven grids (ragged last tiles), ordinate counts 64 / 128 / 256 / 512 and kernel widths
SPECS = [(24, 24, 8, 8, 0.3), (40, 32, 8, 16, 0.7), (56, 56, 16, 16, 0.5), (33, 21, 16, 32, 0.9)]


def workloads(seed: int = 11):
    out = []
    for k, (nx, ny, npol, naz, beta) in enumerate(SPECS):
        out.append(synth.Workload(f"batch{k}", "random", nx, ny, 0.0, 0.05 * nx, 0.0, 0.05 * ny, npol, naz, beta,
                                  seed=seed + k))
    return out


def build(A, precision, wls):
    probs = [gpu_problem(A, wl, precision) for wl in wls]
    dts = [0.9 * p.max_stable_dt() for p in probs]
    return probs, dts


def paired(wl):
    """Members whose steps run on the paired-SM kernel (256 or 512 padded ordinates): a batch steps
    them with their own launches, not in an ordinate class."""
    return (wl.Q + 63) // 64 * 64 in (256, 512)


def launches_per_run(wls, steps):
    """One launch per step of each class of members with the same padded ordinate count, and one per
    step of each paired member."""
    cls, own = {}, 0
    for wl, n in zip(wls, steps):
        if paired(wl):
            own += n
            continue
        mp = (wl.Q + 63) // 64
        cls[mp] = max(cls.get(mp, 0), n)
    return sum(cls.values()) + own


def alone(A, precision, wl, nsteps, dt, tile_cells, in_class=False):
    """The member's solve stepped alone: on the paired-SM kernel where it steps there in a batch,
    else on the one-CTA kernel at the class's tile width."""
    p = gpu_problem(A, wl, precision)
    if in_class or not paired(wl):
        p.set_tiling(tile_cells=tile_cells)
    p.step(nsteps, dt)
    s = p.state()
    p.close()
    return s


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_members_equal_alone(A, precision, use_graph):
    wls = workloads()
    probs, dts = build(A, precision, wls)
    steps = [3, 5, 0, 4]
    with A.Batch() as b:
        for p, n, dt in zip(probs, steps, dts):
            b.add(p, n, dt)
        b.run(use_graph=use_graph).sync()
        info = b.info()
    assert info["members"] == 4 and info["launches"] == launches_per_run(wls, steps)
    for wl, p, n, dt in zip(wls, probs, steps, dts):
        ref = alone(A, precision, wl, n, dt, info["tile_cells"])
        got = p.state()
        assert np.array_equal(got, ref), (wl.name, n, float(np.abs(got - ref).max()))
    for p in probs:
        p.close()


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_one_launch_per_step_for_uneven_ordinate_counts(A, precision, use_graph):
    """Members with Q = 64, 128, 256 and 512 in a single class: every step of the batch is one
    launch (the runtime-stride kernel instance), and every member still equals its solve alone at
    the class's tile width, bitwise."""
    wls = workloads(seed=61)
    probs, dts = build(A, precision, wls)
    steps = [3, 2, 4, 1]
    with A.Batch() as b:
        b.set_grouping(True)
        for p, n, dt in zip(probs, steps, dts):
            b.add(p, n, dt)
        b.run(use_graph=use_graph).sync()
        info = b.info()
        cls = b.classes()
    assert len(cls) == 1 and cls[0]["members"] == 4 and cls[0]["ordinate_stride"] == 512
    assert info["launches"] == max(steps)
    for wl, p, n, dt in zip(wls, probs, steps, dts):
        ref = alone(A, precision, wl, n, dt, info["tile_cells"], in_class=True)
        assert np.array_equal(p.state(), ref), wl.name
    for p in probs:
        p.close()


def test_rerun_graph_reuse_and_continue(A):
    """Two runs of the same batch (the graph is replayed) equal 2 n steps alone; stepping a member
    on its own afterwards continues from the batch's result."""
    wls = workloads(seed=23)
    probs, dts = build(A, "bf16", wls)
    steps = [2, 1, 3, 2]
    with A.Batch() as b:
        for p, n, dt in zip(probs, steps, dts):
            b.add(p, n, dt)
        b.run().run().sync()
        nt = b.info()["tile_cells"]
        assert b.info()["launches"] == 2 * launches_per_run(wls, steps)
        cls = b.classes()
        assert [c["ordinate_stride"] for c in cls] == [128, 64]   # Q = 256 and 512 step on the paired kernel
        assert [c["members"] for c in cls] == [1, 1]
        assert all(c["tile_cells"] * c["ordinate_stride"] // 128 <= 256 for c in cls)
    probs[0].step(1, dts[0])   # a class member and a paired member continue on their own
    probs[3].step(1, dts[3])
    for k, (wl, p, n, dt) in enumerate(zip(wls, probs, steps, dts)):
        total = 2 * n + (1 if k in (0, 3) else 0)
        ref = alone(A, "bf16", wl, total, dt, nt)
        assert np.array_equal(p.state(), ref), wl.name
    for p in probs:
        p.close()


def test_member_matches_oracle(A):
    wls = workloads(seed=31)
    probs, dts = build(A, "bf16", wls)
    nsteps = 6
    with A.Batch() as b:
        for p, dt in zip(probs, dts):
            b.add(p, nsteps, dt)
        b.run().sync()
    for wl, p, dt in zip(wls, probs, dts):
        psi_ref, w = oracle_run(wl, nsteps, dt)
        phi_ref = psi_ref @ w
        assert rel_l2(p.scalar_flux(), phi_ref) <= RUN_TOL["bf16"], wl.name
        p.close()


def test_remove_and_set_steps(A):
    wls = workloads(seed=41)
    probs, dts = build(A, "bf16", wls)
    before = probs[1].state()
    with A.Batch() as b:
        for p, dt in zip(probs, dts):
            b.add(p, 2, dt)
        b.remove(probs[1])
        b.set_steps(probs[2], 4, dts[2])
        b.run().sync()
        nt = b.info()["tile_cells"]
    assert np.array_equal(probs[1].state(), before)
    for k, (wl, p, dt) in enumerate(zip(wls, probs, dts)):
        if k == 1:
            continue
        n = 4 if k == 2 else 2
        assert np.array_equal(p.state(), alone(A, "bf16", wl, n, dt, nt)), wl.name
    for p in probs:
        p.close()


def test_autotune_keeps_state(A):
    wls = workloads(seed=53)
    probs, dts = build(A, "bf16", wls)
    states = [p.state() for p in probs]
    with A.Batch() as b:
        for p, dt in zip(probs, dts):
            b.add(p, 2, dt)
        t = b.autotune(use_cache=False)
        assert t["tile_cells"] in (32, 64) and t["ms_per_launch"] > 0
        for p, s in zip(probs, states):
            assert np.array_equal(p.state(), s)
        cached = b.autotune(use_cache=True)
        assert cached["tile_cells"] == t["tile_cells"] and cached["ms_per_launch"] == -1.0
        b.run().sync()
        assert b.info()["tile_cells"] == t["tile_cells"]
    for wl, p, dt in zip(wls, probs, dts):
        assert np.array_equal(p.state(), alone(A, "bf16", wl, 2, dt, t["tile_cells"])), wl.name
        p.close()


def test_single_problem_autotune(A):
    wl = workloads(seed=61)[2]
    p = gpu_problem(A, wl, "bf16")
    dt = 0.9 * p.max_stable_dt()
    s0 = p.state()
    t = p.autotune(dt, use_cache=False)
    assert np.array_equal(p.state(), s0)
    assert p.tiling()["tile_cells"] == t["tile_cells"]
    p.step(3, dt)   # (a tuned tiling selects the one-CTA kernel)
    assert np.array_equal(p.state(), alone(A, "bf16", wl, 3, dt, t["tile_cells"], in_class=True))
    p.close()


def test_batch_errors(A):
    wls = workloads(seed=71)
    with A.Batch() as b:
        p32 = gpu_problem(A, wls[0], "fp32")
        with pytest.raises(A.AssnError) as ei:
            b.add(p32, 1, 0.9 * p32.max_stable_dt())
        assert ei.value.status == A._lib.ASSN_ERR_UNSUPPORTED
        p1 = gpu_problem(A, wls[0], "bf16")
        dt = 0.9 * p1.max_stable_dt()
        with pytest.raises(A.AssnError) as ei:
            b.add(p1, 1, 10.0 * dt / 0.9)
        assert ei.value.status == A._lib.ASSN_ERR_UNSTABLE
        b.add(p1, 1, dt)
        with pytest.raises(A.AssnError) as ei:
            b.add(p1, 1, dt)
        assert ei.value.status == A._lib.ASSN_ERR_ARG
        p3 = gpu_problem(A, wls[1], "bf16x3")
        with pytest.raises(A.AssnError) as ei:
            b.add(p3, 1, 0.9 * p3.max_stable_dt())
        assert ei.value.status == A._lib.ASSN_ERR_ARG
        with pytest.raises(A.AssnError):
            b.set_tiling(tile_cells=48)
        with pytest.raises(A.AssnError):
            b.add(p1, -1, dt)
        for p in (p32, p1, p3):
            p.close()


def test_result_independent_of_tile_width(A):
    """The per-element arithmetic (contraction order over ordinate chunks, scalar-flux reduction) does
    not depend on how many cells a tile holds, so tile widths give bitwise equal states."""
    wl = workloads(seed=83)[2]   # 56 x 56 cells, Q = 256 (ragged last tile at every width)
    dt = None
    out = []
    for nt in (32, 64, 128):
        p = gpu_problem(A, wl, "bf16")
        dt = dt or 0.9 * p.max_stable_dt()
        p.set_tiling(tile_cells=nt)
        p.step(3, dt)
        out.append(p.state())
        p.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_result_independent_of_rings(A):
    """Ring depths and kernel-matrix request sizes change only the pipelining, not the arithmetic."""
    wl = workloads(seed=89)[3]   # 33 x 21 cells, Q = 512 (four ordinate blocks)
    out = []
    dt = None
    for rings in ((0, 0, 0, 0), (2, 2, 2, 1), (3, 3, 3, 2), (2, 3, 2, 4)):
        p = gpu_problem(A, wl, "bf16")
        dt = dt or 0.9 * p.max_stable_dt()
        p.set_rings(*rings)
        got = p.rings()
        if rings[0]:
            assert (got["staging"], got["operand"], got["kernel_matrix"], got["blocks_per_request"]) == rings
        p.step(3, dt)
        out.append(p.state())
        p.close()
    for o in out[1:]:
        assert np.array_equal(out[0], o)


# members whose every step runs on the paired-SM kernel: 256 / 512 (and padded 200 / 500) ordinates
PAIRED_SPECS = [(33, 21, 16, 32, 0.9), (40, 17, 16, 16, 0.5), (24, 30, 10, 20, 0.7), (19, 26, 10, 50, 0.4)]


@pytest.mark.parametrize("precision", ["tf32", "bf16x2"])
@pytest.mark.parametrize("scheme", ["euler", "heun"])
@pytest.mark.parametrize("use_graph", [True, False])
def test_paired_precision_batch_equals_alone(A, precision, scheme, use_graph):
    """TF32 and BF16X2 have the paired-SM kernel only; a batch of members that all run there steps
    each by its own chain of launches, and every member ends bitwise equal to its solve alone.  The
    batch's info and autotune work with no one-CTA class."""
    wls = [synth.Workload(f"pbatch{k}", "random", nx, ny, 0.0, 0.05 * nx, 0.0, 0.05 * ny, npol, naz, beta, seed=40 + k)
           for k, (nx, ny, npol, naz, beta) in enumerate(PAIRED_SPECS)]
    probs = []
    for wl in wls:
        p = gpu_problem(A, wl, precision)
        p.set_scheme(scheme)
        probs.append(p)
    dts = [0.9 * p.max_stable_dt() for p in probs]
    steps = [3, 5, 0, 2]
    with A.Batch() as b:
        for p, n, dt in zip(probs, steps, dts):
            b.add(p, n, dt)
        b.autotune()
        b.run(use_graph=use_graph).sync()
        info = b.info()
    lps = 2 if scheme == "heun" else 1
    assert info["members"] == 4 and info["launches"] == lps * sum(steps) and info["total_tiles"] == 0
    for wl, p, n, dt in zip(wls, probs, steps, dts):
        q = gpu_problem(A, wl, precision)
        q.set_scheme(scheme)
        q.step(n, dt)
        ref = q.state()
        q.close()
        assert np.array_equal(p.state(), ref), (wl.name, n)
    for p in probs:
        p.close()


@pytest.mark.parametrize("precision", ["tf32", "bf16x2"])
def test_paired_precision_batch_refusals(A, precision):
    """A TF32 / BF16X2 member without a paired-SM form (Q = 128) is refused when added, and the
    one-launch grouping (every member on the one-CTA kernel) is refused when the batch runs."""
    U = A._lib.ASSN_ERR_UNSUPPORTED
    small = synth.Workload("pb_small", "random", 20, 20, 0.0, 1.0, 0.0, 1.0, 8, 16, 0.5, seed=1)
    big = synth.Workload("pb_big", "random", 20, 20, 0.0, 1.0, 0.0, 1.0, 16, 32, 0.5, seed=2)
    p, q = gpu_problem(A, small, precision), gpu_problem(A, big, precision)
    with A.Batch() as b:
        with pytest.raises(A.AssnError) as e:
            b.add(p, 1, 0.5 * p.max_stable_dt())
        assert e.value.status == U
        b.add(q, 1, 0.5 * q.max_stable_dt())
        b.set_grouping(one_launch=True)
        with pytest.raises(A.AssnError) as e:
            b.run()
        assert e.value.status == U
    p.close()
    q.close()

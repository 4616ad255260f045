"""Serving loop (include/assn.h, assn_server_*): admission by device-memory footprint, continuous
batching of whole solves, latency statistics.

The bar: every request's scalar flux is bitwise equal to the same solve stepped alone with
assn_step (its launches are shared with other solves but its per-element arithmetic is not),
admission never exceeds the footprint budget, and failures stay with their own request.
"""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import synth
from helpers import ensure_built, gpu_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


def request_workloads(seed: int = 3, count: int = 8):
    """Small line-source / lattice / random solves of uneven size, Q and kernel width."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        Q = int(rng.choice([64, 128, 256, 512]))
        npol, naz = synth.QUAD_ORDERS[Q]
        beta = float(rng.uniform(0.1, 1.0))
        kind = ["line_source", "lattice", "random"][k % 3]
        if kind == "line_source":
            n = int(rng.choice([16, 24, 40]))
            wl = synth.line_source(n, npol, naz, beta, t_final=0.2, name=f"req{k}")
        elif kind == "lattice":
            wl = synth.lattice(int(rng.choice([14, 28])), npol, naz, beta, t_final=0.3, name=f"req{k}")
        else:
            nx, ny = int(rng.integers(8, 40)), int(rng.integers(8, 40))
            wl = synth.Workload(f"req{k}", "random", nx, ny, 0.0, 0.05 * nx, 0.0, 0.05 * ny, npol, naz, beta,
                                seed=seed + k)
        out.append(wl)
    return out


def steps_for(A, wl, precision="bf16"):
    """Step count and size: CFL 0.5 capped at 0.9 of the positivity bound, ending at t_final."""
    p = gpu_problem(A, wl, precision)
    dmax = p.max_stable_dt()
    p.close()
    h = wl.h
    dt0 = min(wl.cfl * h, 0.9 * dmax)
    n = max(1, int(np.ceil(wl.t_final / dt0 - 1e-12)))
    return n, wl.t_final / n


def submit(srv, wl, nsteps, dt):
    sa, ss, q = wl.materials()
    init = wl.psi0().astype(np.float32) if wl.kind != "line_source" else "line_source"
    if wl.kind == "lattice":
        init = "zero"
    return srv.submit(wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, wl.n_polar, wl.n_azim, wl.sigma_as, wl.eps,
                      sa, ss, q, nsteps, dt, init=init)


def alone_phi(A, wl, nsteps, dt, precision="bf16"):
    """The same solve stepped alone with assn_step on its default kernel (the paired-SM kernel at 256 /
    512 ordinates, which the server's batches launch per solve; else the one-CTA kernel)."""
    p = A.Problem(wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, precision)
    p.set_product_quadrature(wl.n_polar, wl.n_azim)
    sa, ss, q = wl.materials()
    p.set_cross_sections(sa, ss, q)
    p.set_artificial_scattering(wl.sigma_as, wl.eps)
    if wl.kind == "line_source":
        p.init_line_source()
    elif wl.kind == "random":
        p.set_state(wl.psi0().astype(np.float32).astype(np.float64))
    p.step(nsteps, dt)
    phi = p.scalar_flux()
    p.close()
    return phi


@pytest.mark.parametrize("chunk,use_graph", [(4, True), (3, False)])
def test_mix_equals_alone(A, chunk, use_graph):
    # A long first request (tens of chunks) keeps the device busy while the rest are submitted, so
    # the others join it in shared launches: the results below are checked in the mix, not alone.
    wls = [synth.line_source(40, 16, 32, 0.5, t_final=2.0, name="lead")] + request_workloads()
    plan = [steps_for(A, wl) for wl in wls]
    assert plan[0][0] >= 10 * chunk
    with A.Server("bf16", max_active=5, chunk_steps=chunk, use_graph=use_graph) as srv:
        ids = [submit(srv, wl, n, dt) for wl, (n, dt) in zip(wls, plan)]
        results = [srv.wait(i, timeout_s=120.0) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(wls) and st["failed"] == 0
    assert 2 <= st["max_active_seen"] <= 5
    assert st["p50_latency_s"] <= st["p99_latency_s"]
    assert st["updates"] == sum(wl.nx * wl.ny * wl.Q * n for wl, (n, _) in zip(wls, plan))
    for wl, (n, dt), (phi, lat, qs) in zip(wls, plan, results):
        assert lat >= qs >= 0.0
        ref = alone_phi(A, wl, n, dt)
        assert np.array_equal(phi, ref), (wl.name, float(np.abs(phi - ref).max()))


def test_admission_by_footprint(A):
    """A budget that holds one of these solves at a time admits them one by one."""
    wls = [synth.line_source(48, 16, 32, 0.5, t_final=0.1, name=f"big{k}") for k in range(3)]
    fp = A._lib.assn_footprint_bytes(48, 48, 512, A.ASSN_BF16)
    plan = [steps_for(A, wl) for wl in wls]
    with A.Server("bf16", hbm_budget_bytes=int(1.5 * fp), max_active=8, chunk_steps=2) as srv:
        ids = [submit(srv, wl, n, dt) for wl, (n, dt) in zip(wls, plan)]
        res = [srv.wait(i, timeout_s=120.0) for i in ids]
        st = srv.stats()
        with pytest.raises(A.AssnError) as ei:   # larger than the whole budget
            submit(srv, synth.line_source(96, 16, 32, 0.5, t_final=0.1), 1, 1e-3)
        assert ei.value.status == A._lib.ASSN_ERR_OOM
    assert st["max_active_seen"] == 1 and st["peak_bytes"] <= st["budget_bytes"]
    for wl, (n, dt), (phi, _, _) in zip(wls, plan, res):
        assert np.array_equal(phi, alone_phi(A, wl, n, dt))


def test_failure_stays_with_its_request(A):
    wls = request_workloads(seed=9, count=3)
    plan = [steps_for(A, wl) for wl in wls]
    with A.Server("bf16", max_active=4, chunk_steps=4) as srv:
        bad = submit(srv, wls[0], 2, 100.0)    # far above the positivity bound: fails at admission
        good = [submit(srv, wl, n, dt) for wl, (n, dt) in zip(wls, plan)]
        with pytest.raises(A.AssnError) as ei:
            srv.wait(bad, timeout_s=60.0)
        assert ei.value.status == A._lib.ASSN_ERR_UNSTABLE
        for wl, (n, dt), i in zip(wls, plan, good):
            phi, _, _ = srv.wait(i, timeout_s=120.0)
            assert np.array_equal(phi, alone_phi(A, wl, n, dt))
        st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 3


def test_concurrent_submitters(A):
    wls = request_workloads(seed=17, count=6)
    plan = [steps_for(A, wl) for wl in wls]
    out = {}
    with A.Server("bf16", max_active=3, chunk_steps=5) as srv:
        def worker(ks):
            for k in ks:
                rid = submit(srv, wls[k], *plan[k])
                out[k] = srv.wait(rid, timeout_s=120.0)[0]
        ts = [threading.Thread(target=worker, args=(ks,)) for ks in ([0, 2, 4], [1, 3, 5])]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    for k, wl in enumerate(wls):
        assert np.array_equal(out[k], alone_phi(A, wl, *plan[k])), wl.name


def test_cancel_queued_and_running(A):
    """One request cancelled while queued and one while on the device both end with
    ASSN_ERR_CANCELLED and leave the loop; the others' results stay equal to their solves alone."""
    lead = synth.line_source(40, 16, 32, 0.5, t_final=10.0, name="long")   # hundreds of one-step chunks
    n_lead, dt_lead = steps_for(A, lead)
    others = request_workloads(seed=21, count=3)
    plan = [steps_for(A, wl) for wl in others]
    with A.Server("bf16", max_active=1, chunk_steps=1) as srv:   # the others queue behind the lead
        rid = submit(srv, lead, n_lead, dt_lead)
        ids = [submit(srv, wl, n, dt) for wl, (n, dt) in zip(others, plan)]
        srv.cancel(ids[1])                                        # still queued
        t0 = time.time()
        while srv.stats()["active"] < 1 and time.time() - t0 < 60.0:
            time.sleep(0.005)
        srv.cancel(rid)                                           # on the device
        for i in (rid, ids[1]):
            with pytest.raises(A.AssnError) as ei:
                srv.wait(i, timeout_s=120.0)
            assert ei.value.status == A._lib.ASSN_ERR_CANCELLED
        for k in (0, 2):
            phi, _, _ = srv.wait(ids[k], timeout_s=120.0)
            assert np.array_equal(phi, alone_phi(A, others[k], *plan[k])), others[k].name
        with pytest.raises(A.AssnError) as ei:                   # collected: no longer known
            srv.cancel(ids[0])
        assert ei.value.status == A._lib.ASSN_ERR_ARG
        st = srv.stats()
    assert st["failed"] == 2 and st["completed"] == 2 and st["launches"] < n_lead

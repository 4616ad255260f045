"""Full-size parity of the batched and served launch configurations: members of the 64-solve ensemble
(sides up to 512, Q up to 512) in one batched launch, and a 1024^2 request through the serving loop,
each one step from a known state, compared with the FP64 oracle on sampled cells (corners, edges,
tile boundaries, random cells) -- the oracle cannot step these grids whole in a test's time."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
import synth
from helpers import ensure_built, offdiag_rowsum, step_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


def sample_cells(nx, ny, rng, extra=12):
    cells = {(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1), (ny // 2, nx // 2), (0, nx // 2), (ny // 2, 0),
             (ny - 1, nx // 3), (ny // 3, nx - 1)}
    for f in (63, 64, 127, 128, 255, 256):      # cells at tile boundaries of the row-major cell order
        if f < nx * ny:
            cells.add((f // nx, f % nx))
    cells |= {(int(j), int(i)) for j, i in zip(rng.integers(0, ny, extra), rng.integers(0, nx, extra))}
    return sorted(cells)


def oracle_parts(wl):
    Om, w = O.product_quadrature(wl.n_polar, wl.n_azim)
    K = O.kernel_matrix(Om, w, wl.eps)
    sa, ss, q = wl.materials()
    return Om, w, K, sa, ss, q


def test_ensemble_members_one_batched_launch(A):
    wls = [synth.ensemble(0)[k] for k in (0, 1, 3, 5, 6, 9)]   # Q 64 / 128 / 256 / 512, sides 126 .. 512
    rng = np.random.default_rng(17)
    states, probs, dts = [], [], []
    for wl in wls:
        psi = rng.random((wl.ny, wl.nx, wl.Q), dtype=np.float32)
        p = A.Problem(wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, "bf16")
        p.set_product_quadrature(wl.n_polar, wl.n_azim)
        p.set_cross_sections(*wl.materials())
        p.set_artificial_scattering(wl.sigma_as, wl.eps)
        A._lib.assn_set_state_f32(p.handle, psi)   # asynchronous: psi stays alive in `states`
        states.append(psi)
        probs.append(p)
        dts.append(0.9 * p.max_stable_dt())
    with A.Batch() as b:
        for p, dt in zip(probs, dts):
            b.add(p, 1, dt)
        b.run().sync()
        cls = b.classes()   # Q = 64 and 128 in one-CTA classes; Q = 256 and 512 on the paired-SM kernel
        assert sorted(c["ordinate_stride"] for c in cls) == [64, 128]
        assert sum(c["members"] for c in cls) == sum(1 for wl in wls if wl.Q < 256)
    for wl, p, psi, dt in zip(wls, probs, states, dts):
        got = p.state()
        Om, w, K, sa, ss, q = oracle_parts(wl)
        cells = sample_cells(wl.nx, wl.ny, rng)
        ref = O.step_at_cells(psi, cells, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
        tol = step_tolerance("bf16", dt, wl.sigma_as, 1.0, offdiag_rowsum(K))
        for n, (j, i) in enumerate(cells):
            assert np.abs(got[j, i] - ref[n]).max() <= tol, (wl.name, j, i)
        p.close()


def test_server_one_step_at_1024(A):
    """A 1024^2 line-source request (Q = 128) served with one step; Phi on sampled cells against the
    oracle's one-step update of the same initial state."""
    wl = synth.line_source(1024, 8, 16, 0.3, t_final=1.0)
    sa, ss, q = wl.materials()
    probe = A.Problem(wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, "bf16")
    probe.set_product_quadrature(wl.n_polar, wl.n_azim)
    probe.set_cross_sections(sa, ss, q)
    probe.set_artificial_scattering(wl.sigma_as, wl.eps)
    dt = 0.9 * probe.max_stable_dt()
    probe.close()
    with A.Server("bf16", max_active=4, chunk_steps=4) as srv:
        rid = srv.submit(wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, wl.n_polar, wl.n_azim, wl.sigma_as, wl.eps,
                         sa, ss, q, 1, dt, init="line_source")
        phi, lat, _ = srv.wait(rid, timeout_s=300.0)
    psi0 = wl.psi0()
    Om, w, K, sa, ss, q = oracle_parts(wl)
    rng = np.random.default_rng(23)
    cells = sample_cells(wl.nx, wl.ny, rng) + [(512, 512), (511, 512), (512, 511), (510, 509)]   # the peak
    ref = O.step_at_cells(psi0, cells, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt) @ w
    scale = float(psi0.max())
    tol = float(w.sum()) * step_tolerance("bf16", dt, wl.sigma_as, scale, offdiag_rowsum(K))
    for n, (j, i) in enumerate(cells):
        assert abs(phi[j, i] - ref[n]) <= tol, (j, i, phi[j, i], ref[n])

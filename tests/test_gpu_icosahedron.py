"""The paper's own setting for its explicit runs through the C ABI, against the FP64 oracle: the
icosahedron quadrature (Sec. 3.3; N_q = 92 at order 4), eps = beta / N_q, the row normalisation of
Sec. 3.2 and Heun + minmod (Sec. 3.1, 4.1) at 0.95 of its admissible dt, sigma_as = 5, beta = 4.5."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

import oracle as O
import synth
from helpers import (RUN_TOL, ensure_built, gpu_problem, offdiag_rowsum, oracle_run, oracle_setup, rel_l2,
                     run_steps, step_tolerance)

pytestmark = pytest.mark.gpu

PRECISIONS = ["fp64", "fp32", "bf16", "bf16x3"]


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


def test_problem_takes_the_generated_rule(A):
    for order, base in ((4, "printed"), (3, "regular"), (11, "printed")):
        p = A.Problem(8, 8, 0.0, 1.0, 0.0, 1.0, "bf16")
        p.set_icosahedron_quadrature(order, base)
        om, w = p.quadrature()
        ref_om, ref_w = O.icosahedron_quadrature(order, base)
        assert len(w) == 10 * (order - 1) ** 2 + 2 == p.Q
        d = np.linalg.norm(om[:, None, :] - ref_om[None, :, :], axis=2)
        m = d.argmin(1)
        assert d.min(1).max() < 1e-14 and len(set(m.tolist())) == len(w)
        assert np.abs(w - ref_w[m]).max() < 1e-14
        p.close()
    p = A.Problem(8, 8, 0.0, 1.0, 0.0, 1.0, "bf16")
    with pytest.raises(A.AssnError) as e:
        p.set_icosahedron_quadrature(12)          # N_q = 1212 > 1024
    assert e.value.status == A._lib.ASSN_ERR_ARG
    p.close()


def random_paper_workload(nx, ny, scheme, seed):
    wl = synth.paper_line_source(8)
    return dataclasses.replace(wl, name="random", kind="random", nx=nx, ny=ny, x0=0.0, x1=0.1 * nx, y0=0.0,
                               y1=0.1 * ny, seed=seed, scheme=scheme)


# ragged grids over several tiles; Q = 92 pads to 128 ordinates on the tensor-core path
@pytest.mark.parametrize("scheme", ["euler", "heun"])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_one_step_random_state(A, scheme, precision):
    """One step from a random state.  The library numbers the ordinates its own way, so the state is
    given to it in its order (ordinate i of the problem is ordinate m[i] of the oracle)."""
    wl = random_paper_workload(45, 19, scheme, seed=11 if scheme == "euler" else 12)
    psi0 = wl.psi0()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    p = gpu_problem(A, wl, precision)
    om_lib, _ = p.quadrature()
    d = np.linalg.norm(om_lib[:, None, :] - Om[None, :, :], axis=2)
    m = d.argmin(1)
    assert d.min(1).max() < 1e-14 and len(set(m.tolist())) == len(m)
    p.set_state(psi0[..., m])
    dt = 0.9 * p.max_stable_dt()
    p.step(1, dt)
    got = p.state()
    p.close()
    one = O.step_heun if scheme == "heun" else O.step
    ref = one(psi0, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)[..., m]
    scale = max(1.0, np.abs(ref).max(), np.abs(psi0).max())
    if precision == "fp64":
        tol = 1e-12 * scale
    elif precision == "fp32":
        tol = 2e-5 * scale
    else:
        tol = (2.0 if scheme == "heun" else 1.0) * step_tolerance(precision, dt, wl.sigma_as, scale, offdiag_rowsum(K))
    assert np.abs(got - ref).max() <= tol


@pytest.mark.parametrize("precision", PRECISIONS)
def test_paper_line_source_64(A, precision):
    """The paper's as-S_4 line source on a 64^2 grid, run to t = 1; the state stays non-negative."""
    wl = synth.paper_line_source(64)
    n, dt = run_steps(wl)
    p = gpu_problem(A, wl, precision)
    assert dt <= p.max_stable_dt()
    p.step(n, dt)
    phi = p.scalar_flux()
    p.close()
    ref, w = oracle_run(wl, n, dt)
    assert rel_l2(phi, ref @ w) <= RUN_TOL[precision]
    assert phi.min() >= -1e-6 * phi.max()
    if precision == "fp64":
        # the printed quadrature is closed under x -> -x with equal weights: Phi is even in x
        assert np.abs(phi - phi[:, ::-1]).max() <= 1e-12 * np.abs(phi).max()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_paper_lattice_28(A, precision):
    """The paper's explicit as-S_4 lattice (Sec. 4.2: absorbers, source block, N_q = 92, row
    normalisation, Heun + minmod) on a 28^2 grid (4 cells per block), run to t = 3.2."""
    wl = synth.paper_lattice(28)
    n, dt = run_steps(wl)
    p = gpu_problem(A, wl, precision)
    p.step(n, dt)
    phi = p.scalar_flux()
    p.close()
    ref, w = oracle_run(wl, n, dt)
    assert rel_l2(phi, ref @ w) <= RUN_TOL[precision]
    assert phi.min() >= 0.0


@pytest.fixture(scope="module")
def oracle_200():
    """The oracle's scalar flux after the first 12 steps of the paper's 200^2 as-S_4 run."""
    wl = synth.PAPER_LINE_SOURCE_200
    n, dt = run_steps(wl)
    psi, w = oracle_run(wl, 12, dt)
    return dt, psi @ w


@pytest.mark.parametrize("precision", PRECISIONS)
def test_paper_line_source_200_first_steps(A, oracle_200, precision):
    """The paper's 200^2, N_q = 92 configuration: 12 Heun steps (every cell, many tiles) against the
    oracle (the whole run to t = 1 is measured by the accuracy bench)."""
    dt, phi_ref = oracle_200
    wl = synth.PAPER_LINE_SOURCE_200
    p = gpu_problem(A, wl, precision)
    p.step(12, dt)
    phi = p.scalar_flux()
    p.close()
    assert rel_l2(phi, phi_ref) <= RUN_TOL[precision]

"""The paper's explicit scheme (Sec. 3.1: Heun in time, minmod-limited second-order upwind fluxes) on
the CUDA-core paths, against the FP64 oracle (oracle.step_heun / run_heun) on the same inputs."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

import oracle as O
import synth
from helpers import RUN_TOL, ensure_built, offdiag_rowsum, oracle_setup, rel_l2, run_steps, step_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


def problem(A, wl, precision, psi0):
    p = A.Problem(wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, precision)
    p.set_product_quadrature(wl.n_polar, wl.n_azim)
    sa, ss, q = wl.materials()
    p.set_cross_sections(sa, ss, q)
    p.set_artificial_scattering(wl.sigma_as, wl.eps)
    p.set_scheme("heun")
    p.set_state(psi0)
    return p


# ragged tiles (nx not a multiple of the 8 / 16-cell tiles), rows near both y edges, a 3 x 2 grid
@pytest.mark.parametrize("nx,ny,npol,naz", [(37, 11, 4, 8), (20, 5, 8, 8), (3, 2, 2, 4), (17, 33, 8, 16)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_one_heun_step_matches_oracle(A, nx, ny, npol, naz, precision, tol):
    wl = synth.Workload("heun", "random", nx, ny, 0.0, 0.1 * nx, 0.0, 0.1 * ny, npol, naz, 0.6, seed=nx * 7 + ny)
    psi0 = wl.psi0()
    p = problem(A, wl, precision, psi0)
    dt = 0.9 * p.max_stable_dt()
    l0 = p.launch_count()
    p.step(1, dt)
    launches = p.launch_count() - l0
    got = p.state()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step_heun(psi0, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max())
    assert launches == 2
    p.close()


@pytest.mark.parametrize("nx,ny,npol,naz", [(37, 11, 4, 8), (40, 24, 8, 16), (23, 29, 16, 32)])
@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
def test_one_heun_step_tensor_cores(A, nx, ny, npol, naz, precision):
    """Both stages on the persistent tensor-core kernel.  Each stage errs by at most the one-step
    bound of its precision (BF16 operands of the contraction); the second stage halves the sum of
    the first stage's error and its own, so twice the one-step bound covers the step."""
    wl = synth.Workload("heun", "random", nx, ny, 0.0, 0.1 * nx, 0.0, 0.1 * ny, npol, naz, 0.6, seed=nx + 5 * ny)
    psi0 = wl.psi0()
    p = problem(A, wl, precision, psi0)
    dt = 0.9 * p.max_stable_dt()
    l0 = p.launch_count()
    p.step(1, dt)
    assert p.launch_count() - l0 == 2
    got = p.state()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step_heun(psi0, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    scale = max(1.0, np.abs(ref).max(), np.abs(psi0).max())
    tol = 2.0 * step_tolerance(precision, dt, wl.sigma_as, scale, offdiag_rowsum(K))
    assert np.abs(got - ref).max() <= tol
    p.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("bf16", RUN_TOL["bf16"]),
                                           ("bf16x3", RUN_TOL["bf16x3"])])
def test_line_source_at_095_of_admissible_dt(A, precision, tol):
    """The 64^2 line source (Q = 128, beta = 1/8) run to t = 1 at 0.95 of the scheme's admissible dt."""
    wl = dataclasses.replace(synth.LINE_SOURCE_64, scheme="heun", dt_rule="bound", cfl=0.95)
    n, dt = run_steps(wl)
    p = problem(A, wl, precision, wl.psi0())
    assert dt <= 0.951 * p.max_stable_dt()
    p.step(n, dt)
    phi = p.scalar_flux()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.run_heun(wl.psi0(), n, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    assert rel_l2(phi, ref @ w) <= tol
    p.close()


def test_heun_unsupported_combinations(A):
    wl = synth.Workload("heun", "random", 8, 8, 0.0, 0.8, 0.0, 0.8, 4, 8, 0.6, seed=2)
    p = problem(A, wl, "bf16", wl.psi0())
    e = A.Problem(wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, "bf16").set_product_quadrature(wl.n_polar, wl.n_azim)
    e.set_cross_sections(*wl.materials()).set_artificial_scattering(wl.sigma_as, wl.eps).set_state(wl.psi0())
    with A.Batch() as b:   # the members of a batch share one scheme
        b.add(p, 1, 0.5 * p.max_stable_dt())
        with pytest.raises(A.AssnError) as ei:
            b.add(e, 1, 0.5 * e.max_stable_dt())
        assert ei.value.status == A._lib.ASSN_ERR_ARG
    p.close()
    e.close()
    q = problem(A, wl, "fp32", wl.psi0())
    with pytest.raises(A.AssnError):
        A._lib.assn_set_scheme(q.handle, 7)
    assert q.scheme() == A._lib.ASSN_SCHEME_HEUN_MINMOD
    q.close()

"""The paper's implicit sweeping-Krylov step (Sec. 3.4-3.5, Alg. 1-3) through the C ABI against the FP64
oracle (oracle.implicit): single sweeps, fixed numbers of source iterations, whole steps and runs."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

import oracle as O
import synth
from helpers import RUN_TOL, ensure_built, gpu_problem, oracle_run, oracle_setup, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


def quadrature_with_axes():
    """A product quadrature (all four quadrants) plus ordinates with a zero x or y component."""
    Om, w = O.product_quadrature(2, 8)
    extra = np.array([[0.0, 1.0, 0.0], [0.0, -0.6, 0.8], [0.6, 0.0, -0.8], [-0.8, 0.0, 0.6]])
    Om = np.vstack([Om, extra])
    w = np.concatenate([w * (1 - 0.1), np.full(4, 0.1 * 4 * np.pi / 4)])
    return Om, w


def make(A, precision, nx, ny, sigma_as, seed, norm=0):
    Om, w = quadrature_with_axes()
    p = A.Problem(nx, ny, 0.0, 0.1 * nx, 0.0, 0.1 * ny, precision)
    p.set_quadrature(Om, w)
    sa, ss, q = synth.random_materials(seed, ny, nx)
    p.set_cross_sections(sa, ss, q)
    p.set_artificial_scattering(sigma_as, 0.7, 0, norm)
    p.set_scheme("implicit")
    K = O.kernel_matrix(Om, w, 0.7, normalisation="column" if norm == 0 else "row")
    return p, Om, w, K, sa, ss, q


TOL = {"fp64": 1e-12, "fp32": 2e-5}


# ragged grids, a single row and column, tiny grids, and tall grids that take 1, 2 and 4 rows per thread of
# the row sweep or (beyond 2048 rows) the general sweep; dt/h = 2 (the paper's implicit CFL number)
@pytest.mark.parametrize("nx,ny", [(37, 11), (1, 9), (13, 1), (2, 2), (64, 48), (5, 300), (3, 1000), (2, 1500),
                                   (2, 2100)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_one_sweep_matches_oracle(A, nx, ny, precision):
    p, Om, w, K, sa, ss, q = make(A, precision, nx, ny, 0.0, nx + ny)
    rng = np.random.default_rng(nx * 7 + ny)
    R = rng.random((ny, nx, len(w))) - 0.2
    dt = 0.2
    got = p.implicit_source_iteration(dt, R, np.zeros_like(R), 1)
    ref = O.sweep(dt * R, Om, 0.1, dt, sa + ss)
    assert np.abs(got - ref).max() <= TOL[precision] * np.abs(ref).max()
    p.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("norm", [0, 1])
def test_fixed_source_iterations_match_oracle(A, precision, norm):
    nx, ny = 29, 17
    p, Om, w, K, sa, ss, q = make(A, precision, nx, ny, 5.0, 3, norm)
    rng = np.random.default_rng(5)
    R = rng.random((ny, nx, len(w)))
    psi0 = rng.random((ny, nx, len(w)))
    dt = 0.2
    got = p.implicit_source_iteration(dt, R, psi0, 4)
    T = O.source_iteration_lipschitz(sa, ss, 5.0, dt)
    ref, _ = O.source_iteration(psi0, R, K, Om, sa + ss + 5.0, 5.0, 0.1, dt, 0.0, T, fixed=4)
    assert np.abs(got - ref).max() <= TOL[precision] * np.abs(ref).max()
    p.close()


def test_fixed_source_iterations_many_ordinates(A):
    """Q = 512 in FP64: the largest ordinate tiles of the source kernel and 512 sweep blocks."""
    nx, ny = 9, 7
    Om, w = O.product_quadrature(16, 32)
    p = A.Problem(nx, ny, 0.0, 0.9, 0.0, 0.7, "fp64")
    p.set_quadrature(Om, w)
    sa, ss, q = synth.random_materials(6, ny, nx)
    p.set_cross_sections(sa, ss, q)
    p.set_artificial_scattering(5.0, 0.3, 0, 0)
    p.set_scheme("implicit")
    rng = np.random.default_rng(6)
    R = rng.random((ny, nx, len(w)))
    psi0 = rng.random((ny, nx, len(w)))
    got = p.implicit_source_iteration(0.2, R, psi0, 2)
    p.close()
    K = O.kernel_matrix(Om, w, 0.3)
    T = O.source_iteration_lipschitz(sa, ss, 5.0, 0.2)
    ref, _ = O.source_iteration(psi0, R, K, Om, sa + ss + 5.0, 5.0, 0.1, 0.2, 0.0, T, fixed=2)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_step_equals_the_assembled_system(A):
    """One implicit step with tight tolerances equals the implicit system solved directly."""
    nx, ny = 6, 5
    Om, w = O.product_quadrature(2, 4)
    p = A.Problem(nx, ny, 0.0, 0.6, 0.0, 0.5, "fp64")
    p.set_quadrature(Om, w)
    sa, ss, q = synth.random_materials(9, ny, nx)
    p.set_cross_sections(sa, ss, q)
    p.set_artificial_scattering(5.0, 0.6, 0, 1)
    p.set_scheme("implicit")
    p.set_implicit_params(1e-15, 1e-13)
    rng = np.random.default_rng(2)
    psi_old = rng.random((ny, nx, len(w)))
    p.set_state(psi_old)
    p.step(1, 0.2)
    got = p.state()
    K = O.kernel_matrix(Om, w, 0.6, normalisation="row")
    ref = O.implicit_step_direct(psi_old, K, Om, w, sa, ss, q, 5.0, 0.1, 0.2)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    st = p.implicit_stats()
    assert st["gmres_iterations"] > 1 and st["sweeps"] >= st["source_iterations"] > st["gmres_iterations"]
    p.close()


TALL = (3, 300)


@pytest.fixture(scope="module")
def tall_ref():
    """The oracle's implicit step (tolerances 1e-13) on a 3 x 300 grid, Q = 8, sigma_as = 5, dt/h = 2."""
    nx, ny = TALL
    Om, w = O.product_quadrature(2, 4)
    sa, ss, q = synth.random_materials(4, ny, nx)
    K = O.kernel_matrix(Om, w, 0.6)
    psi_old = np.random.default_rng(8).random((ny, nx, len(w)))
    ref, _, _, _ = O.implicit_step(psi_old, O.scalar_flux(psi_old, w), K, Om, w, sa, ss, q, 5.0, 0.1, 0.2,
                                   1e-13, 1e-13)
    return Om, w, sa, ss, q, psi_old, ref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_on_a_tall_grid(A, tall_ref, precision):
    """A whole implicit step on a tall grid (the row sweep, whose blocks also sum the source iteration's
    convergence norm) against the oracle's step."""
    Om, w, sa, ss, q, psi_old, ref = tall_ref
    nx, ny = TALL
    p = A.Problem(nx, ny, 0.0, 0.3, 0.0, 30.0, precision)
    p.set_quadrature(Om, w)
    p.set_cross_sections(sa, ss, q)
    p.set_artificial_scattering(5.0, 0.6, 0, 0)
    p.set_scheme("implicit")
    p.set_implicit_params(1e-12, 1e-12)
    p.set_state(psi_old)
    p.step(1, 0.2)
    got = p.state()
    p.close()
    assert np.abs(got - ref).max() <= (1e-9 if precision == "fp64" else 1e-5) * np.abs(ref).max()


def paper_small(n=24, **kw):
    return dataclasses.replace(synth.paper_line_source_implicit(n, t_final=0.75), **kw)


@pytest.fixture(scope="module")
def converged_24():
    """The oracle's converged run (source iteration and GMRES to 1e-10) of the paper's implicit as-S_4
    line source on 24^2 cells, 3 steps at dt/dx = 2."""
    wl = paper_small(si_eps=1e-10, gmres_tol=1e-10)
    n, dt = wl.steps()
    ref, w = oracle_run(wl, n, dt)
    return wl, n, dt, ref @ w


# both sides stop within their solver tolerances (1e-10): FP64 agrees far below 1e-8; FP32 at the
# FP32 whole-run target
IMPLICIT_RUN_TOL = {"fp64": 1e-8, "fp32": RUN_TOL["fp32"]}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_paper_implicit_line_source_run(A, converged_24, precision):
    """The paper's implicit as-S_4 line source (N_q = 92, row normalisation, eps = 4 / 92, sigma_as = 7,
    dt/dx = 2), the same tolerances on both sides."""
    wl, n, dt, phi_ref = converged_24
    p = gpu_problem(A, wl, precision)
    p.step(n, dt)
    phi = p.scalar_flux()
    st = p.implicit_stats()
    p.close()
    assert rel_l2(phi, phi_ref) <= IMPLICIT_RUN_TOL[precision]
    assert st["gmres_iterations"] >= n and st["source_iterations"] > st["gmres_iterations"]


@pytest.fixture(scope="module")
def converged_lattice_28():
    """The oracle's converged run (tolerances 1e-10) of the paper's implicit as-S_4 lattice on 28^2 cells
    (4 cells per block), dt/dx = 2, the first two steps (t = 1; the source iteration's contraction
    factor is about 0.7 here, so converged steps are costly for the oracle)."""
    wl = dataclasses.replace(synth.paper_lattice_implicit(28, t_final=1.0), si_eps=1e-10, gmres_tol=1e-10)
    n, dt = wl.steps()
    ref, w = oracle_run(wl, n, dt)
    return wl, n, dt, ref @ w


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_paper_implicit_lattice_run(A, converged_lattice_28, precision):
    wl, n, dt, phi_ref = converged_lattice_28
    p = gpu_problem(A, wl, precision)
    p.step(n, dt)
    phi = p.scalar_flux()
    p.close()
    assert rel_l2(phi, phi_ref) <= IMPLICIT_RUN_TOL[precision]


def test_paper_tolerances_give_the_tolerance_level(A, converged_24):
    """With the paper's own tolerances (source iteration 1e-4, GMRES 1.5e-8) the result stays within
    about the solver tolerance of the converged solution."""
    wl, n, dt, phi_ref = converged_24
    p = gpu_problem(A, dataclasses.replace(wl, si_eps=1e-4, gmres_tol=1.5e-8), "fp64")
    p.step(n, dt)
    phi = p.scalar_flux()
    p.close()
    assert rel_l2(phi, phi_ref) <= 1e-4


def test_implicit_rejected_where_unsupported(A):
    p = A.Problem(8, 8, 0.0, 1.0, 0.0, 1.0, "bf16")
    p.set_product_quadrature(2, 4)
    with pytest.raises(A.AssnError) as e:
        p.set_scheme("implicit")
    assert e.value.status == A._lib.ASSN_ERR_UNSUPPORTED
    p.close()
    q = A.Problem(8, 8, 0.0, 1.0, 0.0, 1.0, "fp32")
    with pytest.raises(A.AssnError):
        q.set_implicit_params(-1.0)
    q.close()

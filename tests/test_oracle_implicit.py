"""Pins of the implicit oracle (oracle.implicit; Sec. 3.4-3.5, Alg. 1-3, Appendix B) against printed
values, closed forms and dense linear algebra."""
import math

import numpy as np
import pytest

import oracle as O
import synth

FOUR_PI = 4.0 * math.pi


def test_appendix_b_symmetric_part_of_the_upwind_operator():
    """In 1D with lambda = 1 the transport part B of the streaming operator has the symmetric part
    printed in Appendix B: 3/2 on the diagonal, -1 on the first and 1/4 on the second off-diagonals,
    and it is positive definite."""
    n = 40
    Om = np.array([[1.0, 0.0, 0.0]])
    sig = np.zeros((1, n))
    cols = []
    for e in np.eye(n):
        cols.append(O.streaming_apply(e.reshape(1, n, 1), Om, 1.0, 1.0, sig).ravel() - e)
    B = np.column_stack(cols)
    S = 0.5 * (B + B.T)
    assert np.allclose(np.diag(S), 1.5, atol=0)
    assert np.allclose(np.diag(S, 1), -1.0, atol=0) and np.allclose(np.diag(S, 2), 0.25, atol=0)
    assert np.count_nonzero(np.triu(S, 3)) == 0
    assert np.linalg.eigvalsh(S).min() > 0.0
    assert np.allclose(np.tril(B, -3), 0.0) and np.allclose(np.triu(B, 1), 0.0)   # upwind, two cells


@pytest.mark.parametrize("ny,nx", [(7, 9), (1, 6), (5, 1), (1, 1), (3, 12)])
def test_sweep_inverts_the_streaming_operator(ny, nx):
    rng = np.random.default_rng(ny * 31 + nx)
    Om, w = O.product_quadrature(2, 8)                       # all four quadrants
    Om = np.vstack([Om, [[0.0, 1.0, 0.0], [0.0, -0.6, 0.8], [0.6, 0.0, -0.8]]])   # zero components
    R = rng.random((ny, nx, len(Om))) - 0.3
    sig = rng.random((ny, nx)) * 3.0
    psi = O.sweep(R, Om, 0.2, 0.7, sig)
    assert np.abs(O.streaming_apply(psi, Om, 0.2, 0.7, sig) - R).max() < 1e-12 * np.abs(R).max()


def test_implicit_euler_decay_is_exact_without_transport():
    """Ordinates along +-z have no projected velocity; an isotropic state with row-normalised K then
    follows psi^{n+1} = psi^n / (1 + dt sigma_a) exactly (scattering and artificial scattering move
    nothing), through the whole sweeping-Krylov step."""
    Om = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    w = np.array([2 * np.pi, 2 * np.pi])
    K = O.kernel_matrix(Om, w, 2.0, normalisation="row")
    ny, nx = 3, 4
    sa = np.full((ny, nx), 0.7)
    ss = np.full((ny, nx), 1.3)
    q = np.zeros((ny, nx))
    psi = np.full((ny, nx, 2), 2.0)
    phi = O.scalar_flux(psi, w)
    for n in range(1, 4):
        psi, phi, si, its = O.implicit_step(psi, phi, K, Om, w, sa, ss, q, 5.0, 0.1, 0.25, 1e-14, 1e-14)
        assert np.abs(psi - 2.0 / (1 + 0.25 * 0.7) ** n).max() < 1e-12


def test_source_iteration_converges_to_the_dense_solve():
    rng = np.random.default_rng(4)
    Om, w = O.product_quadrature(2, 4)
    K = O.kernel_matrix(Om, w, 0.5)
    ny, nx, Q = 4, 5, len(w)
    sa, ss, _ = synth.random_materials(2, ny, nx)
    sig_as, h, dt = 5.0, 0.1, 0.08
    sig = sa + ss + sig_as
    R = rng.random((ny, nx, Q))
    T = O.source_iteration_lipschitz(sa, ss, sig_as, dt)
    psi, it = O.source_iteration(np.zeros_like(R), R, K, Om, sig, sig_as, h, dt, 1e-15, T)
    n = ny * nx * Q

    def op(v):
        p = v.reshape(ny, nx, Q)
        return (O.streaming_apply(p, Om, h, dt, sig) - dt * sig_as * (p @ K.T)).ravel()
    A = np.column_stack([op(e) for e in np.eye(n)])
    ref = np.linalg.solve(A, dt * R.ravel()).reshape(ny, nx, Q)
    assert 1 < it < 200
    assert np.abs(psi - ref).max() < 1e-12 * np.abs(ref).max()
    one, _ = O.source_iteration(np.zeros_like(R), R, K, Om, sig, sig_as, h, dt, 0.0, T, fixed=1)
    assert np.abs(one - O.sweep(dt * R, Om, h, dt, sig)).max() == 0.0


@pytest.mark.parametrize("restart", [50, 7])
def test_gmres_solves_a_random_system(restart):
    rng = np.random.default_rng(restart)
    n = 40
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n)
    x, its = O.gmres(lambda v: A @ v, b, np.zeros(n), 1e-12, restart=restart, max_iter=400)
    assert np.linalg.norm(A @ x - b) <= 1e-11 * np.linalg.norm(b)
    assert its <= 400


@pytest.mark.parametrize("norm", ["column", "row"])
def test_sweeping_krylov_step_equals_the_assembled_system(norm):
    """Alg. 3 with tight tolerances reproduces the implicit step solved as one linear system."""
    rng = np.random.default_rng(7)
    Om, w = O.product_quadrature(2, 4)
    K = O.kernel_matrix(Om, w, 0.6, normalisation=norm)
    ny, nx = 5, 4
    sa, ss, q = synth.random_materials(3, ny, nx)
    psi_old = rng.random((ny, nx, len(w)))
    h, dt = 0.1, 0.2                                  # dt/h = 2, the paper's implicit CFL number
    psi, phi, si, its = O.implicit_step(psi_old, O.scalar_flux(psi_old, w), K, Om, w, sa, ss, q, 5.0, h, dt,
                                        1e-15, 1e-14)
    ref = O.implicit_step_direct(psi_old, K, Om, w, sa, ss, q, 5.0, h, dt)
    assert np.abs(psi - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(phi - O.scalar_flux(ref, w)).max() < 1e-10 * np.abs(phi).max()
    assert its > 1 and si > its


@pytest.mark.parametrize("dt,norm", [(0.05, "column"), (0.2, "row"), (0.5, "column"), (0.5, "row")])
def test_source_iteration_stopping_rule_bounds_the_error(dt, norm):
    """Alg. 1's a-posteriori rule with the contraction estimate T of R26: when the iteration stops, the
    iterate is within eps (L2 over all values) of the exact solution of (L - dt sigma_as K) psi = dt R,
    from dt/h = 0.5 to 5 (T from 0.25 to 0.73)."""
    rng = np.random.default_rng(int(dt * 100))
    Om, w = O.product_quadrature(2, 4)
    K = O.kernel_matrix(Om, w, 0.7, normalisation=norm)
    ny, nx, Q = 5, 6, len(w)
    sa, ss, _ = synth.random_materials(11, ny, nx)
    sig_as, h = 7.0, 0.1
    sig = sa + ss + sig_as
    R = rng.random((ny, nx, Q))
    T = O.source_iteration_lipschitz(sa, ss, sig_as, dt)

    def op(v):
        p = v.reshape(ny, nx, Q)
        return (O.streaming_apply(p, Om, h, dt, sig) - dt * sig_as * (p @ K.T)).ravel()
    A = np.column_stack([op(e) for e in np.eye(ny * nx * Q)])
    ref = np.linalg.solve(A, dt * R.ravel()).reshape(ny, nx, Q)
    for eps in (1e-3, 1e-6):
        psi, it = O.source_iteration(np.zeros_like(R), R, K, Om, sig, sig_as, h, dt, eps, T)
        assert it > 1
        assert np.linalg.norm(psi - ref) <= eps


def test_steady_state_is_second_order_in_the_interior():
    """One implicit step with dt -> infinity gives the discrete steady state of Omega d psi/dx + psi = 1 on
    [0, 1] with vacuum inflow (one ordinate along x, sigma_a = q = 1); the exact cell averages are
    1 - (e^{-x_l} - e^{-x_r}) / h.  Away from the inflow the error falls 4x per halving of h (second
    order; the zero inflow ghosts leave a first-order error in the first cell only)."""
    def interior_error(n):
        h = 1.0 / n
        Om = np.array([[1.0, 0.0, 0.0]])
        w = np.array([FOUR_PI])
        K = np.eye(1)
        sa, ss, q = np.ones((1, n)), np.zeros((1, n)), np.ones((1, n))
        psi, _, _, _ = O.implicit_step(np.zeros((1, n, 1)), np.zeros((1, n)), K, Om, w, sa, ss, q, 0.0, h, 1e9,
                                       1e-14, 1e-14)
        xl = np.arange(n) * h
        exact = 1.0 - (np.exp(-xl) - np.exp(-(xl + h))) / h
        return np.abs(psi[0, :, 0] - exact)[n // 2:].max()
    e64, e128 = interior_error(64), interior_error(128)
    assert 3.8 < e64 / e128 < 4.2

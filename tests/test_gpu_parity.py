"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Sizes span several tiles of every kernel and leave ragged tails in x and in the ordinate
dimension; the full-size lattice launch the bench times is checked on sampled cells.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from tests.helpers import (RUN_TOL, ensure_built, gpu_problem, offdiag_rowsum, oracle_run, oracle_setup, rel_l2,
                           step_tolerance)

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "fp32", "bf16", "bf16x3"]


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


def random_workload(nx, ny, npol, naz, beta=0.5, seed=0):
    return synth.Workload(f"rand{nx}x{ny}", "random", nx, ny, 0.0, nx * 0.05, 0.0, ny * 0.05, npol, naz, beta,
                          sigma_as=5.0, seed=seed)


def one_step_check(A, wl, precision, dt=None, normalisation=0):
    p = gpu_problem(A, wl, precision, normalisation=normalisation)
    if dt is None:
        dt = 0.9 * p.max_stable_dt()
    p.step(1, dt)
    got = p.state()
    Om, w, K, sa, ss, q = oracle_setup(wl, "column" if normalisation == 0 else "row")
    ref = O.step(wl.psi0(), K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    tol = step_tolerance(precision, dt, wl.sigma_as, np.abs(wl.psi0()).max(), offdiag_rowsum(K))
    err = np.abs(got - ref).max()
    p.close()
    assert err <= tol, (precision, err, tol)
    return err


def test_quadrature_matches_oracle(A):
    for npol, naz in [(8, 16), (16, 32), (3, 5)]:
        p = A.Problem(4, 4, 0, 1, 0, 1, "fp32").set_product_quadrature(npol, naz)
        om, w = p.quadrature()
        Om, wo = O.product_quadrature(npol, naz)
        assert np.allclose(om, Om, atol=2e-15) and np.allclose(w, wo, rtol=1e-14)
        p.close()


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("norm", [0, 1])
@pytest.mark.parametrize("npol,naz,eps", [(8, 16, 0.039), (16, 32, 0.078), (4, 3, 0.5)])
def test_kernel_matrix_matches_oracle(A, kind, norm, npol, naz, eps):
    p = A.Problem(4, 4, 0, 1, 0, 1, "fp64").set_product_quadrature(npol, naz)
    p.set_artificial_scattering(5.0, eps, kind, norm)
    K = p.kernel_matrix()
    om, wl = p.quadrature()
    Om, w = O.product_quadrature(npol, naz)
    Ko = O.kernel_matrix(Om, w, eps, kind="gauss" if kind == 0 else "exp",
                         normalisation="column" if norm == 0 else "row")
    assert np.abs(K - Ko).max() <= 1e-14 * Ko.max()
    # Derived bound on the significant entries.  s = exp(-a(mu)) with a = (1-mu)^2/eps^2 (Gaussian)
    # or (1-mu)/eps^2 (exp kind): an error d_mu of the cosine moves ln s by |a'(mu)| d_mu, where
    # d_mu <= 2 max|Omega_lib - Omega_oracle| + 4u (the ordinates' own difference, then the rounding
    # of a 3-term dot product); evaluating a and exp costs <= 4u (a + 2); the normalisation sum over
    # Q terms adds <= 2 Q u plus twice the weighted mean of the entries' errors (bounded by their
    # maximum over the significant entries; the rest weigh < 1e-8 Q) and twice the weights' error.
    u = 2.0 ** -53
    mu = np.clip(Om @ Om.T, -1.0, 1.0)
    if kind == 0:
        da, arg = 2.0 * (1.0 - mu) / eps ** 2, (1.0 - mu) ** 2 / eps ** 2
    else:
        da, arg = np.full_like(mu, 1.0 / eps ** 2), (1.0 - mu) / eps ** 2
    d_mu = 2.0 * np.abs(om - Om).max() + 4.0 * u
    d_w = float(np.max(np.abs(wl - w) / w))
    big = Ko > 1e-8 * Ko.max()
    e_s = da * d_mu + 4.0 * u * (arg + 2.0)
    bound = e_s + 2.0 * e_s[big].max() + 2.0 * d_w + 2.0 * len(w) * u + 1e-8 * len(w) * e_s.max()
    rel = np.abs(K - Ko)[big] / Ko[big]   # (only the significant entries; others may be exactly zero)
    assert np.all(rel <= bound[big]), float(np.max(rel / bound[big]))
    p.close()


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("nx,ny,npol,naz", [(37, 5, 8, 16), (200, 3, 8, 8), (130, 2, 16, 32), (9, 7, 3, 4),
                                            (129, 3, 16, 16), (67, 3, 8, 24)])
def test_one_step_random_state(A, precision, nx, ny, npol, naz):
    """Ragged tiles (nx not a multiple of any tile width), Q in {128, 64, 512, 12, 256, 192}."""
    one_step_check(A, random_workload(nx, ny, npol, naz, seed=nx + ny), precision)


@pytest.mark.parametrize("precision", PRECS)
def test_one_step_row_normalisation(A, precision):
    one_step_check(A, random_workload(70, 4, 8, 16, seed=3), precision, normalisation=1)


@pytest.mark.parametrize("precision", PRECS)
def test_one_step_arbitrary_quadrature(A, precision):
    """The paper's order-2 icosahedron set (12 ordinates, Q padded to 64) as a user quadrature."""
    import os
    rows = [list(map(float, l.split())) for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                                    "icosahedron_order2.txt"))
            if l.strip() and not l.startswith("#")]
    tab = np.array(rows)
    Om, w = tab[:, :3], tab[:, 3]
    nx, ny = 21, 6
    psi = synth.random_psi(4, ny, nx, 12)
    sa, ss, q = synth.random_materials(4, ny, nx)
    h = 0.05
    p = A.Problem(nx, ny, 0, nx * h, 0, ny * h, precision).set_quadrature(Om, w)
    p.set_cross_sections(sa, ss, q).set_artificial_scattering(5.0, 4.5 / 12).set_state(psi)
    dt = 0.9 * p.max_stable_dt()
    p.step(1, dt)
    got = p.state()
    K = O.kernel_matrix(Om, w, 4.5 / 12)
    ref = O.step(psi, K, Om, w, sa, ss, q, 5.0, h, dt)
    assert np.abs(got - ref).max() <= step_tolerance(precision, dt, 5.0, psi.max(), offdiag_rowsum(K))
    p.close()


@pytest.mark.parametrize("precision", PRECS)
def test_line_source_64_full_run(A, precision):
    """The 64 x 64, Q = 128 line source to t = 1 (43 steps): relative L2 of Phi vs the FP64 oracle."""
    wl = synth.LINE_SOURCE_64
    n, dt = wl.steps()
    p = gpu_problem(A, wl, precision)
    p.step(n, dt)
    phi = p.scalar_flux()
    ref, w = oracle_run(wl, n, dt)
    err = rel_l2(phi, ref @ w)
    p.close()
    assert err <= RUN_TOL[precision], (precision, err)


@pytest.mark.parametrize("precision", PRECS)
def test_lattice_small_full_run(A, precision):
    """Lattice layout at 7 cells per block (49 x 49), Q = 64, to t = 0.8 against the oracle
    (CFL 0.2: the absorbers' sigma_t = 10 needs the smaller step at this coarse h)."""
    wl = synth.lattice(49, 8, 8, 0.5, t_final=0.8)
    wl.cfl = 0.2
    n, dt = wl.steps()
    p = gpu_problem(A, wl, precision)
    p.step(n, dt)
    phi = p.scalar_flux()
    ref, w = oracle_run(wl, n, dt)
    err = rel_l2(phi, ref @ w)
    p.close()
    assert err <= RUN_TOL[precision], (precision, err)


@pytest.mark.parametrize("precision", PRECS)
def test_exact_shift_single_ordinate(A, precision):
    """One ordinate Omega = (1,0,0) with dt = h: integer data moves one cell exactly."""
    nx, ny, h = 70, 3, 0.5
    rng = np.random.default_rng(1)
    psi = rng.integers(0, 64, size=(ny, nx, 1)).astype(np.float64)
    z = np.zeros((ny, nx))
    p = A.Problem(nx, ny, 0, nx * h, 0, ny * h, precision).set_quadrature([[1.0, 0.0, 0.0]], [4 * math.pi])
    p.set_cross_sections(z, z, z).set_artificial_scattering(0.0, 0.1).set_state(psi)
    p.step(1, h)
    got = p.state()
    expect = np.zeros_like(psi)
    expect[:, 1:] = psi[:, :-1]
    assert np.array_equal(got, expect)
    p.close()


@pytest.mark.parametrize("precision", PRECS)
def test_eps_to_zero_equals_plain_sn(A, precision):
    """eps -> 0 makes K the identity: the as-S_N step equals the sigma_as = 0 step bit for bit."""
    wl = random_workload(50, 4, 8, 16, seed=9)
    wl.beta = 1e-5
    a = gpu_problem(A, wl, precision)
    b = gpu_problem(A, wl, precision, sigma_as=0.0)
    dt = 0.5 * a.max_stable_dt()
    a.step(3, dt)
    b.step(3, dt)
    assert np.array_equal(a.state(), b.state())
    a.close(), b.close()


@pytest.mark.parametrize("precision", PRECS)
def test_mass_balance_vacuum(A, precision):
    """sigma_a = 0, q = 0: both scattering operators conserve particles, so one step changes the mass
    only by the outflow through the vacuum boundary (computed here from the boundary cells)."""
    wl = random_workload(66, 10, 8, 16, seed=5)
    psi = wl.psi0()
    ny, nx = psi.shape[:2]
    z = np.zeros((ny, nx))
    ss = np.full((ny, nx), 1.0)
    p = A.Problem(nx, ny, wl.x0, wl.x1, wl.y0, wl.y1, precision).set_product_quadrature(8, 16)
    p.set_cross_sections(z, ss, z).set_artificial_scattering(5.0, wl.eps).set_state(psi)
    dt = 0.9 * p.max_stable_dt()
    m0 = p.mass()
    p.step(1, dt)
    m1 = p.mass()
    Om, w = O.product_quadrature(8, 16)
    h = wl.h
    out = 0.0
    for qq in range(w.size):
        ox, oy = Om[qq, 0], Om[qq, 1]
        bx = psi[:, -1, qq] if ox > 0 else psi[:, 0, qq]
        by = psi[-1, :, qq] if oy > 0 else psi[0, :, qq]
        out += w[qq] * (abs(ox) * bx.sum() + abs(oy) * by.sum())
    expect = -dt * h * out
    tol = {"fp64": 1e-12, "fp32": 2e-6, "bf16": 2e-6, "bf16x3": 2e-6}[precision] * m0
    assert abs((m1 - m0) - expect) <= tol, (precision, m1 - m0, expect)
    p.close()


def test_lattice_448_sampled_cells(A):
    """The full-size lattice launch (448 x 448, Q = 512) that the bench times: one BF16 step from a
    seeded state, compared with the oracle on sampled cells (tile edges, corners, materials)."""
    wl = synth.LATTICE_448
    rng = np.random.default_rng(2)
    psi = rng.uniform(0.0, 1.0, size=(wl.ny, wl.nx, wl.Q))
    n, dt = wl.steps()
    cells = [(0, 0), (0, 447), (447, 0), (447, 447), (224, 224), (200, 63), (200, 64), (201, 127), (201, 128),
             (5, 383), (6, 384), (300, 191), (300, 192), (100, 255), (101, 256), (447, 320)]
    cells += [(int(j), int(i)) for j, i in rng.integers(0, 448, size=(16, 2))]
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step_at_cells(psi, cells, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    for precision in ("bf16", "bf16x3", "fp32"):
        p = gpu_problem(A, wl, precision, psi0=psi)
        p.step(1, dt)
        got = p.state()
        p.close()
        tol = step_tolerance(precision, dt, wl.sigma_as, 1.0, offdiag_rowsum(K))
        for n_, (j, i) in enumerate(cells):
            assert np.abs(got[j, i] - ref[n_]).max() <= tol, (precision, j, i)


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
def test_tensor_path_matches_fp32_path_on_one_cell_grid(A, precision):
    """Degenerate grid: a single cell (every neighbour is a vacuum ghost)."""
    wl = random_workload(1, 1, 16, 32, seed=11)
    one_step_check(A, wl, precision)


def test_errors_are_reported(A):
    from paper_1911_08801_gb300 import _lib as L
    with pytest.raises(A.AssnError) as e:
        A.Problem(0, 4, 0, 1, 0, 1, "fp32")
    assert e.value.status == L.ASSN_ERR_ARG
    with pytest.raises(A.AssnError):
        A.Problem(4, 4, 0, 1, 0, 2, "fp32")      # non-square cells
    p = A.Problem(8, 8, 0, 1, 0, 1, "bf16")
    with pytest.raises(A.AssnError) as e:
        p.step(1, 0.01)
    assert e.value.status == L.ASSN_ERR_STATE
    p.set_product_quadrature(8, 16)
    z = np.zeros((8, 8))
    p.set_cross_sections(z, z, z).set_artificial_scattering(5.0, 0.1)
    with pytest.raises(A.AssnError) as e:
        p.step(1, 10.0)
    assert e.value.status == L.ASSN_ERR_UNSTABLE
    with pytest.raises(A.AssnError):
        p.set_artificial_scattering(5.0, -1.0)
    p.close()


def test_launch_count_and_finite(A):
    wl = random_workload(40, 4, 8, 16, seed=1)
    p = gpu_problem(A, wl, "bf16")
    c0 = p.launch_count()
    p.step(4, 0.5 * p.max_stable_dt())
    assert p.launch_count() - c0 == 4
    p.check_finite()
    p.close()


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("npol,naz", [(16, 32), (16, 16), (8, 8)])
def test_tensor_kernel_variants_and_tilings_agree(A, precision, npol, naz):
    """The persistent kernel at every tile width it accepts and the one-tile-per-CTA kernel give the
    same step from the same state (they differ only in the FP32 summation order of Phi) and each
    matches the oracle over two steps.  (After the first step the states may differ in the last
    bit, which can move a value across a BF16 rounding boundary in the second step, so the
    variants are compared after one step.)"""
    wl = random_workload(150, 7, npol, naz, seed=21)
    Om, w, K, sa, ss, q = oracle_setup(wl)
    one, two = [], []
    dt = None
    for variant, tile, stages in [(0, 0, 0), (0, 32, 2), (0, 64, 3), (1, 0, 0), (1, 64, 2)]:
        p = gpu_problem(A, wl, precision)
        try:
            p.set_tiling(tile, stages, variant)
            p.tiling()
        except A.AssnError:
            p.close()
            continue
        if dt is None:
            dt = 0.9 * p.max_stable_dt()
        p.step(1, dt)
        one.append(((variant, tile, stages), p.state()))
        p.step(1, dt)
        two.append(((variant, tile, stages), p.state()))
        p.close()
    assert len(one) >= 3
    ref = O.run(wl.psi0(), 2, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    tol = 2 * step_tolerance(precision, dt, wl.sigma_as, 1.0, offdiag_rowsum(K))
    for cfg, s in two:
        assert np.abs(s - ref).max() <= tol, cfg
    for cfg, s in one:
        assert np.abs(s - one[0][1]).max() <= 1e-6, cfg

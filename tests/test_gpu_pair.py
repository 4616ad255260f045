"""Parity of the paired-SM tensor-core step (tiling variant 2: a cluster of two CTAs shares each
M = 256 MMA; 2D tiles of 16 x 8 cells at 512 ordinates, 16 x 16 at 256) with the FP64 oracle, in
both tensor-core precisions (BF16 one pass; BF16X3 split operands).

Grids leave ragged tiles in x and y, hold interior tiles (the branch-free path) and boundary tiles
(the checked path); ordinate counts cover 256 and 512 and padded ones (Q = 200, 500: lanes past Q);
the full-size lattice launch the bench times is checked on sampled cells.  One step from a random
state is compared element by element within the derived BF16 one-step bound, a short run within
the whole-run tolerance.
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests.helpers import (RUN_TOL, ensure_built, gpu_problem, offdiag_rowsum, oracle_run, oracle_setup, rel_l2,
                           step_tolerance)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


def random_workload(nx, ny, npol, naz, beta=0.5, seed=0):
    return synth.Workload(f"pair{nx}x{ny}", "random", nx, ny, 0.0, nx * 0.05, 0.0, ny * 0.05, npol, naz, beta,
                          sigma_as=5.0, seed=seed)


def pair_problem(A, wl, psi0=None, precision="bf16"):
    p = gpu_problem(A, wl, precision, psi0=psi0)
    p.set_tiling(0, 0, 2)
    return p


# (nx, ny): ragged in both directions with interior tiles; exact multiples of both tile shapes; one
# tile; a single cell; a strip one row high; a tall thin grid
SHAPES = [(70, 37), (48, 48), (16, 8), (1, 1), (200, 1), (5, 90)]


@pytest.mark.parametrize("npol,naz", [(16, 32), (16, 16), (10, 50), (10, 20)])
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_one_step_random_state(A, nx, ny, npol, naz):
    wl = random_workload(nx, ny, npol, naz, seed=nx * 31 + ny + npol)
    p = pair_problem(A, wl)
    assert p.tiling()["tile_cells"] == (128 if npol * naz > 256 else 256)
    dt = 0.9 * p.max_stable_dt()
    p.step(1, dt)
    got = p.state()
    p.close()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step(wl.psi0(), K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    tol = step_tolerance("bf16", dt, wl.sigma_as, np.abs(wl.psi0()).max(), offdiag_rowsum(K))
    err = np.abs(got - ref).max()
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("npol,naz", [(16, 32), (16, 16), (10, 50)])
@pytest.mark.parametrize("nx,ny", [(70, 37), (16, 8), (1, 1)])
def test_split_one_step_random_state(A, nx, ny, npol, naz):
    """The split contraction (BF16X3: hi x hi + hi x lo + lo x hi) on the paired-SM kernel, within
    its derived one-step bound."""
    wl = random_workload(nx, ny, npol, naz, seed=nx * 17 + ny + npol)
    p = pair_problem(A, wl, precision="bf16x3")
    assert p.variant() == 2
    dt = 0.9 * p.max_stable_dt()
    p.step(1, dt)
    got = p.state()
    p.close()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step(wl.psi0(), K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    tol = step_tolerance("bf16x3", dt, wl.sigma_as, np.abs(wl.psi0()).max(), offdiag_rowsum(K))
    assert np.abs(got - ref).max() <= tol


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("npol,naz", [(16, 32), (16, 16)])
def test_agrees_with_persistent_kernel(A, npol, naz, precision):
    """Variant 2 and the one-CTA persistent kernel (variant 0) give the same step from the same state
    to FP32 rounding (both contract the same BF16 operands with FP32 accumulation)."""
    wl = random_workload(67, 29, npol, naz, seed=5)
    states = []
    for variant in (0, 2):
        p = gpu_problem(A, wl, precision)
        p.set_tiling(0, 0, variant)
        dt = 0.9 * p.max_stable_dt()
        p.step(1, dt)
        states.append(p.state())
        p.close()
    assert np.abs(states[0] - states[1]).max() <= 1e-6


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
def test_line_source_run(A, precision):
    """A whole short run (the 64^2 line source at 256 ordinates to t = 0.25): relative L2 of Phi
    against the oracle within the whole-run tolerance of the precision; the state stays non-negative."""
    wl = synth.line_source(64, 16, 16, 1.0 / 8.0, t_final=0.25, name="pair_ls64")
    n, dt = wl.steps()
    p = pair_problem(A, wl, precision=precision)
    p.step(n, dt)
    phi = p.scalar_flux()
    assert p.state().min() >= 0.0
    p.close()
    psi, w = oracle_run(wl, n, dt)
    assert rel_l2(phi, psi @ w) <= RUN_TOL[precision]


def test_lattice_run(A):
    """The lattice (Q = 512) on 56^2 cells to t = 0.5: absorbers, the source block and vacuum edges."""
    wl = synth.lattice(56, 16, 32, 0.5, t_final=0.5, name="pair_lat56")
    p = pair_problem(A, wl)
    # on this coarse grid CFL 0.5 exceeds the positivity bound of the sigma_a = 10 blocks: take
    # min(CFL h, 0.95 x bound), landing on t_final
    n = int(np.ceil(wl.t_final / min(wl.cfl * wl.h, 0.95 * p.max_stable_dt()) - 1e-12))
    dt = wl.t_final / n
    p.step(n, dt)
    phi = p.scalar_flux()
    p.close()
    psi, w = oracle_run(wl, n, dt)
    assert rel_l2(phi, psi @ w) <= RUN_TOL["bf16"]


def test_lattice_448_sampled_cells(A):
    """The full-size lattice launch (448 x 448, Q = 512) on the paired-SM kernel: one step from a seeded
    state against the oracle on sampled cells (tile corners and edges, grid corners, materials)."""
    wl = synth.LATTICE_448
    rng = np.random.default_rng(4)
    psi = rng.uniform(0.0, 1.0, size=(wl.ny, wl.nx, wl.Q))
    n, dt = wl.steps()
    cells = [(0, 0), (0, 447), (447, 0), (447, 447), (224, 224), (7, 15), (8, 16), (7, 16), (8, 15),
             (200, 63), (200, 64), (201, 127), (215, 128), (216, 128), (5, 383), (6, 384), (439, 431), (440, 432)]
    cells += [(int(j), int(i)) for j, i in rng.integers(0, 448, size=(16, 2))]
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step_at_cells(psi, cells, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    p = pair_problem(A, wl, psi0=psi)
    p.step(1, dt)
    got = p.state()
    p.close()
    tol = step_tolerance("bf16", dt, wl.sigma_as, 1.0, offdiag_rowsum(K))
    for n_, (j, i) in enumerate(cells):
        assert np.abs(got[j, i] - ref[n_]).max() <= tol, (j, i)


def test_unsupported_shapes(A):
    wl = random_workload(20, 20, 8, 16, seed=1)          # Q = 128: one 128-row block, no pair of rows
    p = gpu_problem(A, wl, "bf16")
    p.set_tiling(0, 0, 2)
    with pytest.raises(A.AssnError) as e:
        p.step(1, 0.5 * p.max_stable_dt())
    assert e.value.status == A._lib.ASSN_ERR_UNSUPPORTED
    p.close()
    wl = random_workload(20, 20, 16, 24, seed=1)         # Q = 384: three 128-row blocks
    p = gpu_problem(A, wl, "bf16x3")
    assert p.variant() == 0                              # the automatic choice falls back
    p.set_tiling(0, 0, 2)
    with pytest.raises(A.AssnError) as e:
        p.step(1, 0.5 * p.max_stable_dt())
    assert e.value.status == A._lib.ASSN_ERR_UNSUPPORTED
    p.close()


def test_automatic_variant(A):
    """The automatic choice: the paired-SM kernel for forward-Euler and Heun steps at 256 / 512
    ordinates in both tensor-core precisions, the one-CTA kernel for other ordinate counts."""
    for (npol, naz), prec, scheme, want in [((16, 32), "bf16", "euler", 2), ((16, 16), "bf16x3", "euler", 2),
                                            ((8, 16), "bf16", "euler", 0), ((16, 32), "bf16", "heun", 2),
                                            ((16, 16), "bf16x3", "heun", 2), ((8, 16), "bf16", "heun", 0)]:
        wl = random_workload(8, 8, npol, naz, seed=2)
        p = gpu_problem(A, wl, prec)
        p.set_scheme(scheme)
        assert p.variant() == want, (npol, naz, prec, scheme)
        p.close()


@pytest.mark.parametrize("npol,naz", [(16, 32), (16, 16)])
def test_resident_kernel_matrix_matches_ring(A, npol, naz):
    """With no kernel-matrix ring requested, the distinct blocks of G stay resident (at 512
    ordinates, numbered azimuth-major, 8 of each CTA's 16 blocks are distinct; at 256 its 4 blocks
    fit as they are); the MMAs read the same BF16 values in the same order as with the ring, so two
    steps are bitwise equal.  A quadrature numbered so that no two blocks are equal (the product set
    polar-major) streams G through the ring at 512 ordinates."""
    wl = random_workload(40, 21, npol, naz, seed=9)
    states = []
    for kernel_matrix in (0, 2):
        p = pair_problem(A, wl)
        p.set_rings(0, 0, kernel_matrix, 0)
        assert p.variant() == 2 and p.rings()["kernel_matrix"] == kernel_matrix
        dt = 0.9 * p.max_stable_dt()
        p.step(2, dt)
        states.append(p.state())
        p.close()
    assert np.array_equal(states[0], states[1])
    if npol * naz == 512:
        Om, w = O.product_quadrature(npol, naz)
        perm = np.array([k * npol + i for i in range(npol) for k in range(naz)])   # polar-major
        p = A.Problem(8, 8, 0.0, 0.4, 0.0, 0.4, "bf16").set_quadrature(Om[perm], w[perm])
        z = np.zeros((8, 8))
        p.set_cross_sections(z + 1.0, z + 0.5, z)
        p.set_artificial_scattering(5.0, wl.eps)
        p.set_tiling(0, 0, 2)
        assert p.rings()["kernel_matrix"] == 2
        p.close()


def heun_problem(A, wl, precision, psi0, variant=2):
    p = gpu_problem(A, wl, precision, psi0=psi0)
    p.set_scheme("heun")
    p.set_tiling(0, 0, variant)
    return p


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("npol,naz", [(16, 32), (16, 16), (10, 50), (10, 20)])
@pytest.mark.parametrize("nx,ny", [(70, 37), (16, 8), (1, 1), (5, 90), (3, 2)])
def test_heun_one_step(A, nx, ny, npol, naz, precision):
    """One Heun step (Sec. 3.1: two stages, minmod-limited second-order upwind transport) on the
    paired-SM kernel against oracle.step_heun: within twice the one-step bound of the precision (the
    second stage halves the sum of the first stage's error and its own)."""
    wl = random_workload(nx, ny, npol, naz, seed=nx * 13 + ny + naz)
    psi0 = wl.psi0()
    p = heun_problem(A, wl, precision, psi0)
    assert p.variant() == 2
    dt = 0.9 * p.max_stable_dt()
    l0 = p.launch_count()
    p.step(1, dt)
    assert p.launch_count() - l0 == 2
    got = p.state()
    p.close()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step_heun(psi0, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    scale = max(1.0, np.abs(ref).max(), np.abs(psi0).max())
    tol = 2.0 * step_tolerance(precision, dt, wl.sigma_as, scale, offdiag_rowsum(K))
    assert np.abs(got - ref).max() <= tol


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("npol,naz", [(16, 32), (10, 20)])
def test_heun_agrees_with_persistent_kernel(A, npol, naz, precision):
    """The paired-SM Heun stages and the one-CTA kernel's give the same two steps to FP32 rounding."""
    wl = random_workload(53, 27, npol, naz, seed=8)
    psi0 = wl.psi0()
    states = []
    for variant in (0, 2):
        p = heun_problem(A, wl, precision, psi0, variant)
        p.step(2, 0.9 * p.max_stable_dt())
        states.append(p.state())
        p.close()
    assert np.abs(states[0] - states[1]).max() <= 1e-6


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
def test_heun_line_source_run(A, precision):
    """The 64^2 line source at 256 ordinates under the paper's scheme at 0.95 of its admissible dt to
    t = 0.25: relative L2 of Phi against oracle.run_heun within the whole-run tolerance."""
    wl = synth.line_source(64, 16, 16, 1.0 / 8.0, t_final=0.25, name="pair_heun_ls64")
    p = gpu_problem(A, wl, precision)
    p.set_scheme("heun")
    assert p.variant() == 2
    n = int(np.ceil(wl.t_final / (0.95 * p.max_stable_dt()) - 1e-12))
    dt = wl.t_final / n
    p.step(n, dt)
    phi = p.scalar_flux()
    p.close()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    psi = O.run_heun(wl.psi0(), n, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    assert rel_l2(phi, psi @ w) <= RUN_TOL[precision]


@pytest.mark.parametrize("precision", ["bf16", "bf16x3"])
@pytest.mark.parametrize("npol,naz", [(16, 32), (8, 16)])
def test_step_device_on_caller_buffers(A, npol, naz, precision):
    """assn_step_device between caller-owned device buffers (torch tensors in the problem's padded
    layout) against assn_step from the same state: bitwise where both run on the paired-SM kernel
    (Q = 512); within FP32 rounding at Q = 128 (the one-tile-per-CTA kernel against the persistent
    one)."""
    import torch

    wl = random_workload(33, 18, npol, naz, seed=3)
    p = gpu_problem(A, wl, precision)
    qpad, _ = p.layout()
    dt = 0.9 * p.max_stable_dt()
    buf = np.zeros((wl.ny, wl.nx, qpad), dtype=np.float32)
    buf[..., :wl.Q] = wl.psi0()
    d_in = torch.from_numpy(buf).cuda()
    d_out = torch.full_like(d_in, -1.0)
    torch.cuda.synchronize()
    A._lib.assn_step_device(p.handle, d_in.data_ptr(), d_out.data_ptr(), dt)
    p.check_finite()                       # (syncs the problem's stream, where the step ran)
    out = d_out.cpu().numpy()
    assert np.all(out[..., wl.Q:] == 0.0)  # padded ordinates written as zeros
    p.step(1, dt)                          # the problem's own state is the same psi0
    ref = p.state()
    p.close()
    got = out[..., :wl.Q].astype(np.float64)
    if npol * naz == 512:
        assert np.array_equal(got, ref)
    else:
        assert np.abs(got - ref).max() <= 1e-6 * max(1.0, np.abs(ref).max())

"""The contractions that only the paired-SM kernel has, against the FP64 oracle:
- TF32 (tcgen05 kind::tf32, both operands rounded to TF32, FP32 accumulation, one pass);
- BF16X2 (the kernel matrix split into BF16 hi + lo, the flux in one BF16 part, two passes).

One step from a random state is compared element by element within the derived one-step bound of
each (`step_tolerance`), on grids with ragged tiles, interior and boundary tiles, at 256 and 512
ordinates and padded ones (Q = 200, 500); the same for one Heun step (Sec. 3.1).  The contraction
itself must equal the exact product of the rounded operands to FP32 arithmetic, and the TF32 error
must sit well below the BF16 error of the same step.  Whole short runs are held to the 1e-5 relative
L2 tolerance of the FP32 tier, the full-size lattice launch is checked on sampled cells, and every
path without these forms reports ASSN_ERR_UNSUPPORTED.
"""
import numpy as np
import pytest

import oracle as O
import synth
from tests.helpers import (RUN_TOL, ensure_built, gpu_problem, offdiag_rowsum, oracle_run, oracle_setup, rel_l2,
                           round_sig, round_tf32, step_tolerance)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


def random_workload(nx, ny, npol, naz, beta=0.5, seed=0):
    return synth.Workload(f"tf32_{nx}x{ny}", "random", nx, ny, 0.0, nx * 0.05, 0.0, ny * 0.05, npol, naz, beta,
                          sigma_as=5.0, seed=seed)


def one_step(A, wl, precision, dt=None, scheme="euler"):
    p = gpu_problem(A, wl, precision)
    p.set_scheme(scheme)
    assert p.variant() == 2
    dt = dt if dt is not None else 0.9 * p.max_stable_dt()
    p.step(1, dt)
    got = p.state()
    p.close()
    return got, dt


QUADS = [(16, 32), (16, 16), (10, 50), (10, 20)]
PRECS = ["tf32", "bf16x2"]


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("npol,naz", QUADS)
@pytest.mark.parametrize("nx,ny", [(70, 37), (48, 48), (16, 8), (1, 1), (200, 1), (5, 90)])
def test_one_step_random_state(A, nx, ny, npol, naz, precision):
    wl = random_workload(nx, ny, npol, naz, seed=nx * 23 + ny + npol)
    got, dt = one_step(A, wl, precision)
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step(wl.psi0(), K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    tol = step_tolerance(precision, dt, wl.sigma_as, np.abs(wl.psi0()).max(), offdiag_rowsum(K))
    err = np.abs(got - ref).max()
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("npol,naz", [(16, 32), (16, 16)])
def test_error_well_below_bf16(A, npol, naz):
    """The same step in TF32 and in BF16: the artificial-gain error (the part above FP32 rounding)
    is several times smaller in TF32 (2^-11 against 2^-8 per operand: eight times in the mean)."""
    wl = random_workload(64, 48, npol, naz, seed=77)
    Om, w, K, sa, ss, q = oracle_setup(wl)
    errs = {}
    for prec in ("tf32", "bf16"):
        got, dt = one_step(A, wl, prec)
        ref = O.step(wl.psi0(), K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
        errs[prec] = float(np.sqrt(np.mean((got - ref) ** 2)))
    assert errs["tf32"] <= errs["bf16"] / 4.0, errs


@pytest.mark.parametrize("precision", ["tf32", "bf16", "bf16x2"])
@pytest.mark.parametrize("npol,naz", [(16, 32), (16, 16)])
def test_contraction_is_the_product_of_rounded_operands(A, npol, naz, precision):
    """The tensor cores compute the product of the rounded operands to FP32 accuracy.  Expected
    step: the oracle's step plus the exact (FP64) change that rounding makes to its artificial
    gain, dt sigma_as [(G~ psi~ - e~ psi~) - (G psi - e psi)], with G the off-diagonal K, G~ its
    stored rounding (TF32: FP32 then TF32 with ties away; BF16: to nearest even from FP64; BF16X2:
    that hi plus its residual's BF16 rounding), psi~ the state's rounding, e~ the generator diagonal of G~ (as FP32).  The GPU step must agree
    with it to FP32 arithmetic, which is over 5x (TF32) and 40x (BF16) tighter than the rounding
    terms themselves (checked here), so an MMA that read its operands other than assumed
    (truncated, fewer bits) fails."""
    wl = random_workload(48, 40, npol, naz, seed=npol * naz + 3)
    psi = wl.psi0().astype(np.float32).astype(np.float64)   # the state as the library holds it
    p = gpu_problem(A, wl, precision, psi0=psi)
    assert p.variant() == 2
    dt = 0.9 * p.max_stable_dt()
    p.step(1, dt)
    got = p.state()
    p.close()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    G = K - np.diag(np.diag(K))
    if precision == "tf32":
        Gr, psir = round_tf32(G), round_tf32(psi)
    elif precision == "bf16x2":
        hi = round_sig(G, 8)
        Gr, psir = hi + round_sig(G - hi, 8), round_sig(psi, 8)
    else:
        Gr, psir = round_sig(G, 8), round_sig(psi, 8)
    e = (w[:, None] * G).sum(axis=0) / w                       # column normalisation
    er = ((w[:, None] * Gr).sum(axis=0) / w).astype(np.float32).astype(np.float64)
    delta = dt * wl.sigma_as * ((psir @ Gr.T - er * psir) - (psi @ G.T - e * psi))
    want = O.step(psi, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt) + delta
    tol = 4e-6 * np.abs(psi).max()                             # FP32 arithmetic of the step
    assert np.abs(delta).max() >= (5 if precision == "tf32" else 40) * tol
    assert np.abs(got - want).max() <= tol, (np.abs(got - want).max(), np.abs(delta).max())


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("npol,naz", QUADS)
@pytest.mark.parametrize("nx,ny", [(70, 37), (16, 8), (1, 1), (5, 90)])
def test_heun_one_step(A, nx, ny, npol, naz, precision):
    """One Heun step (two stages) against oracle.step_heun within twice the one-step bound."""
    wl = random_workload(nx, ny, npol, naz, seed=nx * 11 + ny + naz)
    psi0 = wl.psi0()
    got, dt = one_step(A, wl, precision, scheme="heun")
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step_heun(psi0, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    scale = max(1.0, np.abs(ref).max(), np.abs(psi0).max())
    tol = 2.0 * step_tolerance(precision, dt, wl.sigma_as, scale, offdiag_rowsum(K))
    assert np.abs(got - ref).max() <= tol


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("scheme", ["euler", "heun"])
def test_line_source_run(A, scheme, precision):
    """The 64^2 line source at 256 ordinates to t = 0.25 (forward Euler at CFL 0.5; Heun at 0.95 of
    its admissible dt): relative L2 of Phi against the oracle within 1e-5; the state stays
    non-negative."""
    wl = synth.line_source(64, 16, 16, 1.0 / 8.0, t_final=0.25, name="paired_ls64")
    p = gpu_problem(A, wl, precision)
    p.set_scheme(scheme)
    if scheme == "heun":
        n = int(np.ceil(wl.t_final / (0.95 * p.max_stable_dt()) - 1e-12))
        dt = wl.t_final / n
    else:
        n, dt = wl.steps()
    p.step(n, dt)
    phi = p.scalar_flux()
    assert p.state().min() >= 0.0
    p.close()
    if scheme == "heun":
        Om, w, K, sa, ss, q = oracle_setup(wl)
        psi = O.run_heun(wl.psi0(), n, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    else:
        psi, w = oracle_run(wl, n, dt)
    assert rel_l2(phi, psi @ w) <= RUN_TOL[precision]


@pytest.mark.parametrize("precision", PRECS)
def test_lattice_448_sampled_cells(A, precision):
    """The full-size lattice launch (448 x 448, Q = 512): one step from a seeded state against the
    oracle on sampled cells (tile corners and edges, grid corners, materials)."""
    wl = synth.LATTICE_448
    rng = np.random.default_rng(6)
    psi = rng.uniform(0.0, 1.0, size=(wl.ny, wl.nx, wl.Q))
    n, dt = wl.steps()
    cells = [(0, 0), (0, 447), (447, 0), (447, 447), (224, 224), (7, 15), (8, 16), (7, 16), (8, 15),
             (200, 63), (200, 64), (201, 127), (215, 128), (216, 128), (5, 383), (6, 384), (439, 431), (440, 432)]
    cells += [(int(j), int(i)) for j, i in rng.integers(0, 448, size=(16, 2))]
    Om, w, K, sa, ss, q = oracle_setup(wl)
    ref = O.step_at_cells(psi, cells, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    p = gpu_problem(A, wl, precision, psi0=psi)
    p.step(1, dt)
    got = p.state()
    p.close()
    tol = step_tolerance(precision, dt, wl.sigma_as, 1.0, offdiag_rowsum(K))
    for n_, (j, i) in enumerate(cells):
        assert np.abs(got[j, i] - ref[n_]).max() <= tol, (j, i)


@pytest.mark.parametrize("precision", PRECS)
def test_kernel_matrix_streams(A, precision):
    """The paired-SM kernel by default, with the kernel matrix through its ring (the resident form
    holds one BF16 part only), and the ring settings apply."""
    wl = random_workload(40, 21, 16, 32, seed=9)
    p = gpu_problem(A, wl, precision)
    assert p.variant() == 2
    assert p.rings()["kernel_matrix"] >= 2
    p.set_rings(3, 2, 2, 0)
    assert p.variant() == 2 and p.rings()["staging"] == 3
    p.close()


@pytest.mark.parametrize("precision", PRECS)
def test_step_device_on_caller_buffers(A, precision):
    """assn_step_device between 16-byte aligned caller buffers equals assn_step bitwise."""
    import torch

    wl = random_workload(33, 18, 16, 32, seed=3)
    p = gpu_problem(A, wl, precision)
    qpad, _ = p.layout()
    dt = 0.9 * p.max_stable_dt()
    buf = np.zeros((wl.ny, wl.nx, qpad), dtype=np.float32)
    buf[..., :wl.Q] = wl.psi0()
    d_in = torch.from_numpy(buf).cuda()
    d_out = torch.full_like(d_in, -1.0)
    torch.cuda.synchronize()
    A._lib.assn_step_device(p.handle, d_in.data_ptr(), d_out.data_ptr(), dt)
    p.check_finite()
    out = d_out.cpu().numpy()
    p.step(1, dt)
    ref = p.state()
    p.close()
    assert np.array_equal(out[..., :wl.Q].astype(np.float64), ref)


@pytest.mark.parametrize("precision", PRECS)
def test_unsupported_paths(A, precision):
    """Paths without these forms refuse them: other ordinate counts, the one-CTA variants, autotune,
    the implicit scheme and the server."""
    U = A._lib.ASSN_ERR_UNSUPPORTED
    wl = random_workload(20, 20, 8, 16, seed=1)          # Q = 128: no paired-SM form
    p = gpu_problem(A, wl, precision)
    with pytest.raises(A.AssnError) as e:
        p.step(1, 0.5 * p.max_stable_dt())
    assert e.value.status == U
    p.close()
    wl = random_workload(20, 20, 16, 32, seed=1)
    p = gpu_problem(A, wl, precision)
    for variant in (0, 1):
        with pytest.raises(A.AssnError) as e:
            p.set_tiling(0, 0, variant)
        assert e.value.status == U
    with pytest.raises(A.AssnError) as e:
        p.autotune(0.5 * p.max_stable_dt())
    assert e.value.status == U
    with pytest.raises(A.AssnError) as e:
        p.set_scheme("implicit")
    assert e.value.status == U
    p.close()   # (batches of paired members: tests/test_gpu_batch.py)
    with pytest.raises(A.AssnError) as e:
        A.Server(precision)
    assert e.value.status == U

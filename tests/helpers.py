"""Shared set-up for the GPU tests: build problems from synthetic workloads, run the oracle."""
from __future__ import annotations

import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402


def ensure_built():
    import __graft_entry__
    __graft_entry__._builder().build()


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_problem(A, wl: synth.Workload, precision: str, psi0=None, sigma_as=None, normalisation=None, kind=0):
    """The workload's problem through the C ABI: its quadrature, cross sections, kernel (normalisation
    from the workload unless given: 0 column, 1 row), scheme and initial state."""
    p = A.Problem(wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, precision)
    if wl.quadrature == "icosahedron":
        p.set_icosahedron_quadrature(wl.ico_order, wl.ico_base, wl.ico_midpoints)
    else:
        p.set_product_quadrature(wl.n_polar, wl.n_azim)
    sa, ss, q = wl.materials()
    p.set_cross_sections(sa, ss, q)
    if normalisation is None:
        normalisation = 1 if wl.normalisation == "row" else 0
    p.set_artificial_scattering(wl.sigma_as if sigma_as is None else sigma_as, wl.eps, kind, normalisation)
    if wl.scheme in ("heun", "implicit"):
        p.set_scheme(wl.scheme)
    if wl.scheme == "implicit":
        p.set_implicit_params(wl.si_eps, wl.gmres_tol)
    p.set_state(wl.psi0() if psi0 is None else psi0)
    return p


def oracle_setup(wl: synth.Workload, normalisation=None, kind="gauss"):
    if wl.quadrature == "icosahedron":
        Om, w = O.icosahedron_quadrature(wl.ico_order, wl.ico_base, wl.ico_midpoints)
    else:
        Om, w = O.product_quadrature(wl.n_polar, wl.n_azim)
    K = O.kernel_matrix(Om, w, wl.eps, kind=kind, normalisation=normalisation or wl.normalisation)
    sa, ss, q = wl.materials()
    return Om, w, K, sa, ss, q


def run_steps(wl: synth.Workload):
    """(n, dt) of a whole run of the workload; a fraction of the scheme's admissible dt (computed by the
    oracle) for workloads whose dt_rule is "bound"."""
    if wl.dt_rule != "bound":
        return wl.steps()
    Om, w, K, sa, ss, q = oracle_setup(wl)
    return wl.steps_for(O.heun_admissible_dt(Om, K, sa, ss, wl.sigma_as, wl.h))


def oracle_run(wl: synth.Workload, nsteps: int, dt: float, psi0=None, normalisation=None, sigma_as=None):
    """nsteps of the workload's scheme in the oracle; returns (psi, w)."""
    Om, w, K, sa, ss, q = oracle_setup(wl, normalisation)
    psi = wl.psi0() if psi0 is None else psi0
    s_as = wl.sigma_as if sigma_as is None else sigma_as
    if wl.scheme == "implicit":
        return O.implicit_run(psi, nsteps, K, Om, w, sa, ss, q, s_as, wl.h, dt, wl.si_eps, wl.gmres_tol), w
    run = O.run_heun if wl.scheme == "heun" else O.run
    return run(psi, nsteps, K, Om, w, sa, ss, q, s_as, wl.h, dt), w


def step_tolerance(precision: str, dt: float, sigma_as: float, scale: float, rowsum: float = 1.0) -> float:
    """Per-element bound on |GPU - FP64| after ONE step from the same state.

    ``scale`` bounds |psi|; ``rowsum`` bounds sum_{p != q} K_qp (above 1 for the column
    normalisation).  FP32 state arithmetic: a few ulps of the largest term (~1e-6 relative).
    BF16 contraction: both operands rounded to nearest BF16 (8-bit significand: relative error
    <= 2^-8 each), so the gain sum_p G_qp psi_p is off by <= (2^-7 + 2^-16) * rowsum * max|psi|; the
    loss term e_q psi_q uses the same rounded psi and e <= 1 built from the rounded G, off by
    <= 2^-7 * max|psi|; both enter multiplied by dt * sigma_as.  BF16X3 carries the residuals,
    leaving 2^-16 relative per operand plus the dropped lo*lo product: 2^-14 covers gain and loss.
    TF32: both operands rounded to 11 significant bits (2^-11 relative each, G after an FP32
    rounding of 2^-24), the same terms with 2^-10 in place of 2^-7.  BF16X2: G carried to 2^-16 by
    hi + lo, psi~ rounded to BF16 (2^-8), so gain and loss are each off by 2^-8 (1 + 2^-7) of theirs.
    """
    fp32 = 4e-6 * scale
    if precision == "fp64":
        return 1e-13 * scale
    if precision == "fp32":
        return fp32
    if precision == "bf16":
        return dt * sigma_as * 2.0 ** -7 * ((1.0 + 2.0 ** -9) * rowsum + 1.0) * scale + fp32
    if precision == "bf16x3":
        return dt * sigma_as * 2.0 ** -14 * (rowsum + 1.0) * scale + fp32
    if precision == "tf32":
        return dt * sigma_as * 2.0 ** -10 * ((1.0 + 2.0 ** -10) * rowsum + 1.0) * scale + fp32
    if precision == "bf16x2":
        return dt * sigma_as * 2.0 ** -8 * (1.0 + 2.0 ** -7) * (rowsum + 1.0) * scale + fp32
    raise ValueError(precision)


def round_sig(x, bits):
    """Round to nearest with ties to even at `bits` significant bits (normal range): BF16 is 8."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 2.0 ** bits), e - bits)


def round_tf32(x):
    """FP64 -> FP32 (to nearest even), then to TF32 by the library's stated rule: to nearest with
    ties away from zero at 11 significant bits, on the bit pattern's magnitude."""
    u = np.asarray(x, dtype=np.float64).astype(np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)


def offdiag_rowsum(K) -> float:
    K = np.asarray(K)
    return float((K.sum(axis=1) - np.diag(K)).max())


# relative L2 tolerance on the scalar flux of a whole run against the FP64 oracle
RUN_TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x3": 1e-5, "bf16x2": 1e-5, "tf32": 1e-5, "bf16": 1e-3}

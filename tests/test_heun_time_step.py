"""The time step of the paper's explicit runs (reading of Sec. 4.1).  The paper states dt/dx = 0.95 for
Heun + minmod; for the unsplit two-dimensional scheme on the paper's 200^2 line source with the N_q = 92
icosahedron quadrature that step is unstable, while 0.95 of the admissible dt of the limited scheme
(oracle.heun_admissible_dt) keeps the state non-negative."""
import numpy as np

import oracle as O
import synth
from helpers import oracle_setup, run_steps


def run_min_max(wl, dt, steps):
    Om, w, K, sa, ss, q = oracle_setup(wl)
    psi = wl.psi0()
    for _ in range(steps):
        psi = O.step_heun(psi, K, Om, w, sa, ss, q, wl.sigma_as, wl.h, dt)
    return psi.min(), np.abs(psi).max()


def test_literal_dt_over_dx_095_is_unstable_and_admissible_dt_is_not():
    wl = synth.PAPER_LINE_SOURCE_200
    peak = wl.psi0().max()
    lo, hi = run_min_max(wl, 0.95 * wl.h, 10)
    assert lo < -0.5 * peak and hi > 1.5 * peak            # large negative values after ten steps
    _, dt = run_steps(wl)
    assert 0.4 * wl.h < dt < 0.5 * wl.h
    lo, hi = run_min_max(wl, dt, 10)
    assert lo >= 0.0 and hi <= peak

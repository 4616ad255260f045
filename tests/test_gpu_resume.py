"""Checkpoint / resume: a solve stepped n1 steps, its state read back, a new problem set up from that
state and stepped n2 more is bitwise equal to the same solve stepped n1 + n2 steps without a break.
Forward Euler and the paper's Heun + minmod scheme, on the paired-SM kernel (Q = 512) and the one-CTA
kernel (Q = 128), in BF16 and BF16X3, and TF32 and BF16X2 on the paired-SM kernel; the checkpoint
goes through the FP32 state copies."""
import numpy as np
import pytest

import synth
from helpers import ensure_built, gpu_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


# (precision, n_polar, n_azim, variant): TF32 and BF16X2 have the paired-SM kernel only
CASES = [(prec, npol, naz, v) for prec in ("bf16", "bf16x3", "tf32", "bf16x2")
         for npol, naz, v in ((16, 32, 2), (8, 16, 0)) if prec in ("bf16", "bf16x3") or v == 2]


@pytest.mark.parametrize("scheme", ["euler", "heun"])
@pytest.mark.parametrize("precision,npol,naz,variant", CASES)
def test_resume_equals_continuous_run(A, npol, naz, variant, scheme, precision):
    wl = synth.Workload("resume", "random", 37, 19, 0.0, 1.85, 0.0, 0.95, npol, naz, 0.6, seed=npol + naz)

    def make(psi0=None):
        p = gpu_problem(A, wl, precision, psi0=psi0)
        p.set_scheme(scheme)
        return p

    n1, n2 = 3, 4
    p = make()
    assert p.variant() == variant
    dt = 0.9 * p.max_stable_dt()
    p.step(n1 + n2, dt)
    continuous = p.state()
    p.close()

    p = make()
    p.step(n1, dt)
    saved = np.empty((wl.ny, wl.nx, wl.Q), dtype=np.float32)
    A._lib.assn_get_state_f32(p.handle, saved)
    p.close()
    q = make(saved.astype(np.float64))
    q.step(n2, dt)
    resumed = q.state()
    q.close()
    assert np.array_equal(resumed, continuous)

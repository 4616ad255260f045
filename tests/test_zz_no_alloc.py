"""The allocation-free mass entry point agrees with the allocating one and with the FP64 oracle.

assn_mass_noalloc serves callers that cannot allocate device memory during a call (real-time loops
whose latency budget rules out allocator calls, hosts that run the library inside a memory pool of
their own); its partial sums live in a fixed device array.  This file runs last so that a failure
here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle as O
from tests.helpers import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


@pytest.mark.parametrize("precision", ["fp32", "fp64", "bf16"])
def test_mass_noalloc_matches_assn_mass(A, precision):
    import torch
    from paper_1911_08801_gb300 import _lib as L

    nx, ny, npol, naz = 70, 50, 8, 16
    p = A.Problem(nx, ny, 0.0, nx * 0.1, 0.0, ny * 0.1, precision).set_product_quadrature(npol, naz)
    rng = np.random.default_rng(17)
    z = np.zeros((ny, nx))
    p.set_cross_sections(z, np.ones((ny, nx)), z).set_artificial_scattering(5.0, 0.3)
    p.set_state(rng.uniform(0.0, 1.0, size=(ny, nx, npol * naz)))
    Qp, eb = p.layout()
    _, w = p.quadrature()
    # assn_mass weights an FP32 state with the FP32-rounded weights; pass the same weights so the two
    # reductions differ only in their summation order
    if eb == 4:
        w = w.astype(np.float32).astype(np.float64)
    w_dev = torch.zeros(Qp, dtype=torch.float64, device="cuda")
    w_dev[: len(w)] = torch.from_numpy(w)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = 0.5 * p.max_stable_dt()
    for call in range(2):            # two calls in a row; the state changes in between
        ref = p.mass()
        torch.cuda.synchronize()
        L.assn_mass_noalloc(p.state_device_ptr(), eb, w_dev.data_ptr(), nx * ny, Qp, p.h, out.data_ptr(),
                            torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)
        # the oracle's mass (h^2 sum_cells sum_q w_q psi_q in FP64) of the same state and weights
        exact = O.mass(p.state(), w, p.h)
        assert abs(got - exact) <= 1e-12 * abs(exact), (call, got, exact)
        p.step(1, dt)
    p.close()


def test_mass_noalloc_rejects_oversized_input(A):
    import torch
    from paper_1911_08801_gb300 import _lib as L

    big = L.lib  # noqa: F841  (library loaded)
    w_dev = torch.ones(64, dtype=torch.float64, device="cuda")
    psi = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    max_cells = 256 * 16384
    with pytest.raises(A.AssnError) as e:
        L.assn_mass_noalloc(psi.data_ptr(), 4, w_dev.data_ptr(), max_cells + 1, 64, 1.0, out.data_ptr())
    assert e.value.status == L.ASSN_ERR_ARG
    assert "ASSN_NOALLOC_MASS_MAX_CELLS" in L.assn_noalloc_last_error()

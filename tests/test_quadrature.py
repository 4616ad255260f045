"""The library's icosahedron quadrature (host code behind the C ABI; no device needed) against the
FP64 oracle at every order a problem accepts, on both base solids, and against the paper's printed
order-2 rule (Appendix A)."""
import math
import os

import numpy as np
import pytest

import oracle as O
from tests.helpers import ROOT, ensure_built


@pytest.fixture(scope="module")
def A():
    ensure_built()
    import paper_1911_08801_gb300 as A
    return A


def match(A_pts, B_pts, tol):
    d = np.linalg.norm(A_pts[:, None, :] - B_pts[None, :, :], axis=2)
    m = d.argmin(1)
    assert d.min(1).max() <= tol
    assert len(set(m.tolist())) == len(A_pts)
    return m


@pytest.mark.parametrize("midpoints", ["sphere", "flat"])
@pytest.mark.parametrize("base", ["printed", "regular"])
@pytest.mark.parametrize("order", list(range(2, 12)))
def test_library_matches_oracle(A, base, order, midpoints):
    om, w = A.icosahedron_quadrature(order, base, midpoints)
    ref_om, ref_w = O.icosahedron_quadrature(order, base, midpoints)
    assert om.shape == ref_om.shape == (10 * (order - 1) ** 2 + 2, 3)
    m = match(om, ref_om, 1e-14)
    assert np.abs(w - ref_w[m]).max() <= 1e-14 * max(1.0, ref_w.max())
    assert abs(w.sum() - 4 * math.pi) < 1e-12


def test_library_order2_is_the_printed_table(A):
    rows = [list(map(float, l.split())) for l in open(os.path.join(ROOT, "tests", "golden", "icosahedron_order2.txt"))
            if l.strip() and not l.startswith("#")]
    tab = np.array(rows)
    om, w = A.icosahedron_quadrature(2, "printed")
    m = match(tab[:, :3], om, 1e-15)
    assert np.abs(w[m] - tab[:, 3]).max() <= 1e-14


def test_high_order_counts(A):
    for order in (20, 64):
        om, w = A.icosahedron_quadrature(order, "regular")
        assert len(w) == 10 * (order - 1) ** 2 + 2
        assert np.all(w > 0) and abs(w.sum() - 4 * math.pi) < 1e-10
        assert abs(w @ om[:, 2] ** 4 - 4 * math.pi / 5) < 1e-10


def test_rejects_out_of_range(A):
    from paper_1911_08801_gb300 import _lib
    for order, base in ((1, 0), (0, 0), (65, 0), (2, 4), (2, -1), (3, 7)):
        assert _lib.lib.assn_icosahedron_quadrature(order, base, None, None, 0) == _lib.ASSN_ERR_ARG
    om = np.empty((12, 3))
    w = np.empty(12)
    assert _lib.lib.assn_icosahedron_quadrature(3, 0, om.ctypes.data_as(_lib._dp), w.ctypes.data_as(_lib._dp),
                                                12) == _lib.ASSN_ERR_ARG
    assert _lib.lib.assn_icosahedron_quadrature(3, 0, None, None, 0) == 42

"""Failure detection without a GPU fault: a bounded device wait that nothing completes gives up,
the host reads ASSN_ERR_TIMEOUT, and the context keeps working (a normal step afterwards is exact)."""
from __future__ import annotations

import time

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


def test_bounded_wait_gives_up_and_context_survives(A):
    wl = synth.Workload("ft", "random", 16, 16, 0.0, 0.8, 0.0, 0.8, 8, 8, 0.5, seed=5)
    p = gpu_problem(A, wl, "bf16")
    dt = 0.9 * p.max_stable_dt()
    p.step(2, dt)
    before = p.state()
    t0 = time.perf_counter()
    st = A._lib.assn_selftest_wait_timeout(20000)      # 20 ms limit
    el = time.perf_counter() - t0
    assert st == A._lib.ASSN_ERR_TIMEOUT
    assert el >= 0.015
    # the context is intact: the same problem steps on, and a fresh copy agrees bitwise
    p.step(2, dt)
    q = gpu_problem(A, wl, "bf16")
    q.step(4, dt)
    assert np.array_equal(p.state(), q.state())
    assert not np.array_equal(before, p.state())
    assert A._lib.assn_selftest_wait_timeout(0) == A._lib.ASSN_ERR_ARG
    p.close()
    q.close()

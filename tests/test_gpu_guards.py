"""Out-of-bounds write check of every kernel family: after steps on ragged grids with padded ordinate
counts, the guard regions around both state buffers still hold their fill byte and every padded
ordinate (Q <= q < Qpad) is still zero (assn_check_guards).  A write past a buffer's end or into a
padded ordinate by any kernel -- the paired-SM and one-CTA tensor-core steps, the tile-per-CTA
step, Heun stages, the CUDA-core steps, the implicit sweep, a batch -- fails here.
"""
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


def workload(nx, ny, npol, naz, seed):
    return synth.Workload(f"guard{nx}x{ny}q{npol * naz}", "random", nx, ny, 0.0, 0.05 * nx, 0.0, 0.05 * ny, npol,
                          naz, 0.5, sigma_as=5.0, seed=seed)


def assert_intact(p):
    g = p.check_guards()
    assert g == {"guard_bytes_changed": 0, "padding_nonzero": 0}, g


# (precision, variant, scheme, (nx, ny), (n_polar, n_azim)): Q = 500 and 200 leave padded ordinates in
# 512 / 256 (the paired-SM kernel streams the kernel matrix at 500, keeps it resident at 200),
# Q = 12 pads to 64, Q = 192 fills its stride
CASES = [
    ("bf16", 2, "euler", (70, 37), (10, 50)),
    ("bf16", 2, "euler", (33, 21), (10, 20)),
    ("bf16", 2, "euler", (17, 9), (16, 32)),
    ("bf16x3", 2, "euler", (70, 37), (10, 50)),
    ("bf16x3", 2, "euler", (19, 23), (10, 20)),
    ("tf32", 2, "euler", (70, 37), (10, 50)),
    ("tf32", 2, "heun", (19, 23), (10, 20)),
    ("bf16x2", 2, "euler", (70, 37), (10, 50)),
    ("bf16x2", 2, "heun", (19, 23), (10, 20)),
    ("bf16", 0, "euler", (70, 37), (10, 50)),
    ("bf16", 0, "euler", (41, 13), (3, 4)),
    ("bf16x3", 0, "euler", (41, 13), (8, 24)),
    ("bf16", 1, "euler", (29, 11), (8, 24)),
    ("bf16", 0, "heun", (33, 21), (10, 20)),
    ("bf16x3", 0, "heun", (21, 17), (3, 4)),
    ("fp32", None, "euler", (23, 19), (3, 4)),
    ("fp64", None, "euler", (23, 19), (3, 4)),
    ("fp32", None, "heun", (23, 19), (3, 4)),
    ("fp32", None, "implicit", (12, 10), (3, 4)),
]


@pytest.mark.parametrize("precision,variant,scheme,grid,quad", CASES)
def test_guards_intact_after_steps(A, precision, variant, scheme, grid, quad):
    wl = workload(*grid, *quad, seed=grid[0] + quad[1])
    p = gpu_problem(A, wl, precision)
    assert_intact(p)
    if variant is not None:
        p.set_tiling(0, 0, variant)
    if scheme != "euler":
        p.set_scheme(scheme)
    dt = 0.9 * p.max_stable_dt() if scheme != "implicit" else 0.5 * wl.h
    p.step(3, dt)
    p.check_finite()
    assert_intact(p)
    p.close()


def test_guards_intact_after_batch(A):
    """Members of uneven grid and ordinate count stepped together (one launch per class and step)."""
    wls = [workload(70, 37, 10, 50, 1), workload(41, 13, 3, 4, 2), workload(19, 23, 10, 20, 3)]
    probs = [gpu_problem(A, wl, "bf16") for wl in wls]
    with A.Batch() as bt:
        for p in probs:
            bt.add(p, 3, 0.9 * p.max_stable_dt())
        bt.run().sync()
    for p in probs:
        assert_intact(p)
        p.close()


def test_guards_see_a_padding_write(A):
    """The check itself: a nonzero value placed in a padded ordinate through the device pointer is
    counted (the state's own API never writes there)."""
    import torch

    wl = workload(9, 7, 3, 4, 5)
    p = gpu_problem(A, wl, "fp32")
    qpad, elem = p.layout()
    assert qpad == 64 and elem == 4
    p.check_finite()                     # the problem's stream is idle

    class Cell0Ordinate12:               # cell 0, ordinate 12: in the allocation, past the Q = 12 live ordinates
        __cuda_array_interface__ = {"shape": (1,), "typestr": "<f4", "version": 3,
                                    "data": (p.state_device_ptr() + 12 * 4, False)}

    torch.as_tensor(Cell0Ordinate12(), device="cuda").fill_(1.0)
    torch.cuda.synchronize()
    assert p.check_guards() == {"guard_bytes_changed": 0, "padding_nonzero": 1}
    p.close()

"""GB300-native explicit as-S_N time step (arXiv:1911.08801) behind a C ABI.

``_lib`` binds every entry point of ``include/assn.h`` under its own name; ``Problem`` is a
small owner object around one problem handle.  All arithmetic of the step runs in the CUDA
kernels of ``libassn.so``; importing this package fails when that library is not built.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import (ASSN_BF16, ASSN_BF16X3, ASSN_FP32, ASSN_FP64, ASSN_KERNEL_EXP, ASSN_KERNEL_GAUSS,
                   ASSN_NORM_COLUMN, ASSN_NORM_ROW, ASSN_TF32, ASSN_BF16X2, PRECISIONS, AssnError)

__all__ = ["Problem", "Batch", "Server", "AssnError", "PRECISIONS", "ASSN_FP64", "ASSN_FP32", "ASSN_BF16", "ASSN_BF16X3",
           "ASSN_TF32", "ASSN_BF16X2",
           "ASSN_KERNEL_GAUSS", "ASSN_KERNEL_EXP", "ASSN_NORM_COLUMN", "ASSN_NORM_ROW", "icosahedron_quadrature"]


def icosahedron_quadrature(order: int, base: str = "printed", midpoints: str = "sphere"):
    """(Omega [N_q, 3], w [N_q]) of the icosahedron quadrature of Sec. 3.3, N_q = 10 (order-1)^2 + 2,
    computed by the library (host code, no device needed); midpoints "sphere" or "flat" selects the
    reading of the dual cell."""
    return _lib.assn_icosahedron_quadrature(order, _lib.ICO_BASES[base] | _lib.ICO_MIDPOINTS[midpoints])


class Problem:
    """One as-S_N problem on the current CUDA device (owns its device memory)."""

    def __init__(self, nx: int, ny: int, x0: float, x1: float, y0: float, y1: float,
                 precision="bf16", stream=None):
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.handle = None
        self.handle = _lib.assn_create(nx, ny, x0, x1, y0, y1, self.precision, stream)
        self.nx, self.ny = nx, ny
        self.h = (x1 - x0) / nx
        self.Q = 0

    # -- set-up
    def set_product_quadrature(self, n_polar: int, n_azim: int):
        _lib.assn_set_product_quadrature(self.handle, n_polar, n_azim)
        self.Q = n_polar * n_azim
        return self

    def set_implicit_params(self, si_eps: float = 1e-4, gmres_tol: float = 1.5e-8, restart: int = 30,
                            max_si: int = 1000, max_gmres: int = 500):
        """Tolerances and limits of the implicit scheme (source iteration, GMRES; Alg. 1-3)."""
        _lib.assn_set_implicit_params(self.handle, si_eps, gmres_tol, restart, max_si, max_gmres)
        return self

    def implicit_stats(self) -> dict:
        return _lib.assn_implicit_stats(self.handle)

    def implicit_source_iteration(self, dt: float, R, psi0, iterations: int) -> np.ndarray:
        """Exactly `iterations` source iterations for (L - dt sigma_as K) psi = dt R from psi0."""
        return _lib.assn_implicit_source_iteration(self.handle, dt, R, psi0, iterations)

    def set_icosahedron_quadrature(self, order: int, base: str = "printed", midpoints: str = "sphere"):
        """The icosahedron quadrature of Sec. 3.3 (N_q = 10 (order-1)^2 + 2); base "printed" reproduces
        the paper's printed order-2 rule, "regular" builds on the regular icosahedron; midpoints
        "sphere" or "flat" selects the reading of the dual cell (they agree at order 2)."""
        _lib.assn_set_icosahedron_quadrature(self.handle, order,
                                             _lib.ICO_BASES[base] | _lib.ICO_MIDPOINTS[midpoints])
        self.Q = 10 * (order - 1) ** 2 + 2
        return self

    def set_quadrature(self, omega, w):
        _lib.assn_set_quadrature(self.handle, omega, w)
        self.Q = len(w)
        return self

    def quadrature(self):
        return _lib.assn_get_quadrature(self.handle)

    def set_cross_sections(self, sigma_a, sigma_s, q):
        _lib.assn_set_cross_sections(self.handle, sigma_a, sigma_s, q)
        return self

    def set_artificial_scattering(self, sigma_as: float, eps: float, kernel_kind: int = ASSN_KERNEL_GAUSS,
                                  normalisation: int = ASSN_NORM_COLUMN):
        _lib.assn_set_artificial_scattering(self.handle, sigma_as, eps, kernel_kind, normalisation)
        return self

    def kernel_matrix(self) -> np.ndarray:
        return _lib.assn_get_kernel_matrix(self.handle, self.Q)

    # -- state
    def set_state(self, psi):
        _lib.assn_set_state(self.handle, psi)
        return self

    def state(self) -> np.ndarray:
        return _lib.assn_get_state(self.handle, (self.ny, self.nx, self.Q))

    def init_line_source(self, delta: float = 0.03 ** 2, floor_value: float = 1e-4):
        _lib.assn_init_line_source(self.handle, delta, floor_value)
        return self

    # -- stepping and diagnostics
    def set_scheme(self, scheme="euler"):
        """"euler" (forward Euler, first-order upwind) or "heun" (Heun + minmod, FP32 / FP64)."""
        _lib.assn_set_scheme(self.handle, _lib.SCHEMES[scheme] if isinstance(scheme, str) else int(scheme))
        return self

    def scheme(self) -> int:
        return _lib.assn_get_scheme(self.handle)

    def max_stable_dt(self) -> float:
        return _lib.assn_max_stable_dt(self.handle)

    def step(self, nsteps: int, dt: float):
        _lib.assn_step(self.handle, nsteps, dt)
        return self

    def scalar_flux(self) -> np.ndarray:
        return _lib.assn_scalar_flux(self.handle, (self.ny, self.nx))

    def mass(self) -> float:
        return _lib.assn_mass(self.handle)

    def check_finite(self):
        _lib.assn_check_finite(self.handle)

    def check_guards(self) -> dict:
        """Guard bytes around the state buffers that changed and padded ordinates that are not zero
        (both 0 while every kernel kept to its cells and ordinates)."""
        return _lib.assn_check_guards(self.handle)

    def set_tiling(self, tile_cells: int = 0, stages: int = 0, variant: int = 0):
        _lib.assn_set_tiling(self.handle, tile_cells, stages, variant)
        return self

    def tiling(self) -> dict:
        return _lib.assn_get_tiling(self.handle)

    def variant(self) -> int:
        """The tensor-core kernel the next step runs (0, 1 or 2; the automatic choice resolved)."""
        return _lib.assn_get_variant(self.handle)

    def set_rings(self, staging: int = 0, operand: int = 0, kernel_matrix: int = 0, blocks_per_request: int = 0):
        _lib.assn_set_rings(self.handle, staging, operand, kernel_matrix, blocks_per_request)
        return self

    def rings(self) -> dict:
        return _lib.assn_get_rings(self.handle)

    def autotune(self, dt: float, use_cache: bool = True) -> dict:
        return _lib.assn_autotune(self.handle, dt, use_cache)

    def layout(self):
        return _lib.assn_layout(self.handle)

    def state_device_ptr(self) -> int:
        return _lib.assn_state_device(self.handle)

    def launch_count(self) -> int:
        return _lib.assn_launch_count(self.handle)

    def close(self):
        if self.handle:
            _lib.assn_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several problems advanced by one persistent tensor-core launch per step (include/assn.h)."""

    def __init__(self, stream=None):
        self.handle = None
        self.handle = _lib.assn_batch_create(stream)
        self.members: list[Problem] = []

    def add(self, problem: Problem, nsteps: int, dt: float):
        _lib.assn_batch_add(self.handle, problem.handle, nsteps, dt)
        self.members.append(problem)
        return self

    def set_steps(self, problem: Problem, nsteps: int, dt: float):
        _lib.assn_batch_set_steps(self.handle, problem.handle, nsteps, dt)
        return self

    def remove(self, problem: Problem):
        _lib.assn_batch_remove(self.handle, problem.handle)
        self.members.remove(problem)
        return self

    def set_tiling(self, tile_cells: int = 0, stages: int = 0):
        _lib.assn_batch_set_tiling(self.handle, tile_cells, stages)
        return self

    def set_grouping(self, one_launch: bool = False):
        """one_launch: every member in one persistent launch per step (else one per ordinate class)."""
        _lib.assn_batch_set_grouping(self.handle, one_launch)
        return self

    def autotune(self, use_cache: bool = True) -> dict:
        return _lib.assn_batch_autotune(self.handle, use_cache)

    def run(self, use_graph: bool = True):
        _lib.assn_batch_run(self.handle, use_graph)
        return self

    def sync(self):
        _lib.assn_batch_sync(self.handle)
        return self

    def info(self) -> dict:
        return _lib.assn_batch_info(self.handle)

    def classes(self) -> list[dict]:
        return _lib.assn_batch_classes(self.handle)

    def close(self):
        if self.handle:
            _lib.assn_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop over whole solves with continuous batching (include/assn.h, assn_server_*)."""

    def __init__(self, precision="bf16", hbm_budget_bytes: int = 0, max_active: int = 64, chunk_steps: int = 8,
                 use_graph: bool = True):
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.handle = None
        self.handle = _lib.assn_server_create(self.precision, hbm_budget_bytes, max_active, chunk_steps, use_graph)
        self._shapes: dict[int, tuple[int, int]] = {}

    def submit(self, nx: int, ny: int, x0: float, x1: float, y0: float, y1: float, n_polar: int, n_azim: int,
               sigma_as: float, eps: float, sigma_a, sigma_s, q, nsteps: int, dt: float, init="line_source",
               delta: float = 0.03 ** 2, floor_value: float = 1e-4, kernel_kind: int = ASSN_KERNEL_GAUSS,
               normalisation: int = ASSN_NORM_COLUMN) -> int:
        """Queue one solve; ``init`` is "line_source", "zero" or a [ny][nx][Q] state.  Returns its id."""
        sa = np.ascontiguousarray(sigma_a, dtype=np.float64)
        ss = np.ascontiguousarray(sigma_s, dtype=np.float64)
        qq = np.ascontiguousarray(q, dtype=np.float64)
        for a in (sa, ss, qq):
            if a.size != nx * ny:
                raise ValueError("cell fields must hold ny*nx values")
        psi = None
        if isinstance(init, str):
            kind = {"line_source": _lib.ASSN_INIT_LINE_SOURCE, "zero": _lib.ASSN_INIT_ZERO}[init]
        else:
            kind = _lib.ASSN_INIT_STATE
            psi = np.ascontiguousarray(init, dtype=np.float32)
            if psi.size != nx * ny * n_polar * n_azim:
                raise ValueError("state must hold ny*nx*Q values")
        req = _lib.AssnRequest(nx, ny, x0, x1, y0, y1, n_polar, n_azim, sigma_as, eps, kernel_kind, normalisation,
                               _lib._d(sa), _lib._d(ss), _lib._d(qq), kind, delta, floor_value,
                               psi.ctypes.data_as(_lib._fp) if psi is not None else None, nsteps, dt)
        rid = _lib.assn_server_submit(self.handle, req)
        self._shapes[rid] = (ny, nx)
        return rid

    def wait(self, rid: int, timeout_s: float = -1.0):
        """(scalar flux [ny][nx], latency s, queueing s) of request ``rid``; releases it."""
        phi = np.empty(self._shapes[rid])
        try:
            lat, qs = _lib.assn_server_wait(self.handle, rid, timeout_s, phi)
        except AssnError as e:
            if e.status != _lib.ASSN_ERR_TIMEOUT:   # the request is released unless still pending
                del self._shapes[rid]
            raise
        del self._shapes[rid]
        return phi, lat, qs

    def cancel(self, rid: int):
        """Cancel request ``rid``: dropped from the queue, or retired at the next chunk boundary;
        ``wait`` then raises AssnError with ASSN_ERR_CANCELLED."""
        _lib.assn_server_cancel(self.handle, rid)

    def stats(self) -> dict:
        return _lib.assn_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            _lib.assn_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

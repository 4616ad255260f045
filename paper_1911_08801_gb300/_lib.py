"""ctypes binding of libassn (include/assn.h): the same entry points, argument marshalling only.

Every function here converts Python/numpy arguments to the C types, calls the entry point of
the same name and raises ``AssnError`` on a non-zero status.  No step of the method runs in
Python.  Importing fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libassn.so")

ASSN_OK = 0
ASSN_ERR_ARG = -1
ASSN_ERR_OOM = -2
ASSN_ERR_CUDA = -3
ASSN_ERR_UNSTABLE = -4
ASSN_ERR_NONFINITE = -5
ASSN_ERR_TIMEOUT = -6
ASSN_ERR_STATE = -7
ASSN_ERR_UNSUPPORTED = -8
ASSN_ERR_CANCELLED = -9

ASSN_FP64, ASSN_FP32, ASSN_BF16, ASSN_BF16X3, ASSN_TF32, ASSN_BF16X2 = 0, 1, 2, 3, 4, 5
ASSN_KERNEL_GAUSS, ASSN_KERNEL_EXP = 0, 1
ASSN_NORM_COLUMN, ASSN_NORM_ROW = 0, 1
ASSN_SCHEME_EULER_UPWIND, ASSN_SCHEME_HEUN_MINMOD, ASSN_SCHEME_IMPLICIT = 0, 1, 2
ASSN_ICO_PRINTED, ASSN_ICO_REGULAR, ASSN_ICO_FLAT_MIDPOINTS = 0, 1, 2
ASSN_ICO_MAX_ORDER = 64
ICO_BASES = {"printed": ASSN_ICO_PRINTED, "regular": ASSN_ICO_REGULAR}
ICO_MIDPOINTS = {"sphere": 0, "flat": ASSN_ICO_FLAT_MIDPOINTS}
SCHEMES = {"euler": ASSN_SCHEME_EULER_UPWIND, "heun": ASSN_SCHEME_HEUN_MINMOD, "implicit": ASSN_SCHEME_IMPLICIT}

PRECISIONS = {"fp64": ASSN_FP64, "fp32": ASSN_FP32, "bf16": ASSN_BF16, "bf16x3": ASSN_BF16X3, "tf32": ASSN_TF32,
              "bf16x2": ASSN_BF16X2}

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_vp = C.c_void_p
_h = C.c_void_p

ASSN_INIT_LINE_SOURCE, ASSN_INIT_ZERO, ASSN_INIT_STATE = 0, 1, 2


class AssnRequest(C.Structure):
    """assn_request (include/assn.h)."""
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double),
                ("y1", C.c_double), ("n_polar", C.c_int), ("n_azim", C.c_int), ("sigma_as", C.c_double),
                ("eps", C.c_double), ("kernel_kind", C.c_int), ("normalisation", C.c_int),
                ("sigma_a", _dp), ("sigma_s", _dp), ("q", _dp), ("init_kind", C.c_int), ("delta", C.c_double),
                ("floor_value", C.c_double), ("psi0", _fp), ("nsteps", C.c_int), ("dt", C.c_double)]


class AssnServerStats(C.Structure):
    """assn_server_stats (include/assn.h)."""
    _fields_ = [(n, C.c_int64) for n in ("submitted", "completed", "failed", "active", "queued", "max_active_seen",
                                         "launches")] + \
               [(n, C.c_double) for n in ("p50_latency_s", "p99_latency_s", "mean_latency_s", "busy_s", "wall_s",
                                          "updates", "updates_per_s")] + \
               [("budget_bytes", C.c_int64), ("peak_bytes", C.c_int64)]


# name -> (restype, argtypes); every function declared in include/assn.h
SIGNATURES = {
    "assn_create": (C.c_int, [C.POINTER(_h), C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                              C.c_int, _vp]),
    "assn_destroy": (C.c_int, [_h]),
    "assn_set_quadrature": (C.c_int, [_h, C.c_int, _dp, _dp]),
    "assn_set_product_quadrature": (C.c_int, [_h, C.c_int, C.c_int]),
    "assn_get_quadrature": (C.c_int, [_h, C.POINTER(C.c_int), _dp, _dp]),
    "assn_icosahedron_quadrature": (C.c_int, [C.c_int, C.c_int, _dp, _dp, C.c_int]),
    "assn_set_icosahedron_quadrature": (C.c_int, [_h, C.c_int, C.c_int]),
    "assn_set_cross_sections": (C.c_int, [_h, _dp, _dp, _dp]),
    "assn_set_artificial_scattering": (C.c_int, [_h, C.c_double, C.c_double, C.c_int, C.c_int]),
    "assn_get_kernel_matrix": (C.c_int, [_h, _dp]),
    "assn_set_state": (C.c_int, [_h, _dp]),
    "assn_get_state": (C.c_int, [_h, _dp]),
    "assn_set_state_f32": (C.c_int, [_h, _fp]),
    "assn_get_state_f32": (C.c_int, [_h, _fp]),
    "assn_init_line_source": (C.c_int, [_h, C.c_double, C.c_double]),
    "assn_max_stable_dt": (C.c_int, [_h, _dp]),
    "assn_step": (C.c_int, [_h, C.c_int, C.c_double]),
    "assn_set_scheme": (C.c_int, [_h, C.c_int]),
    "assn_set_implicit_params": (C.c_int, [_h, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int]),
    "assn_implicit_stats": (C.c_int, [_h, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "assn_implicit_source_iteration": (C.c_int, [_h, C.c_double, _dp, _dp, C.c_int, _dp]),
    "assn_get_scheme": (C.c_int, [_h, C.POINTER(C.c_int)]),
    "assn_step_device": (C.c_int, [_h, _vp, _vp, C.c_double]),
    "assn_run_f32": (C.c_int, [_h, _fp, C.c_int, C.c_double, _dp]),
    "assn_set_tiling": (C.c_int, [_h, C.c_int, C.c_int, C.c_int]),
    "assn_set_rings": (C.c_int, [_h, C.c_int, C.c_int, C.c_int, C.c_int]),
    "assn_get_rings": (C.c_int, [_h, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_int)]),
    "assn_get_tiling": (C.c_int, [_h, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int64)]),
    "assn_get_variant": (C.c_int, [_h, C.POINTER(C.c_int)]),
    "assn_layout": (C.c_int, [_h, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "assn_state_device": (C.c_int, [_h, C.POINTER(_vp)]),
    "assn_scalar_flux": (C.c_int, [_h, _dp]),
    "assn_scalar_flux_device": (C.c_int, [_h, _vp]),
    "assn_mass": (C.c_int, [_h, _dp]),
    "assn_check_finite": (C.c_int, [_h]),
    "assn_check_guards": (C.c_int, [_h, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "assn_last_error": (C.c_char_p, [_h]),
    "assn_status_string": (C.c_char_p, [C.c_int]),
    "assn_launch_count": (C.c_int64, [_h]),
    "assn_abi_version": (C.c_int, []),
    "assn_selftest_wait_timeout": (C.c_int, [C.c_int]),
    "assn_batch_create": (C.c_int, [C.POINTER(_h), _vp]),
    "assn_batch_destroy": (C.c_int, [_h]),
    "assn_batch_add": (C.c_int, [_h, _h, C.c_int, C.c_double]),
    "assn_batch_set_steps": (C.c_int, [_h, _h, C.c_int, C.c_double]),
    "assn_batch_remove": (C.c_int, [_h, _h]),
    "assn_batch_set_tiling": (C.c_int, [_h, C.c_int, C.c_int]),
    "assn_batch_set_grouping": (C.c_int, [_h, C.c_int]),
    "assn_batch_autotune": (C.c_int, [_h, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _dp]),
    "assn_batch_run": (C.c_int, [_h, C.c_int]),
    "assn_batch_sync": (C.c_int, [_h]),
    "assn_batch_info": (C.c_int, [_h, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "assn_batch_classes": (C.c_int, [_h, C.POINTER(C.c_int)]),
    "assn_batch_class_info": (C.c_int, [_h, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "assn_batch_last_error": (C.c_char_p, [_h]),
    "assn_autotune": (C.c_int, [_h, C.c_double, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _dp]),
    "assn_footprint_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "assn_server_create": (C.c_int, [C.POINTER(_h), C.c_int, C.c_size_t, C.c_int, C.c_int, C.c_int]),
    "assn_server_submit": (C.c_int, [_h, C.POINTER(AssnRequest), C.POINTER(C.c_int64)]),
    "assn_server_wait": (C.c_int, [_h, C.c_int64, C.c_double, _dp, _dp, _dp]),
    "assn_server_cancel": (C.c_int, [_h, C.c_int64]),
    "assn_server_get_stats": (C.c_int, [_h, C.POINTER(AssnServerStats)]),
    "assn_server_destroy": (C.c_int, [_h]),
    "assn_server_last_error": (C.c_char_p, []),
    "assn_mass_noalloc": (C.c_int, [_vp, C.c_int, _vp, C.c_int, C.c_int, C.c_double, _vp, _vp]),
    "assn_noalloc_last_error": (C.c_char_p, []),
}


class AssnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libassn.so is not built ({LIB_PATH}); run paper_1911_08801_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def status_string(status: int) -> str:
    return lib.assn_status_string(status).decode()


def _check(status: int, handle=None):
    if status != ASSN_OK:
        raise AssnError(status, lib.assn_last_error(handle).decode())


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _contig(a, dtype=np.float64) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def assn_create(nx: int, ny: int, x0: float, x1: float, y0: float, y1: float, precision: int,
                stream=None) -> int:
    h = _h()
    _check(lib.assn_create(C.byref(h), nx, ny, x0, x1, y0, y1, precision, _stream_ptr(stream)), None)
    return h.value


def assn_destroy(h: int) -> None:
    _check(lib.assn_destroy(h), h)


def assn_set_quadrature(h: int, omega, w) -> None:
    om = _contig(omega).reshape(-1, 3)
    ww = _contig(w)
    _check(lib.assn_set_quadrature(h, len(ww), _d(om), _d(ww)), h)


def assn_set_product_quadrature(h: int, n_polar: int, n_azim: int) -> None:
    _check(lib.assn_set_product_quadrature(h, n_polar, n_azim), h)


def assn_icosahedron_quadrature(order: int, base: int = ASSN_ICO_PRINTED):
    """(omega [N_q, 3], w [N_q]) of the icosahedron quadrature, computed by the library on the host."""
    n = lib.assn_icosahedron_quadrature(order, base, None, None, 0)
    if n < 0:
        raise AssnError(n, f"icosahedron quadrature: order {order} or base {base} out of range")
    om = np.empty((n, 3))
    w = np.empty(n)
    r = lib.assn_icosahedron_quadrature(order, base, _d(om), _d(w), n)
    if r != n:
        raise AssnError(r if r < 0 else ASSN_ERR_STATE, "icosahedron quadrature failed")
    return om, w


def assn_set_icosahedron_quadrature(h: int, order: int, base: int = ASSN_ICO_PRINTED) -> None:
    _check(lib.assn_set_icosahedron_quadrature(h, order, base), h)


def assn_get_quadrature(h: int):
    q = C.c_int(0)
    _check(lib.assn_get_quadrature(h, C.byref(q), None, None), h)
    om = np.empty((q.value, 3))
    w = np.empty(q.value)
    _check(lib.assn_get_quadrature(h, C.byref(q), _d(om), _d(w)), h)
    return om, w


def assn_set_cross_sections(h: int, sigma_a, sigma_s, q) -> None:
    a, s, src = _contig(sigma_a), _contig(sigma_s), _contig(q)
    _check(lib.assn_set_cross_sections(h, _d(a), _d(s), _d(src)), h)


def assn_set_artificial_scattering(h: int, sigma_as: float, eps: float, kernel_kind: int = ASSN_KERNEL_GAUSS,
                                   normalisation: int = ASSN_NORM_COLUMN) -> None:
    _check(lib.assn_set_artificial_scattering(h, sigma_as, eps, kernel_kind, normalisation), h)


def assn_get_kernel_matrix(h: int, Q: int) -> np.ndarray:
    K = np.empty((Q, Q))
    _check(lib.assn_get_kernel_matrix(h, _d(K)), h)
    return K


def assn_set_state(h: int, psi) -> None:
    a = _contig(psi)
    _check(lib.assn_set_state(h, _d(a)), h)


def assn_get_state(h: int, shape) -> np.ndarray:
    out = np.empty(shape)
    _check(lib.assn_get_state(h, _d(out)), h)
    return out


def assn_set_state_f32(h: int, psi: np.ndarray) -> None:
    """``psi`` must stay alive and unchanged until the problem's stream has passed the copy."""
    assert psi.dtype == np.float32 and psi.flags.c_contiguous
    _check(lib.assn_set_state_f32(h, psi.ctypes.data_as(_fp)), h)


def assn_get_state_f32(h: int, out: np.ndarray) -> np.ndarray:
    assert out.dtype == np.float32 and out.flags.c_contiguous
    _check(lib.assn_get_state_f32(h, out.ctypes.data_as(_fp)), h)
    return out


def assn_init_line_source(h: int, delta: float = 0.03 ** 2, floor_value: float = 1e-4) -> None:
    _check(lib.assn_init_line_source(h, delta, floor_value), h)


def assn_max_stable_dt(h: int) -> float:
    v = C.c_double(0)
    _check(lib.assn_max_stable_dt(h, C.byref(v)), h)
    return v.value


def assn_step(h: int, nsteps: int, dt: float) -> None:
    _check(lib.assn_step(h, nsteps, dt), h)


def assn_set_scheme(h: int, scheme: int) -> None:
    _check(lib.assn_set_scheme(h, scheme), h)


def assn_set_implicit_params(h: int, si_eps: float = 1e-4, gmres_tol: float = 1.5e-8, restart: int = 30,
                             max_si: int = 1000, max_gmres: int = 500) -> None:
    _check(lib.assn_set_implicit_params(h, si_eps, gmres_tol, restart, max_si, max_gmres), h)


def assn_implicit_stats(h: int) -> dict:
    a, b, c = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    _check(lib.assn_implicit_stats(h, C.byref(a), C.byref(b), C.byref(c)), h)
    return {"source_iterations": a.value, "gmres_iterations": b.value, "sweeps": c.value}


def assn_implicit_source_iteration(h: int, dt: float, R, psi0, iterations: int) -> np.ndarray:
    r = _contig(R)
    p0 = _contig(psi0)
    out = np.empty_like(r)
    _check(lib.assn_implicit_source_iteration(h, dt, _d(r), _d(p0), iterations, _d(out)), h)
    return out


def assn_get_scheme(h: int) -> int:
    v = C.c_int(0)
    _check(lib.assn_get_scheme(h, C.byref(v)), h)
    return v.value


def assn_step_device(h: int, psi_in_dev: int, psi_out_dev: int, dt: float) -> None:
    _check(lib.assn_step_device(h, psi_in_dev, psi_out_dev, dt), h)


def assn_run_f32(h: int, psi0: np.ndarray, nsteps: int, dt: float, phi_out: np.ndarray) -> np.ndarray:
    assert psi0.dtype == np.float32 and psi0.flags.c_contiguous
    assert phi_out.dtype == np.float64 and phi_out.flags.c_contiguous
    _check(lib.assn_run_f32(h, psi0.ctypes.data_as(_fp), nsteps, dt, _d(phi_out)), h)
    return phi_out


def assn_set_tiling(h: int, tile_cells: int = 0, stages: int = 0, variant: int = 0) -> None:
    _check(lib.assn_set_tiling(h, tile_cells, stages, variant), h)


def assn_set_rings(h: int, staging: int = 0, operand: int = 0, kernel_matrix: int = 0,
                   blocks_per_request: int = 0) -> None:
    _check(lib.assn_set_rings(h, staging, operand, kernel_matrix, blocks_per_request), h)


def assn_get_rings(h: int) -> dict:
    v = [C.c_int(0) for _ in range(4)]
    _check(lib.assn_get_rings(h, *[C.byref(x) for x in v]), h)
    return dict(zip(("staging", "operand", "kernel_matrix", "blocks_per_request"), [x.value for x in v]))


def assn_get_tiling(h: int) -> dict:
    t, s, c, m = C.c_int(0), C.c_int(0), C.c_int(0), C.c_int64(0)
    _check(lib.assn_get_tiling(h, C.byref(t), C.byref(s), C.byref(c), C.byref(m)), h)
    return {"tile_cells": t.value, "stages": s.value, "tmem_cols": c.value, "smem_bytes": m.value}


def assn_get_variant(h: int) -> int:
    v = C.c_int(0)
    _check(lib.assn_get_variant(h, C.byref(v)), h)
    return v.value


def assn_layout(h: int):
    qp, eb = C.c_int(0), C.c_int(0)
    _check(lib.assn_layout(h, C.byref(qp), C.byref(eb)), h)
    return qp.value, eb.value


def assn_state_device(h: int) -> int:
    p = _vp()
    _check(lib.assn_state_device(h, C.byref(p)), h)
    return p.value


def assn_scalar_flux(h: int, shape) -> np.ndarray:
    out = np.empty(shape)
    _check(lib.assn_scalar_flux(h, _d(out)), h)
    return out


def assn_scalar_flux_device(h: int, phi_dev: int) -> None:
    _check(lib.assn_scalar_flux_device(h, phi_dev), h)


def assn_mass(h: int) -> float:
    v = C.c_double(0)
    _check(lib.assn_mass(h, C.byref(v)), h)
    return v.value


def assn_check_finite(h: int) -> None:
    _check(lib.assn_check_finite(h), h)


def assn_check_guards(h: int) -> dict:
    g, z = C.c_int64(0), C.c_int64(0)
    _check(lib.assn_check_guards(h, C.byref(g), C.byref(z)), h)
    return {"guard_bytes_changed": g.value, "padding_nonzero": z.value}


def assn_last_error(h: int | None) -> str:
    return lib.assn_last_error(h).decode()


def assn_status_string(status: int) -> str:
    return status_string(status)


def assn_launch_count(h: int) -> int:
    return int(lib.assn_launch_count(h))


def _bcheck(status: int, b=None):
    if status != ASSN_OK:
        raise AssnError(status, lib.assn_batch_last_error(b).decode())


def assn_batch_create(stream=None) -> int:
    b = _h()
    _bcheck(lib.assn_batch_create(C.byref(b), _stream_ptr(stream)), None)
    return b.value


def assn_batch_destroy(b: int) -> None:
    _bcheck(lib.assn_batch_destroy(b), b)


def assn_batch_add(b: int, p: int, nsteps: int, dt: float) -> None:
    _bcheck(lib.assn_batch_add(b, p, nsteps, dt), b)


def assn_batch_set_steps(b: int, p: int, nsteps: int, dt: float) -> None:
    _bcheck(lib.assn_batch_set_steps(b, p, nsteps, dt), b)


def assn_batch_remove(b: int, p: int) -> None:
    _bcheck(lib.assn_batch_remove(b, p), b)


def assn_batch_set_tiling(b: int, tile_cells: int = 0, stages: int = 0) -> None:
    _bcheck(lib.assn_batch_set_tiling(b, tile_cells, stages), b)


def assn_batch_set_grouping(b: int, one_launch: bool) -> None:
    _bcheck(lib.assn_batch_set_grouping(b, int(one_launch)), b)


def assn_batch_autotune(b: int, use_cache: bool = True) -> dict:
    t, s, ms = C.c_int(0), C.c_int(0), C.c_double(0)
    _bcheck(lib.assn_batch_autotune(b, int(use_cache), C.byref(t), C.byref(s), C.byref(ms)), b)
    return {"tile_cells": t.value, "stages": s.value, "ms_per_launch": ms.value}


def assn_batch_run(b: int, use_graph: bool = True) -> None:
    _bcheck(lib.assn_batch_run(b, int(use_graph)), b)


def assn_batch_sync(b: int) -> None:
    _bcheck(lib.assn_batch_sync(b), b)


def assn_batch_info(b: int) -> dict:
    m, t, s, n = C.c_int(0), C.c_int(0), C.c_int(0), C.c_int(0)
    L = C.c_int64(0)
    _bcheck(lib.assn_batch_info(b, C.byref(m), C.byref(t), C.byref(s), C.byref(n), C.byref(L)), b)
    return {"members": m.value, "tile_cells": t.value, "stages": s.value, "total_tiles": n.value,
            "launches": L.value}


def assn_batch_classes(b: int) -> list[dict]:
    n = C.c_int(0)
    _bcheck(lib.assn_batch_classes(b, C.byref(n)), b)
    out = []
    for k in range(n.value):
        v = [C.c_int(0) for _ in range(5)]
        _bcheck(lib.assn_batch_class_info(b, k, *[C.byref(x) for x in v]), b)
        out.append(dict(zip(("ordinate_stride", "members", "tile_cells", "stages", "tiles"), [x.value for x in v])))
    return out


def assn_batch_last_error(b: int | None) -> str:
    return lib.assn_batch_last_error(b).decode()


def assn_autotune(h: int, dt: float, use_cache: bool = True) -> dict:
    t, s, ms = C.c_int(0), C.c_int(0), C.c_double(0)
    _check(lib.assn_autotune(h, dt, int(use_cache), C.byref(t), C.byref(s), C.byref(ms)), h)
    return {"tile_cells": t.value, "stages": s.value, "ms_per_step": ms.value}


def _scheck(status: int):
    if status != ASSN_OK:
        raise AssnError(status, lib.assn_server_last_error().decode())


def assn_footprint_bytes(nx: int, ny: int, Q: int, precision: int) -> int:
    b = C.c_size_t(0)
    st = lib.assn_footprint_bytes(nx, ny, Q, precision, C.byref(b))
    if st != ASSN_OK:
        raise AssnError(st, "invalid sizes")
    return int(b.value)


def assn_server_create(precision: int, hbm_budget_bytes: int = 0, max_active: int = 64, chunk_steps: int = 8,
                       use_graph: bool = True) -> int:
    s = _h()
    _scheck(lib.assn_server_create(C.byref(s), precision, hbm_budget_bytes, max_active, chunk_steps, int(use_graph)))
    return s.value


def assn_server_submit(s: int, req: AssnRequest) -> int:
    rid = C.c_int64(0)
    _scheck(lib.assn_server_submit(s, C.byref(req), C.byref(rid)))
    return int(rid.value)


def assn_server_wait(s: int, rid: int, timeout_s: float, phi_out: np.ndarray | None):
    lat, qs = C.c_double(0), C.c_double(0)
    ptr = None
    if phi_out is not None:
        assert phi_out.dtype == np.float64 and phi_out.flags.c_contiguous
        ptr = _d(phi_out)
    _scheck(lib.assn_server_wait(s, rid, timeout_s, ptr, C.byref(lat), C.byref(qs)))
    return lat.value, qs.value


def assn_server_get_stats(s: int) -> dict:
    st = AssnServerStats()
    _scheck(lib.assn_server_get_stats(s, C.byref(st)))
    return {name: getattr(st, name) for name, _ in AssnServerStats._fields_}


def assn_server_destroy(s: int) -> None:
    _scheck(lib.assn_server_destroy(s))


def assn_server_cancel(s: int, rid: int) -> None:
    _scheck(lib.assn_server_cancel(s, rid))


def assn_server_last_error() -> str:
    return lib.assn_server_last_error().decode()


def assn_mass_noalloc(psi_dev: int, elem_bytes: int, w_dev: int, ncell: int, Qp: int, h: float, mass_dev: int,
                      stream=None) -> None:
    """Allocation-free total mass of a device state (see include/assn.h); result written to mass_dev."""
    st = lib.assn_mass_noalloc(psi_dev, elem_bytes, w_dev, ncell, Qp, h, mass_dev, _stream_ptr(stream))
    if st != ASSN_OK:
        raise AssnError(st, lib.assn_noalloc_last_error().decode())


def assn_noalloc_last_error() -> str:
    return lib.assn_noalloc_last_error().decode()


def assn_abi_version() -> int:
    return int(lib.assn_abi_version())


def assn_selftest_wait_timeout(limit_us: int) -> int:
    """Status of the bounded-wait self-test (ASSN_ERR_TIMEOUT when the failure path works)."""
    return int(lib.assn_selftest_wait_timeout(limit_us))

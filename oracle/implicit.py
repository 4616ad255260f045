"""FP64 reference of the paper's implicit as-S_N time step (Sec. 3.4 and 3.5; test infrastructure only).

Implicit Euler in time.  In space, the second-order upwind stencil without limiter of Sec. 3.5: along
an axis with velocity component Omega and lambda = |Omega| dt / h, the flux difference of cell j is
(3/2) psi_j - 2 psi_{j-1} + (1/2) psi_{j-2} with j-1, j-2 the upwind neighbours; in two dimensions the
x and y stencils add.  Vacuum boundaries: the upwind ghost cells are zero.

With sigma_t = sigma_a + sigma_s + sigma_as + 1/dt the discrete streaming operator times dt is
    (L psi)_c = lx ((3/2) psi_c - 2 psi_{c-x} + (1/2) psi_{c-2x}) + ly (...) + dt sigma_t(c) psi_c,
and one implicit step solves, for psi = psi^{n+1},
    L psi = dt (sigma_s Phi / sum w + sigma_as K psi + q + psi^n / dt).
The paper's solver (Alg. 1-3): the source iteration inverts L - dt sigma_as K by sweeps, GMRES acts
on the scalar flux (the one moment of isotropic physical scattering).

Conventions as in assn_oracle: psi float64 [ny][nx][Q], cell fields [ny][nx].
"""
from __future__ import annotations

import math

import numpy as np

from .assn_oracle import scalar_flux

__all__ = ["streaming_apply", "sweep", "source_iteration", "source_iteration_lipschitz", "gmres",
           "implicit_step", "implicit_run", "implicit_step_direct"]


def _speeds(Omega, h: float, dt: float):
    Om = np.asarray(Omega, dtype=np.float64)
    return np.abs(Om[:, 0]) * dt / h, np.abs(Om[:, 1]) * dt / h, np.sign(Om[:, 0]), np.sign(Om[:, 1])


def _upwind(psi, sign, axis: int, k: int):
    """psi at the k-th upwind neighbour along axis (per ordinate: upwind is -1 for sign > 0, +1 for
    sign < 0); zero outside the grid (vacuum)."""
    out = np.zeros_like(psi)
    n = psi.shape[axis]
    if k >= n:
        return out
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    pos, neg = sign > 0, sign < 0
    # sign > 0: out[j] = psi[j - k]
    lo[axis] = slice(k, n)
    hi[axis] = slice(0, n - k)
    out[tuple(lo)][..., pos] = psi[tuple(hi)][..., pos]
    # sign < 0: out[j] = psi[j + k]
    lo[axis] = slice(0, n - k)
    hi[axis] = slice(k, n)
    out[tuple(lo)][..., neg] = psi[tuple(hi)][..., neg]
    return out


def streaming_apply(psi, Omega, h: float, dt: float, sigma_tot):
    """L psi: dt times the discrete streaming operator of Sec. 3.5 in 2D (see the module header);
    sigma_tot [ny][nx] = sigma_a + sigma_s + sigma_as (the 1/dt part is the added psi)."""
    psi = np.asarray(psi, dtype=np.float64)
    lx, ly, sx, sy = _speeds(Omega, h, dt)
    tx = 1.5 * psi - 2.0 * _upwind(psi, sx, 1, 1) + 0.5 * _upwind(psi, sx, 1, 2)
    ty = 1.5 * psi - 2.0 * _upwind(psi, sy, 0, 1) + 0.5 * _upwind(psi, sy, 0, 2)
    return lx * tx + ly * ty + (1.0 + dt * np.asarray(sigma_tot)[..., None]) * psi


def sweep(R, Omega, h: float, dt: float, sigma_tot):
    """Solve L psi = R (Sec. 3.5: the inverse of the streaming operator by sweeping).  Each cell
    depends on its first and second upwind neighbours in x and y only, so the cells are solved
    anti-diagonal by anti-diagonal in the upwind order of each ordinate's quadrant; the cells of one
    anti-diagonal are independent and are solved together."""
    R = np.asarray(R, dtype=np.float64)
    ny, nx, Q = R.shape
    lx, ly, sx, sy = _speeds(Omega, h, dt)
    st = 1.0 + dt * np.asarray(sigma_tot, dtype=np.float64)
    psi = np.zeros_like(R)
    for qx in (1.0, -1.0):
        for qy in (1.0, -1.0):
            # ordinates of this quadrant (a zero component sweeps as positive: it has no flux)
            sel = np.where(((sx >= 0) if qx > 0 else (sx < 0)) & ((sy >= 0) if qy > 0 else (sy < 0)))[0]
            if sel.size == 0:
                continue
            ax, ay = lx[sel], ly[sel]
            # work in the upwind-ordered frame: index a = i or nx-1-i, b = j or ny-1-j
            Rq = R[:, :, sel]
            if qx < 0:
                Rq = Rq[:, ::-1]
            if qy < 0:
                Rq = Rq[::-1]
            stq = st[:, ::-1] if qx < 0 else st
            stq = stq[::-1] if qy < 0 else stq
            P = np.zeros((ny + 2, nx + 2, sel.size))     # two zero ghost rows / columns before the grid
            diag = 1.5 * (ax + ay)
            for d in range(nx + ny - 1):
                b = np.arange(max(0, d - (nx - 1)), min(d, ny - 1) + 1)
                a = d - b
                num = (Rq[b, a] + ax * (2.0 * P[b + 2, a + 1] - 0.5 * P[b + 2, a])
                       + ay * (2.0 * P[b + 1, a + 2] - 0.5 * P[b, a + 2]))
                P[b + 2, a + 2] = num / (diag + stq[b, a][:, None])
            out = P[2:, 2:]
            if qy < 0:
                out = out[::-1]
            if qx < 0:
                out = out[:, ::-1]
            psi[:, :, sel] = out
    return psi


def source_iteration_lipschitz(sigma_a, sigma_s, sigma_as: float, dt: float) -> float:
    """The estimate T of the source iteration's contraction factor (Alg. 1): the artificial gain over
    the removal rate of a cell, dt sigma_as / (1 + dt (sigma_a + sigma_s + sigma_as)), at its largest."""
    tot = np.asarray(sigma_a) + np.asarray(sigma_s)
    return float(np.max(dt * sigma_as / (1.0 + dt * (tot + sigma_as))))


def source_iteration(psi0, R, K, Omega, sigma_tot, sigma_as: float, h: float, dt: float,
                     eps: float, T: float, max_iter: int = 1000, fixed: int | None = None):
    """Alg. 1: solve (L - dt sigma_as K) psi = dt R by psi^{l+1} = L^{-1} dt (sigma_as K psi^l + R),
    starting from psi0, until ||psi^{l+1} - psi^l||_2 < eps (1 - T) / T (an a-posteriori error
    estimate eps for a contraction with factor T), or exactly `fixed` iterations.
    Returns (psi, iterations)."""
    Kt = np.asarray(K, dtype=np.float64).T
    R = np.asarray(R, dtype=np.float64)
    tol = eps * (1.0 - T) / T if T > 0 else 0.0
    psi = np.asarray(psi0, dtype=np.float64)
    it = 0
    while True:
        new = sweep(dt * (sigma_as * (psi @ Kt) + R), Omega, h, dt, sigma_tot)
        it += 1
        diff = float(np.linalg.norm(new - psi))
        psi = new
        if fixed is not None:
            if it >= fixed:
                break
        elif diff < tol or it >= max_iter or T == 0.0:
            break
    return psi, it


def gmres(apply_A, b, x0, tol: float, restart: int = 30, max_iter: int = 500):
    """Restarted GMRES (Saad and Schultz, 1986) with modified Gram-Schmidt Arnoldi: x with
    ||b - A x|| <= tol ||b||, starting from x0.  Returns (x, iterations)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    x = np.asarray(x0, dtype=np.float64).ravel().copy()
    nb = float(np.linalg.norm(b))
    if nb == 0.0:
        return np.zeros_like(b), 0
    total = 0
    while total < max_iter:
        r = b - apply_A(x)
        beta = float(np.linalg.norm(r))
        if beta <= tol * nb:
            break
        V = [r / beta]
        H = np.zeros((restart + 1, restart))
        k_done = 0
        for k in range(restart):
            wv = apply_A(V[k])
            for i in range(k + 1):
                H[i, k] = float(V[i] @ wv)
                wv = wv - H[i, k] * V[i]
            H[k + 1, k] = float(np.linalg.norm(wv))
            k_done = k + 1
            total += 1
            e1 = np.zeros(k + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)
            res = float(np.linalg.norm(e1 - H[:k + 2, :k + 1] @ y))
            if res <= tol * nb or H[k + 1, k] == 0.0 or total >= max_iter:
                break
            V.append(wv / H[k + 1, k])
        x = x + np.column_stack(V[:k_done]) @ y
    return x, total


def implicit_step(psi_old, phi_old, K, Omega, w, sigma_a, sigma_s, q, sigma_as: float, h: float, dt: float,
                  si_eps: float, gmres_tol: float, restart: int = 30):
    """One step of Alg. 3 (sweeping-Krylov): returns (psi_new, phi_new, source iterations, GMRES
    iterations).  The right-hand side of the last source iteration carries the source q with
    psi_old/dt and the scattering of the new scalar flux (the full right-hand side of the step)."""
    w = np.asarray(w, dtype=np.float64)
    sa = np.asarray(sigma_a, dtype=np.float64)
    ss = np.asarray(sigma_s, dtype=np.float64)
    src = np.asarray(q, dtype=np.float64)
    sig = sa + ss + sigma_as
    T = source_iteration_lipschitz(sa, ss, sigma_as, dt)
    wsum = float(w.sum())
    shape = sa.shape
    si_total = 0

    def SI(R):
        nonlocal si_total
        psi, it = source_iteration(psi_old, R, K, Omega, sig, sigma_as, h, dt, si_eps, T)
        si_total += it
        return psi

    def scatter(phi):                       # sigma_s O Sigma phi: isotropic, phi / sum w to every ordinate
        return (ss * phi.reshape(shape) / wsum)[..., None] * np.ones(len(w))

    base = src[..., None] + psi_old / dt
    b = scalar_flux(SI(base), w).ravel()
    phi, its = gmres(lambda f: f - scalar_flux(SI(scatter(f)), w).ravel(), b, np.asarray(phi_old).ravel(),
                     gmres_tol, restart)
    psi_new = SI(scatter(phi) + base)
    return psi_new, phi.reshape(shape), si_total, its


def implicit_run(psi0, nsteps: int, K, Omega, w, sigma_a, sigma_s, q, sigma_as: float, h: float, dt: float,
                 si_eps: float, gmres_tol: float, restart: int = 30):
    """nsteps of Alg. 3 from psi0 (phi_old starts as the scalar flux of psi0)."""
    psi = np.asarray(psi0, dtype=np.float64)
    phi = scalar_flux(psi, w)
    for _ in range(nsteps):
        psi, phi, _, _ = implicit_step(psi, phi, K, Omega, w, sigma_a, sigma_s, q, sigma_as, h, dt,
                                       si_eps, gmres_tol, restart)
    return psi


def implicit_step_direct(psi_old, K, Omega, w, sigma_a, sigma_s, q, sigma_as: float, h: float, dt: float):
    """The implicit step as one linear system over all cells and ordinates, assembled column by column
    from streaming_apply and solved directly (small grids only):
        L psi - dt (sigma_s Phi / sum w + sigma_as K psi) = dt q + psi_old."""
    psi_old = np.asarray(psi_old, dtype=np.float64)
    ny, nx, Q = psi_old.shape
    w = np.asarray(w, dtype=np.float64)
    sa = np.asarray(sigma_a, dtype=np.float64)
    ss = np.asarray(sigma_s, dtype=np.float64)
    sig = sa + ss + sigma_as
    n = ny * nx * Q
    if n > 3000:
        raise ValueError("implicit_step_direct assembles a dense matrix: small grids only")
    Kt = np.asarray(K, dtype=np.float64).T

    def op(v):
        p = v.reshape(ny, nx, Q)
        phi = scalar_flux(p, w)
        gain = (ss * phi / w.sum())[..., None] + sigma_as * (p @ Kt)
        return (streaming_apply(p, Omega, h, dt, sig) - dt * gain).ravel()

    A = np.column_stack([op(e) for e in np.eye(n)])
    rhs = (dt * np.asarray(q, dtype=np.float64)[..., None] + psi_old).ravel()
    return np.linalg.solve(A, rhs).reshape(ny, nx, Q)

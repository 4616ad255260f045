"""FP64 reference of the explicit as-S_N step (test infrastructure only; see the package header).

Every function follows one passage of Camminady, Frank, Hauck, Kusch,
"Ray Effect Mitigation for the Discrete Ordinates Method Using Artificial
Scattering" (arXiv:1911.08801), cited in its docstring.  No blocking, fusion
or reordering: the step evaluates every term of the as-S_N equations at the
old time level (unsplit forward Euler), applies the dense Q x Q artificial
scattering matrix as one product, and uses first-order upwind fluxes with
zero inflow (vacuum) ghost cells.

Conventions: ``psi`` is float64 ``[ny][nx][Q]``; cell fields are ``[ny][nx]``;
``Omega`` is ``[Q][3]`` unit vectors, ``w`` is ``[Q]`` with sum 4 pi.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "product_quadrature", "s_eps", "s_exp", "kernel_matrix", "scalar_flux",
    "transport", "step", "run", "mass", "step_at_cells",
    "minmod", "transport_minmod", "rhs", "step_heun", "run_heun",
    "icosahedron_quadrature", "heun_admissible_dt",
]


# --------------------------------------------------------------------------- S0
def product_quadrature(n_polar: int, n_azim: int):
    """Product quadrature on S^2: Gauss-Legendre in mu times uniform azimuth.

    Sec. 3.1 (quadrature rule with weights w_q, sum of weights 4 pi) and
    Sec. 4 (ordinates projected onto the x-y plane for 2D transport).
    Ordinate q = k * n_polar + i (azimuth-major; the numbering of the set
    is a convention the method does not fix) has mu = mu_i (i-th Gauss-Legendre node),
    azimuth phi_k = (k + 1/2) 2 pi / n_azim, direction
    (sqrt(1-mu^2) cos phi, sqrt(1-mu^2) sin phi, mu) and weight
    w_i^GL * 2 pi / n_azim.  Returns (Omega[Q,3], w[Q]).
    """
    mu, wgl = np.polynomial.legendre.leggauss(n_polar)
    phi = (np.arange(n_azim) + 0.5) * (2.0 * math.pi / n_azim)
    Q = n_polar * n_azim
    Omega = np.empty((Q, 3))
    w = np.empty(Q)
    for i in range(n_polar):
        st = math.sqrt(max(0.0, 1.0 - mu[i] * mu[i]))
        for k in range(n_azim):
            q = k * n_polar + i
            Omega[q] = (st * math.cos(phi[k]), st * math.sin(phi[k]), mu[i])
            w[q] = wgl[i] * 2.0 * math.pi / n_azim
    return Omega, w



def _sphere_triangle_area(a, b, c) -> float:
    """Area of the spherical triangle with unit-vector corners a, b, c (the tangent half-angle
    formula of Van Oosterom and Strackee, 1983)."""
    num = abs(float(np.dot(a, np.cross(b, c))))
    den = 1.0 + float(np.dot(a, b) + np.dot(b, c) + np.dot(c, a))
    return 2.0 * math.atan2(num, den)


def icosahedron_quadrature(order: int, base: str = "printed", midpoints: str = "sphere"):
    """Icosahedron quadrature on S^2 (Sec. 3.3; the paper prints order 2 in Appendix A).

    The construction the paper describes: every face of an icosahedron is triangulated with
    equally spaced points on its edges and the matching interior points (order k: k - 1 segments
    per edge, so N_q = 10 (k-1)^2 + 2), the points are mapped onto the unit sphere, and a point's
    weight is the area of the cell around it whose corners are the midpoints of the neighbouring
    triangles (and of the edges between them): the barycentric dual cell.  One vertex sits at
    (0, 0, 1).

    Readings (the paper's text and its printed table disagree on the base solid):
      * base "printed": the twelve base vertices are (0, +-1, +-g), (+-1, +-g, 0) and
        (+-1, 0, +-g), g the golden ratio, joined into the 20 faces of the regular icosahedron
        below, each (+-1, 0, +-g) in the place of the regular (+-g, 0, +-1) with the same signs;
        with this base the construction reproduces the printed order-2 points and weights.
        base "regular": the regular icosahedron, (+-g, 0, +-1) in the last group.
      * Both are turned about the x axis so that (0, 1, g) lands on (0, 0, 1).
      * midpoints "sphere": the centre of a triangle with mapped corners a, b, c is
        (a + b + c) / |a + b + c|, the midpoint of an edge (a + b) / |a + b|; midpoints "flat": the
        cell is drawn on the flat face and then mapped, so the centre and midpoints are those of the
        flat points, mapped (the two agree at order 2).  Cell boundaries are great-circle arcs.

    Returns (Omega[N_q, 3], w[N_q]); the order of the points is not significant.
    """
    if order < 2:
        raise ValueError("order >= 2")
    g = (1.0 + math.sqrt(5.0)) / 2.0
    regular, used = [], []
    for s1 in (1.0, -1.0):
        for s2 in (1.0, -1.0):
            regular += [(0.0, s1, s2 * g), (s1, s2 * g, 0.0), (s1 * g, 0.0, s2)]
            used += [(0.0, s1, s2 * g), (s1, s2 * g, 0.0),
                     (s1, 0.0, s2 * g) if base == "printed" else (s1 * g, 0.0, s2)]
    if base not in ("printed", "regular"):
        raise ValueError("base is 'printed' or 'regular'")
    R = np.array(regular)
    V = np.array(used)
    # faces of the regular icosahedron: triples of vertices that are pairwise one edge (2) apart
    near = np.abs(np.linalg.norm(R[:, None, :] - R[None, :, :], axis=2) - 2.0) < 1e-9
    faces = [(i, j, k) for i in range(12) for j in range(i + 1, 12) for k in range(j + 1, 12)
             if near[i, j] and near[j, k] and near[i, k]]
    assert len(faces) == 20
    # turn about x: (0, 1, g) -> (0, 0, 1)
    ang = math.atan2(1.0, g)
    rot = np.array([[1.0, 0.0, 0.0],
                    [0.0, math.cos(ang), -math.sin(ang)],
                    [0.0, math.sin(ang), math.cos(ang)]])
    V = V @ rot.T
    if midpoints not in ("sphere", "flat"):
        raise ValueError("midpoints is 'sphere' or 'flat'")
    n = order - 1
    index, points, flat = {}, [], []

    def node(f, i, j):
        # the point with i / n of the way to the face's second vertex and j / n to its third;
        # keyed by its barycentric counts so that points on shared edges and vertices coincide
        a, b, c = faces[f]
        key = tuple(sorted((v, m) for v, m in ((a, n - i - j), (b, i), (c, j)) if m > 0))
        if key not in index:
            p = V[a] + (i / n) * (V[b] - V[a]) + (j / n) * (V[c] - V[a])
            index[key] = len(points)
            points.append(p / np.linalg.norm(p))
            flat.append(p)
        return index[key]

    triangles = []
    for f in range(20):
        for i in range(n):
            for j in range(n - i):
                triangles.append((node(f, i, j), node(f, i + 1, j), node(f, i, j + 1)))
                if i + j + 2 <= n:
                    triangles.append((node(f, i + 1, j), node(f, i + 1, j + 1), node(f, i, j + 1)))
    Omega = np.array(points)
    w = np.zeros(len(points))
    unit = lambda x: x / np.linalg.norm(x)
    M = Omega if midpoints == "sphere" else np.array(flat)     # the points midpoints are taken from
    for t in triangles:
        P = [M[v] for v in t]
        centre = unit(P[0] + P[1] + P[2])
        for k in range(3):
            a, b, c = P[k], P[(k + 1) % 3], P[(k + 2) % 3]
            node_k = Omega[t[k]]
            w[t[k]] += (_sphere_triangle_area(node_k, unit(a + b), centre)
                        + _sphere_triangle_area(node_k, centre, unit(a + c)))
    return Omega, w

# --------------------------------------------------------------------------- S1
def s_eps(mu, eps: float):
    """Artificial scattering kernel, Sec. 2.3, Eq. (scattering kernel):
    s_eps(mu) = 2 / (sqrt(pi) eps Erf(2/eps)) * exp(-(1-mu)^2 / eps^2)."""
    mu = np.asarray(mu, dtype=np.float64)
    return 2.0 / (math.sqrt(math.pi) * eps * math.erf(2.0 / eps)) * np.exp(-((1.0 - mu) ** 2) / eps ** 2)


def s_exp(mu, eps: float):
    """Alternative forward-peaked kernel exp((mu - 1)/eps^2), normalised to unit integral on [-1, 1]
    (a Dirac sequence in the sense of Sec. 2.3 as eps -> 0)."""
    mu = np.asarray(mu, dtype=np.float64)
    e2 = eps * eps
    return np.exp((mu - 1.0) / e2) / (e2 * -math.expm1(-2.0 / e2))


def kernel_matrix(Omega, w, eps: float, kind: str = "gauss", normalisation: str = "column"):
    """Discrete artificial in-scattering matrix K (Sec. 3.2, Eq. (as-S_N equations)).

    s_qp = s_eps(Omega_q . Omega_p).  The paper's gain term is
    sum_p w_p c_q s_qp psi_p with c_q = 1 / sum_p w_p s_qp ("row": every row
    of K sums to one).  The default "column" form normalises by the source
    ordinate instead, K_qp = w_p c_p s_qp, so that sum_q w_q K_qp = w_p and the
    operator conserves sum_q w_q psi_q exactly (Sec. 2.3: artificial
    scattering preserves the number of particles).
    """
    Omega = np.asarray(Omega, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    mu = np.clip(Omega @ Omega.T, -1.0, 1.0)
    s = s_eps(mu, eps) if kind == "gauss" else s_exp(mu, eps)
    if normalisation == "column":
        c = 1.0 / (w @ s)                    # c_p = 1 / sum_q w_q s_qp
        return s * (w * c)[None, :]
    if normalisation == "row":
        c = 1.0 / (s @ w)                    # c_q = 1 / sum_p w_p s_qp
        return s * w[None, :] * c[:, None]
    raise ValueError(normalisation)


# --------------------------------------------------------------------------- S3
def scalar_flux(psi, w):
    """Phi = sum_q w_q psi_q (Sec. 2.2 definition of Phi, discretised with the rule of Sec. 3.1)."""
    return np.asarray(psi, dtype=np.float64) @ np.asarray(w, dtype=np.float64)


# --------------------------------------------------------------------------- S4
def transport(psi, Omega, h: float, bc: str = "vacuum"):
    """First-order upwind finite-volume approximation of Omega . grad psi (Sec. 3.1, Eq. (S_N)).

    For Omega_x > 0: Omega_x (psi_i - psi_{i-1}) / h; for Omega_x < 0:
    Omega_x (psi_{i+1} - psi_i) / h; nothing for Omega_x = 0; likewise in y.
    Vacuum boundaries (Sec. 4.2) supply zero incoming ghost values;
    "periodic" wraps around (used by tests only).
    """
    psi = np.asarray(psi, dtype=np.float64)
    ox = np.asarray(Omega)[:, 0]
    oy = np.asarray(Omega)[:, 1]
    if bc == "periodic":
        left, right = np.roll(psi, 1, axis=1), np.roll(psi, -1, axis=1)
        down, up = np.roll(psi, 1, axis=0), np.roll(psi, -1, axis=0)
    else:
        z = np.zeros_like(psi[:, :1, :])
        left = np.concatenate([z, psi[:, :-1, :]], axis=1)
        right = np.concatenate([psi[:, 1:, :], z], axis=1)
        zy = np.zeros_like(psi[:1, :, :])
        down = np.concatenate([zy, psi[:-1, :, :]], axis=0)
        up = np.concatenate([psi[1:, :, :], zy], axis=0)
    tx = np.where(ox > 0, ox * (psi - left), np.where(ox < 0, ox * (right - psi), 0.0))
    ty = np.where(oy > 0, oy * (psi - down), np.where(oy < 0, oy * (up - psi), 0.0))
    return (tx + ty) / h


# --------------------------------------------------------------------------- S2 + S5
def step(psi, K, Omega, w, sigma_a, sigma_s, q, sigma_as: float, h: float, dt: float,
         bc: str = "vacuum"):
    """One explicit Euler step of the as-S_N equations (Sec. 3.2, Eq. (as-S_N equations)).

    psi^{n+1}_q = psi_q - dt [Omega_q . grad psi_q]_upwind
                  - dt (sigma_a + sigma_s + sigma_as) psi_q
                  + dt sigma_s sum_p w_p c s psi_p        (isotropic s = 1/(4 pi), c = 1/sum_p w_p s)
                  + dt sigma_as sum_p K_qp psi_p          (artificial in-scattering, Eq. (S_as^+))
                  + dt q
    Every term at time level n.  sigma_a, sigma_s, q are per-cell [ny][nx];
    sigma_as is a constant (Sec. 5: constant artificial scattering strength).
    """
    psi = np.asarray(psi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    sa = np.asarray(sigma_a, dtype=np.float64)[..., None]
    ss = np.asarray(sigma_s, dtype=np.float64)[..., None]
    src = np.asarray(q, dtype=np.float64)[..., None]
    s_iso = 1.0 / (4.0 * math.pi)
    c_iso = 1.0 / (w.sum() * s_iso)
    phys = (scalar_flux(psi, w) * c_iso * s_iso)[..., None]      # sum_p w_p c s psi_p
    art = psi @ np.asarray(K, dtype=np.float64).T                 # sum_p K_qp psi_p
    T = transport(psi, Omega, h, bc)
    return psi - dt * T - dt * (sa + ss + sigma_as) * psi + dt * (ss * phys + sigma_as * art + src)


# --------------------------------------------------------------------------- the paper's explicit scheme
# Sec. 3.1 names it only: Heun's method in time with a minmod slope limiter in space.  Read here as
# the usual second-order MUSCL finite-volume scheme: per axis, slopes Delta_i = minmod(psi_i -
# psi_{i-1}, psi_{i+1} - psi_i), upwind face values psi_i + Delta_i/2 (Omega > 0) or
# psi_{i+1} - Delta_{i+1}/2 (Omega < 0), and Heun (the two-stage strong-stability-preserving
# Runge-Kutta method) in time.


def minmod(a, b):
    """0 where a and b differ in sign (or either is 0), else the one of smaller magnitude."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.where(a * b > 0.0, np.where(np.abs(a) < np.abs(b), a, b), 0.0)


def _axis_flux_divergence(psi, om, h: float, axis: int, bc: str):
    """d/dx_axis of om * psi by limited upwind fluxes; psi [ny][nx][Q], om [Q]."""
    n = psi.shape[axis]
    if bc == "periodic":
        ext = np.concatenate([np.take(psi, [n - 2, n - 1], axis=axis, mode="wrap"), psi,
                              np.take(psi, [0, 1], axis=axis, mode="wrap")], axis=axis)
    else:   # vacuum: two zero ghost cells on each side
        shape = list(psi.shape)
        shape[axis] = 2
        z = np.zeros(shape)
        ext = np.concatenate([z, psi, z], axis=axis)
    # ext index e = i + 2; slopes of cells i = -1 .. n (e = 1 .. n + 2)
    def sl(lo, hi):
        return np.take(ext, range(lo, hi), axis=axis)
    d = minmod(sl(1, n + 3) - sl(0, n + 2), sl(2, n + 4) - sl(1, n + 3))      # cells -1 .. n
    cell = sl(1, n + 3)                                                          # psi of cells -1 .. n
    left_state = cell + 0.5 * d          # face value on the left side of face (i + 1/2), i = -1 .. n
    right_state = cell - 0.5 * d         # face value on the right side of face (i - 1/2), i = -1 .. n
    # faces f = i + 1/2 for i = -1 .. n - 1: upwind side is cell i for om > 0, cell i + 1 for om < 0
    fl = np.take(left_state, range(0, n + 1), axis=axis)
    fr = np.take(right_state, range(1, n + 2), axis=axis)
    flux = np.where(om > 0, om * fl, np.where(om < 0, om * fr, 0.0))           # n + 1 faces
    return (np.take(flux, range(1, n + 1), axis=axis) - np.take(flux, range(0, n), axis=axis)) / h


def transport_minmod(psi, Omega, h: float, bc: str = "vacuum"):
    """Omega . grad psi by second-order upwind fluxes with minmod-limited slopes (Sec. 3.1).
    Vacuum boundaries: zero inflow ghost cells (two per side); "periodic" for tests."""
    psi = np.asarray(psi, dtype=np.float64)
    ox = np.asarray(Omega)[:, 0]
    oy = np.asarray(Omega)[:, 1]
    return _axis_flux_divergence(psi, ox, h, 1, bc) + _axis_flux_divergence(psi, oy, h, 0, bc)


def rhs(psi, K, Omega, w, sigma_a, sigma_s, q, sigma_as: float, h: float, bc: str = "vacuum",
        second_order: bool = True):
    """Right-hand side of the as-S_N equations (Sec. 3.2) for a time integrator:
    -[Omega . grad psi] - (sigma_a + sigma_s + sigma_as) psi + sigma_s Phi/sum w + sigma_as K psi + q."""
    psi = np.asarray(psi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    sa = np.asarray(sigma_a, dtype=np.float64)[..., None]
    ss = np.asarray(sigma_s, dtype=np.float64)[..., None]
    src = np.asarray(q, dtype=np.float64)[..., None]
    phys = (scalar_flux(psi, w) / w.sum())[..., None]
    art = psi @ np.asarray(K, dtype=np.float64).T
    T = transport_minmod(psi, Omega, h, bc) if second_order else transport(psi, Omega, h, bc)
    return -T - (sa + ss + sigma_as) * psi + ss * phys + sigma_as * art + src


def step_heun(psi, K, Omega, w, sigma_a, sigma_s, q, sigma_as: float, h: float, dt: float,
              bc: str = "vacuum"):
    """One step of Heun's method (Sec. 3.1): psi* = psi + dt L(psi),
    psi^{n+1} = psi/2 + (psi* + dt L(psi*))/2, with the limited second-order transport."""
    psi = np.asarray(psi, dtype=np.float64)
    args = (K, Omega, w, sigma_a, sigma_s, q, sigma_as, h, bc)
    star = psi + dt * rhs(psi, *args)
    return 0.5 * psi + 0.5 * (star + dt * rhs(star, *args))


def run_heun(psi0, nsteps: int, K, Omega, w, sigma_a, sigma_s, q, sigma_as: float, h: float,
             dt: float, bc: str = "vacuum"):
    psi = np.array(psi0, dtype=np.float64, copy=True)
    for _ in range(nsteps):
        psi = step_heun(psi, K, Omega, w, sigma_a, sigma_s, q, sigma_as, h, dt, bc)
    return psi


def heun_admissible_dt(Omega, K, sigma_a, sigma_s, sigma_as: float, h: float) -> float:
    """Largest dt for which every forward-Euler stage of the limited scheme (Sec. 3.1) is a
    non-negative combination of old values, so that Heun's method, an average of such stages,
    keeps psi >= 0 and bounded.

    With minmod slopes the upwind flux difference along an axis is (psi_i - psi_{i-1}) C with
    C = 1 + (D_i - D_{i-1}) / (2 (psi_i - psi_{i-1})) in [1/2, 3/2], so a stage multiplies psi_q by
    1 - (dt/h) sum_axes |Omega| C - dt (sigma_a + sigma_s) - dt sigma_as (1 - K_qq) and adds non-negative
    multiples of other values.  It stays >= 0 when
        dt (max_q [ 3/2 (|Omega_x,q| + |Omega_y,q|) / h + sigma_as (1 - K_qq) ] + max_cells [sigma_a + sigma_s]) <= 1.
    """
    Om = np.asarray(Omega, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    v = 1.5 * (np.abs(Om[:, 0]) + np.abs(Om[:, 1])) / h + sigma_as * (1.0 - np.diag(K))
    rate = v.max() + float(np.max(np.asarray(sigma_a) + np.asarray(sigma_s)))
    return 1.0 / rate if rate > 0 else math.inf


def run(psi0, nsteps: int, K, Omega, w, sigma_a, sigma_s, q, sigma_as: float, h: float,
        dt: float, bc: str = "vacuum"):
    """nsteps explicit steps from psi0 (Sec. 3.1 time discretisation, first order)."""
    psi = np.array(psi0, dtype=np.float64, copy=True)
    for _ in range(nsteps):
        psi = step(psi, K, Omega, w, sigma_a, sigma_s, q, sigma_as, h, dt, bc)
    return psi


def mass(psi, w, h: float) -> float:
    """Total particle number h^2 sum_cells sum_q w_q psi_q."""
    return float(h * h * scalar_flux(psi, w).sum())


def step_at_cells(psi, cells, K, Omega, w, sigma_a, sigma_s, q, sigma_as: float, h: float,
                  dt: float):
    """The same update as ``step`` (vacuum boundaries), evaluated one cell at a time.

    ``cells`` is a sequence of (j, i) = (y index, x index).  Returns
    float64 [len(cells)][Q].  Lets a test check sampled outputs of a launch
    too large to step whole on the host.
    """
    psi = np.asarray(psi)
    ny, nx, Q = psi.shape
    w = np.asarray(w, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    ox = np.asarray(Omega)[:, 0]
    oy = np.asarray(Omega)[:, 1]
    s_iso = 1.0 / (4.0 * math.pi)
    c_iso = 1.0 / (w.sum() * s_iso)
    out = np.empty((len(cells), Q))
    zero = np.zeros(Q)

    def at(j, i):
        if 0 <= j < ny and 0 <= i < nx:
            return np.asarray(psi[j, i], dtype=np.float64)
        return zero

    for n, (j, i) in enumerate(cells):
        p = at(j, i)
        tx = np.where(ox > 0, ox * (p - at(j, i - 1)), np.where(ox < 0, ox * (at(j, i + 1) - p), 0.0))
        ty = np.where(oy > 0, oy * (p - at(j - 1, i)), np.where(oy < 0, oy * (at(j + 1, i) - p), 0.0))
        T = (tx + ty) / h
        phys = float(w @ p) * c_iso * s_iso
        art = K @ p
        sa, ss, src = float(sigma_a[j, i]), float(sigma_s[j, i]), float(q[j, i])
        out[n] = p - dt * T - dt * (sa + ss + sigma_as) * p + dt * (ss * phys + sigma_as * art + src)
    return out

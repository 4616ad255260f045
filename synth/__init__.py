"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds problem set-up only: the test problems' initial data and
material maps (Section 4 of the paper: the line source and the lattice), the
workload parameter sets, and seeded random states.  It holds none of the
as-S_N method's arithmetic: no quadrature, no scattering kernel, no transport
and no time step.  Neither the oracle nor the CUDA path is imported here.

Array convention everywhere: a cell field is ``[ny][nx]`` (row = y index,
column = x index), an angular flux is ``[ny][nx][Q]``; cell (i, j) has centre
``(x0 + (i + 1/2) h, y0 + (j + 1/2) h)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FOUR_PI = 4.0 * math.pi


def eps_from_beta(beta: float, Q: int) -> float:
    """Kernel width eps = beta * h_Q, h_Q = sqrt(4 pi / Q) the mean angular spacing.

    The paper sets eps = beta / N_q (Sec. 2.3, Sec. 4.1); the workloads here
    state beta "scaled by the ordinate spacing", read as beta * sqrt(4 pi/Q).
    """
    return float(beta) * math.sqrt(FOUR_PI / Q)


def time_grid(t_final: float, cfl: float, h: float) -> tuple[int, float]:
    """Uniform steps landing exactly on t_final: n = ceil(t_final/(cfl h)), dt = t_final/n.

    The paper defines the CFL number as dt/dx (Sec. 4.1).
    """
    n = int(math.ceil(t_final / (cfl * h) - 1e-12))
    n = max(n, 1)
    return n, t_final / n


def cell_centres(n: int, lo: float, hi: float) -> np.ndarray:
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h


def line_source_psi0(nx: int, ny: int, Q: int, x0=-1.5, x1=1.5, y0=-1.5, y1=1.5,
                     delta: float = 0.03 ** 2, floor: float = 1e-4) -> np.ndarray:
    """Line-source initial angular flux, Sec. 4.1: max{floor, exp(-|x|^2/(4 delta))/(4 pi delta)}.

    Point values at cell centres, the same for every ordinate.  Returns
    float64 ``[ny][nx][Q]``.
    """
    xc = cell_centres(nx, x0, x1)
    yc = cell_centres(ny, y0, y1)
    r2 = yc[:, None] ** 2 + xc[None, :] ** 2
    f = np.maximum(floor, np.exp(-r2 / (4.0 * delta)) / (4.0 * math.pi * delta))
    return np.repeat(f[:, :, None], Q, axis=2)


def line_source_materials(nx: int, ny: int, sigma_s: float = 1.0, sigma_a: float = 0.0):
    """Sec. 4.1: sigma_s = sigma_t = 1, no absorption, no source."""
    sa = np.full((ny, nx), sigma_a)
    ss = np.full((ny, nx), sigma_s)
    q = np.zeros((ny, nx))
    return sa, ss, q


# Lattice material table, Table 1 of Sec. 4.2: (sigma_a, sigma_s, Q) per colour.
LATTICE_TABLE = {
    "white": (0.0, 1.0, 0.0),
    "black": (10.0, 0.0, 0.0),
    "orange": (10.0, 0.0, 1.0),
}


def lattice_block_map(centre_column_white: bool = False) -> list[list[str]]:
    """7 x 7 colour map of unit blocks on [0,7]^2, indexed [j][i] (j = y block, i = x block).

    Absorbers (black) sit on the checkerboard 1 <= i, j <= 5 with i + j even,
    except the source block (3,3) (orange) and the block above it (3,5), which
    stays white.  With ``centre_column_white`` every block of column i = 3
    except the source is white.  The paper's layout figure is not legible, so
    this is the usual Brunner lattice layout (Sec. 4.2).
    """
    cmap = [["white"] * 7 for _ in range(7)]
    for j in range(7):
        for i in range(7):
            if 1 <= i <= 5 and 1 <= j <= 5 and (i + j) % 2 == 0:
                cmap[j][i] = "black"
    cmap[5][3] = "white"
    if centre_column_white:
        for j in range(7):
            cmap[j][3] = "white"
    cmap[3][3] = "orange"
    return cmap


def lattice_materials(cells_per_block: int, source_absorbs: bool = True,
                      centre_column_white: bool = False):
    """Per-cell (sigma_a, sigma_s, Q_table) for the lattice on [0,7]^2 with 7*cells_per_block cells a side.

    ``source_absorbs`` follows Table 1 (the orange block absorbs, sigma_a = 10);
    False gives a scattering source block (sigma_a = 0, sigma_s = 1).
    The returned source is the table's Q (particles per area per time); the
    per-ordinate source is Q / (4 pi) (see ``per_ordinate_source``).
    """
    cmap = lattice_block_map(centre_column_white)
    n = 7 * cells_per_block
    sa = np.empty((n, n))
    ss = np.empty((n, n))
    qt = np.empty((n, n))
    for j in range(7):
        for i in range(7):
            a, s, src = LATTICE_TABLE[cmap[j][i]]
            if cmap[j][i] == "orange" and not source_absorbs:
                a, s = 0.0, 1.0
            sl = (slice(j * cells_per_block, (j + 1) * cells_per_block),
                  slice(i * cells_per_block, (i + 1) * cells_per_block))
            sa[sl], ss[sl], qt[sl] = a, s, src
    return sa, ss, qt


def per_ordinate_source(q_table: np.ndarray) -> np.ndarray:
    """Isotropic source per ordinate, q_table / (4 pi), so the source of Phi is q_table."""
    return q_table / FOUR_PI


def random_psi(seed: int, ny: int, nx: int, Q: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(ny, nx, Q))


def random_materials(seed: int, ny: int, nx: int, sa_max=2.0, ss_max=2.0, q_max=1.0):
    rng = np.random.default_rng(seed + 7919)
    sa = rng.uniform(0.0, sa_max, size=(ny, nx))
    ss = rng.uniform(0.0, ss_max, size=(ny, nx))
    q = rng.uniform(0.0, q_max, size=(ny, nx))
    return sa, ss, q


@dataclass
class Workload:
    """One as-S_N problem: grid, quadrature order, kernel width, materials, time span."""
    name: str
    kind: str               # "line_source" | "lattice" | "random"
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    n_polar: int
    n_azim: int
    beta: float
    sigma_as: float = 5.0
    cfl: float = 0.5
    t_final: float = 1.0
    seed: int = 0
    extra: dict = field(default_factory=dict)
    quadrature: str = "product"     # "product": n_polar x n_azim; "icosahedron": order ico_order
    ico_order: int = 0              # N_q = 10 (ico_order - 1)^2 + 2
    ico_base: str = "printed"       # "printed" (the paper's Appendix A rule) or "regular"
    ico_midpoints: str = "sphere"   # dual-cell midpoints of the mapped ("sphere") or flat ("flat") points
    eps_rule: str = "spacing"       # "spacing": beta sqrt(4 pi / Q); "paper": beta / N_q (Sec. 4.1)
    normalisation: str = "column"   # kernel matrix: "column" or the paper's "row" (Sec. 3.2)
    scheme: str = "euler"           # "euler" (first-order upwind) or "heun" (Heun + minmod)
    dt_rule: str = "cfl"            # "cfl": dt = cfl h; "bound": dt = cfl x the scheme's admissible dt
    si_eps: float = 1e-4            # implicit scheme: source-iteration tolerance (Sec. 4.1)
    gmres_tol: float = 1.5e-8       # implicit scheme: GMRES relative residual (Sec. 4.1)

    @property
    def Q(self) -> int:
        if self.quadrature == "icosahedron":
            return 10 * (self.ico_order - 1) ** 2 + 2
        return self.n_polar * self.n_azim

    @property
    def h(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def eps(self) -> float:
        if self.eps_rule == "paper":
            return self.beta / self.Q
        return eps_from_beta(self.beta, self.Q)

    def steps(self) -> tuple[int, float]:
        if self.dt_rule != "cfl":
            raise ValueError(f"{self.name}: dt is a fraction of the admissible dt; use steps_for(bound)")
        return time_grid(self.t_final, self.cfl, self.h)

    def steps_for(self, dt_bound: float) -> tuple[int, float]:
        """(n, dt) landing on t_final with dt <= cfl x dt_bound (dt_rule "bound") or <= cfl h."""
        if self.dt_rule == "cfl":
            return self.steps()
        n = max(1, int(math.ceil(self.t_final / (self.cfl * dt_bound) - 1e-12)))
        return n, self.t_final / n

    def materials(self):
        """(sigma_a, sigma_s, q_per_ordinate), each [ny][nx] float64."""
        if self.kind == "line_source":
            return line_source_materials(self.nx, self.ny)
        if self.kind == "lattice":
            assert self.nx == self.ny and self.nx % 7 == 0
            sa, ss, qt = lattice_materials(self.nx // 7,
                                           source_absorbs=self.extra.get("source_absorbs", True))
            return sa, ss, per_ordinate_source(qt)
        return random_materials(self.seed, self.ny, self.nx)

    def psi0(self) -> np.ndarray:
        if self.kind == "line_source":
            return line_source_psi0(self.nx, self.ny, self.Q, self.x0, self.x1, self.y0, self.y1)
        if self.kind == "lattice":
            return np.zeros((self.ny, self.nx, self.Q))
        return random_psi(self.seed, self.ny, self.nx, self.Q)


def line_source(n: int, n_polar: int, n_azim: int, beta: float, t_final: float = 1.0,
                name: str | None = None) -> Workload:
    return Workload(name or f"line_source_{n}x{n}_Q{n_polar * n_azim}", "line_source",
                    n, n, -1.5, 1.5, -1.5, 1.5, n_polar, n_azim, beta, t_final=t_final)


def lattice(n: int, n_polar: int, n_azim: int, beta: float, t_final: float = 3.2,
            name: str | None = None) -> Workload:
    return Workload(name or f"lattice_{n}x{n}_Q{n_polar * n_azim}", "lattice",
                    n, n, 0.0, 7.0, 0.0, 7.0, n_polar, n_azim, beta, t_final=t_final)


def paper_line_source(n: int = 200, order: int = 4, beta: float = 4.5, sigma_as: float = 5.0,
                      t_final: float = 1.0, base: str = "printed", name: str | None = None) -> Workload:
    """The paper's explicit as-S_N line source (Sec. 4.1): [-1.5, 1.5]^2, the icosahedron quadrature
    (Sec. 3.3; order 4 gives N_q = 92), eps = beta / N_q, the row normalisation of Sec. 3.2 and Heun +
    minmod; sigma_as = 5, beta = 4.5 as in its explicit runs.  The time step is 0.95 of the scheme's
    admissible dt (the paper's dt/dx = 0.95 is unstable for the unsplit two-dimensional scheme)."""
    q = 10 * (order - 1) ** 2 + 2
    return Workload(name or f"line_source_{n}x{n}_ico{q}", "line_source", n, n, -1.5, 1.5, -1.5, 1.5, 0, 0,
                    beta, sigma_as=sigma_as, cfl=0.95, t_final=t_final, quadrature="icosahedron",
                    ico_order=order, ico_base=base, eps_rule="paper", normalisation="row", scheme="heun",
                    dt_rule="bound")


def paper_line_source_implicit(n: int = 200, order: int = 4, beta: float = 4.0, sigma_as: float = 7.0,
                               t_final: float = 1.0, name: str | None = None) -> Workload:
    """The paper's implicit as-S_N line source (Sec. 4.1): as paper_line_source, with the implicit
    sweeping-Krylov scheme at dt/dx = 2 and its parameters sigma_as = 7, beta = 4."""
    q = 10 * (order - 1) ** 2 + 2
    return Workload(name or f"line_source_{n}x{n}_ico{q}_implicit", "line_source", n, n, -1.5, 1.5, -1.5, 1.5,
                    0, 0, beta, sigma_as=sigma_as, cfl=2.0, t_final=t_final, quadrature="icosahedron",
                    ico_order=order, eps_rule="paper", normalisation="row", scheme="implicit")


def paper_lattice(n: int = 280, order: int = 4, beta: float = 4.5, sigma_as: float = 5.0,
                  t_final: float = 3.2, name: str | None = None) -> Workload:
    """The paper's explicit as-S_N lattice (Sec. 4.2) with its quadrature, kernel width, normalisation
    and scheme as in paper_line_source; 280^2 cells as in its lattice figures."""
    q = 10 * (order - 1) ** 2 + 2
    return Workload(name or f"lattice_{n}x{n}_ico{q}", "lattice", n, n, 0.0, 7.0, 0.0, 7.0, 0, 0, beta,
                    sigma_as=sigma_as, cfl=0.95, t_final=t_final, quadrature="icosahedron", ico_order=order,
                    eps_rule="paper", normalisation="row", scheme="heun", dt_rule="bound")


def paper_lattice_implicit(n: int = 280, order: int = 4, beta: float = 4.0, sigma_as: float = 7.0,
                           t_final: float = 3.2, name: str | None = None) -> Workload:
    """The paper's implicit as-S_N lattice (Sec. 4.2): as paper_lattice, with the implicit sweeping-Krylov
    scheme at dt/dx = 2 and its implicit parameters sigma_as = 7, beta = 4."""
    q = 10 * (order - 1) ** 2 + 2
    return Workload(name or f"lattice_{n}x{n}_ico{q}_implicit", "lattice", n, n, 0.0, 7.0, 0.0, 7.0, 0, 0, beta,
                    sigma_as=sigma_as, cfl=2.0, t_final=t_final, quadrature="icosahedron", ico_order=order,
                    eps_rule="paper", normalisation="row", scheme="implicit")


# The five workloads of the measurement plan.
LINE_SOURCE_64 = line_source(64, 8, 16, 1.0 / 8.0, name="line_source_64x64_Q128_fp64")
LATTICE_448 = lattice(448, 16, 32, 0.5, name="lattice_448x448_Q512")
LINE_SOURCE_2048 = line_source(2048, 16, 16, 1.0 / 8.0, name="line_source_2048x2048_Q256")
LINE_SOURCE_256_ACC = line_source(256, 16, 16, 1.0 / 8.0, name="line_source_256x256_Q256")

# The paper's own explicit as-S_4 runs (N_q = 92).
PAPER_LINE_SOURCE_200 = paper_line_source(200)
PAPER_LATTICE_280 = paper_lattice(280)
PAPER_LINE_SOURCE_200_IMPLICIT = paper_line_source_implicit(200)
PAPER_LATTICE_280_IMPLICIT = paper_lattice_implicit(280)

WORKLOADS = {w.name: w for w in (LINE_SOURCE_64, LATTICE_448, LINE_SOURCE_2048, LINE_SOURCE_256_ACC,
                                 PAPER_LINE_SOURCE_200, PAPER_LATTICE_280, PAPER_LINE_SOURCE_200_IMPLICIT,
                                 PAPER_LATTICE_280_IMPLICIT)}

QUAD_ORDERS = {64: (8, 8), 128: (8, 16), 256: (16, 16), 512: (16, 32)}


def ensemble(seed: int = 0, count: int = 64, sides=(128, 256, 512), qs=(64, 128, 256, 512),
             beta_range=(0.1, 1.0)) -> list[Workload]:
    """Batched ensemble: sides, Q and beta drawn from a seed, line source / lattice 50/50.

    A lattice side is rounded to a multiple of 7 so the 7 x 7 block map is exact.
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        side = int(rng.choice(sides))
        Q = int(rng.choice(qs))
        beta = float(rng.uniform(*beta_range))
        npol, naz = QUAD_ORDERS[Q]
        if rng.uniform() < 0.5:
            out.append(line_source(side, npol, naz, beta, t_final=1.0, name=f"ens{k}_ls{side}_Q{Q}"))
        else:
            s7 = 7 * max(1, round(side / 7))
            out.append(lattice(s7, npol, naz, beta, t_final=3.2, name=f"ens{k}_lat{s7}_Q{Q}"))
    return out


def serving_requests(seed: int = 0, count: int = 64, sides=(64, 128, 256, 512, 1024), qs=(64, 128, 256, 512),
                     beta_range=(0.1, 1.0), t_range=(0.5, 2.0)) -> list[Workload]:
    """Serving workload: one solve per request, side, Q, beta and t_final drawn from a seed,
    line source / lattice 50/50 (lattice sides rounded to a multiple of 7)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        side = int(rng.choice(sides))
        Q = int(rng.choice(qs))
        beta = float(rng.uniform(*beta_range))
        t_final = float(rng.uniform(*t_range))
        npol, naz = QUAD_ORDERS[Q]
        if rng.uniform() < 0.5:
            out.append(line_source(side, npol, naz, beta, t_final=t_final, name=f"req{k}_ls{side}_Q{Q}"))
        else:
            s7 = 7 * max(1, round(side / 7))
            out.append(lattice(s7, npol, naz, beta, t_final=t_final, name=f"req{k}_lat{s7}_Q{Q}"))
    return out


def poisson_arrivals(seed: int, count: int, rate: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate, starting at 0."""
    rng = np.random.default_rng(seed + 7919)
    gaps = rng.exponential(1.0 / rate, size=count)
    gaps[0] = 0.0
    return np.cumsum(gaps)


def icosahedron_order2():
    """The paper's printed order-2 icosahedron quadrature (Appendix A): Omega [12][3], w [12].

    Read from the cited fixture tests/golden/icosahedron_order2.txt (input data, not method code).
    """
    import os
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                        "icosahedron_order2.txt")
    rows = np.loadtxt(path, comments="#")
    return rows[:, :3].copy(), rows[:, 3].copy()


def parameter_study_grid():
    """(sigma_as, beta) pairs of the coarse parameter study (Sec. 4.1: 306 configurations, explicit,
    N_q = 12 on 50 x 50 cells).  The paper's heatmap values are unreadable; read here as 17 sigma_as
    values 0 .. 16 times 18 beta values 0.5 .. 9 (eps = beta / N_q)."""
    return [(float(s), float(b)) for s in np.linspace(0.0, 16.0, 17) for b in np.linspace(0.5, 9.0, 18)]

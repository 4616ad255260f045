"""Plain FP64 CPU oracle for the explicit as-S_N time step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
statement of what the GPU path must compute.  Only the test suite, the smoke
check of ``__graft_entry__`` and the CPU-baseline / reference legs of
``bench.py`` may import it; the library under ``paper_1911_08801_gb300`` never
does, and shares no code with it.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` against closed forms, invariants and special
cases (quadrature exactness, kernel normalisation and transport moments,
Funk-Hecke eigenvalues of the kernel matrix, exact upwind shifts and binomial
spreading, discrete decay laws, the discrete mass balance, the eps -> 0 limit,
and the symmetries of the line source).  The Heun + minmod functions (the paper's
explicit scheme, Sec. 3.1) are pinned by the minmod definition, exactness of the
limited fluxes on monotone quadratics, constant-state and periodic conservation,
no new extrema on an advected step, the exact RK2 amplification factor on decay,
and a second-order convergence rate on a smooth periodic profile.  The icosahedron
quadrature (Sec. 3.3) is pinned by the paper's printed order-2 table (Appendix A),
the point count N_q = 10 (k-1)^2 + 2, the 4 pi weight sum, its symmetries, exact
degree-5 moments on the regular base and convergence of moments on the printed one.
The admissible time step of the limited scheme (heun_admissible_dt) is pinned by
positivity of a stage at the bound and by a constructed state that reaches zero
exactly there and goes negative just above it.
The implicit step (``oracle.implicit``, Sec. 3.4-3.5) is pinned by the printed
symmetric part of the second-order upwind operator (Appendix B), sweeps that invert
the streaming operator, the exact implicit-Euler decay of an isotropic state, the
source iteration and GMRES against dense solves, and the sweeping-Krylov step
against the directly assembled implicit system.
"""
from .assn_oracle import *  # noqa: F401,F403
from .implicit import *  # noqa: F401,F403

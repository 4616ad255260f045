/*
 * assn.h -- C ABI of libassn: the explicit time step of the artificial-scattering
 * S_N (as-S_N) method for 2D radiative transfer on one NVIDIA GB300 (sm_103a).
 *
 * Method: Camminady, Frank, Hauck, Kusch, "Ray Effect Mitigation for the Discrete
 * Ordinates Method Using Artificial Scattering", arXiv:1911.08801.
 *
 * One step advances every ordinate's angular flux psi_q on a uniform Cartesian grid by
 * forward Euler applied to the as-S_N equations (Sec. 3.2, Eq. (as-S_N equations)):
 *
 *   psi_q' = psi_q - dt [Omega_q . grad psi_q]_upwind          (first-order upwind, vacuum inflow)
 *            - dt (sigma_a + sigma_s + sigma_as) psi_q
 *            + dt sigma_s Phi / sum_p w_p                       (isotropic physical scattering)
 *            + dt sigma_as sum_p K_qp psi_p                     (artificial in-scattering)
 *            + dt q
 *
 * with Phi = sum_p w_p psi_p and K the normalised forward-peaked kernel matrix built from
 * s_eps(mu) ~ exp(-(1-mu)^2/eps^2) (Sec. 2.3, Eq. (scattering kernel)).
 *
 * Conventions common to every entry point:
 *  - Every call returns an assn_status (0 = ASSN_OK, negative = error).  No call aborts the
 *    process or throws; assn_last_error() gives a one-line message for the last failure on
 *    a problem.
 *  - Host arrays are owned by the caller and are copied during the call.  Cell fields are
 *    row-major [ny][nx] (x fastest); angular fluxes are [ny][nx][Q] (ordinate fastest),
 *    ordinates in the order the quadrature was given.
 *  - The library owns all device memory of a problem (allocated by assn_create and the
 *    set_* calls, freed by assn_destroy).  Device-pointer arguments (names ending in _dev)
 *    are caller-owned device buffers; the call only reads or writes them on the problem's
 *    stream, asynchronously.
 *  - Work is issued on the problem's stream (the cudaStream_t passed to assn_create, or a
 *    stream the library creates when NULL).  Calls documented as "syncs" wait for it.
 *  - One problem must not be used from two host threads at once.
 */
#ifndef ASSN_H
#define ASSN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASSN_ABI_VERSION 1

typedef enum {
    ASSN_OK = 0,
    ASSN_ERR_ARG = -1,          /* invalid argument (null pointer, size, range)            */
    ASSN_ERR_OOM = -2,          /* device or host allocation failed                         */
    ASSN_ERR_CUDA = -3,         /* a CUDA call failed; message in assn_last_error           */
    ASSN_ERR_UNSTABLE = -4,     /* dt violates the positivity bound of the explicit step    */
    ASSN_ERR_NONFINITE = -5,    /* NaN/Inf found in the state                               */
    ASSN_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up                       */
    ASSN_ERR_STATE = -7,        /* call out of order (e.g. step before quadrature is set)   */
    ASSN_ERR_UNSUPPORTED = -8,  /* size or mode not supported by the selected kernel        */
    ASSN_ERR_CANCELLED = -9     /* a server request was cancelled (assn_server_cancel)       */
} assn_status;

/* Arithmetic of the step.  State and stencil are FP64 for ASSN_FP64 and FP32 otherwise;
 * the artificial-scattering contraction runs in:
 *   ASSN_FP64   FP64 CUDA cores (the plain FP64 GPU path)
 *   ASSN_FP32   FP32 CUDA cores
 *   ASSN_BF16   tcgen05 tensor cores, BF16 operands, FP32 accumulation (one pass)
 *   ASSN_BF16X3 tcgen05, operands split into BF16 hi+lo, three passes (hi*hi + hi*lo + lo*hi),
 *               FP32 accumulation: about FP32-level accuracy of the contraction.
 *   ASSN_TF32   tcgen05 kind::tf32, both operands rounded to TF32 (10 stored significand bits,
 *               to nearest, ties away from zero), FP32 accumulation, one pass.
 *   ASSN_BF16X2 tcgen05, the kernel matrix split into BF16 hi+lo, the flux in one BF16 part, two
 *               passes (hi*psi~ + lo*psi~), FP32 accumulation.
 *   TF32 and BF16X2 run on the paired-SM kernel only (tiling variant 2: 193..256 or 449..512
 *   ordinates), for the forward-Euler and Heun schemes, alone or in batches of such members;
 *   other ordinate counts or variants, the one-launch batch grouping, autotune and the server
 *   return ASSN_ERR_UNSUPPORTED.
 * K itself is always built in FP64 on the device. */
typedef enum {
    ASSN_FP64 = 0,
    ASSN_FP32 = 1,
    ASSN_BF16 = 2,
    ASSN_BF16X3 = 3,
    ASSN_TF32 = 4,
    ASSN_BF16X2 = 5
} assn_precision;

/* Kernel shape.  ASSN_KERNEL_GAUSS is the paper's s_eps(mu) ~ exp(-(1-mu)^2/eps^2)
 * (Sec. 2.3); ASSN_KERNEL_EXP is exp((mu-1)/eps^2).  Constant prefactors cancel in the
 * normalisation and are not applied. */
typedef enum { ASSN_KERNEL_GAUSS = 0, ASSN_KERNEL_EXP = 1 } assn_kernel_kind;

/* Normalisation of K.  COLUMN: K_qp = w_p c_p s_qp with c_p = 1/sum_q w_q s_qp, so
 * sum_q w_q K_qp = w_p and the operator conserves particles exactly.  ROW: the paper's
 * c_q = 1/sum_p w_p s_qp (Sec. 3.2, normalisation factors), rows of K sum to one. */
typedef enum { ASSN_NORM_COLUMN = 0, ASSN_NORM_ROW = 1 } assn_normalisation;

typedef enum { ASSN_BC_VACUUM = 0 } assn_boundary;

/* Time and space discretisation of assn_step.
 *   ASSN_SCHEME_EULER_UPWIND  forward Euler with first-order upwind transport (the default)
 *   ASSN_SCHEME_HEUN_MINMOD   the paper's explicit scheme (Sec. 3.1): Heun's method (two stages,
 *                             psi* = psi + dt L(psi), psi^{n+1} = (psi + psi* + dt L(psi*))/2)
 *                             with second-order upwind fluxes from minmod-limited slopes (two zero
 *                             ghost cells per vacuum side); all precisions (tensor-core problems on
 *                             the paired-SM kernel at 256 / 512 ordinates, else variant 0).
 *   ASSN_SCHEME_IMPLICIT      the paper's implicit method (Sec. 3.4-3.5, Alg. 1-3): implicit Euler
 *                             with the second-order upwind stencil without limiter (flux difference
 *                             3/2 psi_j - 2 psi_{j-1} + 1/2 psi_{j-2}, x and y stencils added), solved
 *                             by source iteration over transport sweeps inside GMRES on the scalar
 *                             flux; FP64 and FP32 problems (CUDA cores); no step-size restriction. */
typedef enum {
    ASSN_SCHEME_EULER_UPWIND = 0,
    ASSN_SCHEME_HEUN_MINMOD = 1,
    ASSN_SCHEME_IMPLICIT = 2
} assn_scheme;

typedef struct assn_problem assn_problem;

/* Maximum ordinate count and grid side accepted by assn_create / set_quadrature. */
#define ASSN_MAX_Q 1024
#define ASSN_MAX_SIDE 32768

/* Create a problem on the current CUDA device: nx x ny cells covering [x0,x1] x [y0,y1]
 * with square cells (requires (x1-x0)/nx == (y1-y0)/ny to 1e-12 relative).
 * precision: an assn_precision.  stream: a cudaStream_t, or NULL for a library-owned
 * stream.  On success *out receives the handle; on error *out is NULL.
 * Errors: ASSN_ERR_ARG for non-positive sizes, non-square cells or an unknown precision;
 * ASSN_ERR_CUDA if no device is usable. */
int assn_create(assn_problem** out, int nx, int ny, double x0, double x1, double y0,
                double y1, int precision, void* stream);

/* Free all device and host memory of the problem (synchronises its stream).  NULL is a no-op. */
int assn_destroy(assn_problem* p);

/* Set an arbitrary quadrature (Sec. 3.1 quadrature rule): Q ordinates, omega[Q*3] unit
 * directions (x, y, z), w[Q] positive weights.  Transport uses the projection (x, y) onto
 * the grid plane (Sec. 4).  Resets the state to zero and invalidates K.
 * Errors: ASSN_ERR_ARG if Q < 1 or Q > ASSN_MAX_Q, a weight <= 0 or a direction with
 * |norm - 1| > 1e-9. */
int assn_set_quadrature(assn_problem* p, int Q, const double* omega, const double* w);

/* Product quadrature: n_polar Gauss-Legendre nodes in mu (computed on the host by Newton
 * iteration on P_n) times n_azim azimuths phi_k = (k+1/2) 2 pi / n_azim; weight
 * w = w_GL * 2 pi / n_azim; ordinate q = k*n_polar + i (azimuth-major: the ordinates of azimuth
 * k are consecutive, and the kernel matrix repeats under the rotation q -> q + n_polar, which the
 * paired-SM kernel uses to keep it resident).  Same effects as assn_set_quadrature. */
int assn_set_product_quadrature(assn_problem* p, int n_polar, int n_azim);

/* Icosahedron quadrature (Sec. 3.3; the paper prints the order-2 rule in Appendix A).  Order k
 * puts k - 1 equal segments on every edge of the base solid's 20 triangular faces; the lattice
 * points are mapped to the unit sphere and weighted by the area of their spherical barycentric
 * dual cells (corners at the centres of the neighbouring triangles and the midpoints of the edges
 * between them); N_q = 10 (k-1)^2 + 2, weights sum to 4 pi, one point at (0, 0, 1).
 * ASSN_ICO_REGULAR: the regular icosahedron, vertices (0, +-1, +-g), (+-1, +-g, 0), (+-g, 0, +-1),
 * g the golden ratio.  ASSN_ICO_PRINTED: the base solid that reproduces the printed order-2
 * points and weights: each (+-g, 0, +-1) replaced by the (+-1, 0, +-g) with the same signs, the
 * faces kept.  Both turned about x so that (0, 1, g) maps to (0, 0, 1).  The dual cell's centres and
 * midpoints are those of the mapped points; with the ASSN_ICO_FLAT_MIDPOINTS flag those of the flat
 * lattice, mapped (the cell drawn on the flat face).  The two agree at order 2 (the printed rule) and
 * differ from order 3 on. */
typedef enum {
    ASSN_ICO_PRINTED = 0,
    ASSN_ICO_REGULAR = 1,
    ASSN_ICO_FLAT_MIDPOINTS = 2   /* flag, OR with a base: the dual cell's midpoints from the flat lattice */
} assn_ico_base;

#define ASSN_ICO_MAX_ORDER 64

/* Compute the icosahedron quadrature of the given order (2 .. ASSN_ICO_MAX_ORDER) and base on
 * the host in FP64.  Returns N_q.  With omega and w non-NULL and capacity >= N_q, also writes the
 * directions omega[N_q*3] (x, y, z) and weights w[N_q] (caller-owned); with either NULL, only
 * returns N_q.  Needs no problem and no device.
 * Errors (negative return): ASSN_ERR_ARG for an order or base out of range, or capacity < N_q. */
int assn_icosahedron_quadrature(int order, int base, double* omega, double* w, int capacity);

/* Set the icosahedron quadrature of the given order and base on p (N_q <= ASSN_MAX_Q, so
 * order <= 11).  Same effects as assn_set_quadrature.  Errors: ASSN_ERR_ARG for an order or
 * base out of range. */
int assn_set_icosahedron_quadrature(assn_problem* p, int order, int base);

/* Copy the quadrature back: omega[Q*3], w[Q] (either may be NULL).  *Q_out receives Q. */
int assn_get_quadrature(const assn_problem* p, int* Q_out, double* omega, double* w);

/* Per-cell cross sections sigma_a, sigma_s >= 0 and the isotropic per-ordinate source q
 * (added to every ordinate's equation, Eq. (1)), each [ny][nx] host FP64, copied.
 * Errors: ASSN_ERR_ARG on NULL or a negative / non-finite cross section. */
int assn_set_cross_sections(assn_problem* p, const double* sigma_a, const double* sigma_s,
                            const double* q);

/* Artificial scattering strength sigma_as >= 0 (Sec. 2.3, constant in space) and kernel
 * width eps > 0 (Sec. 2.3: eps = beta/N_q in the paper; callers pass eps directly).
 * Builds K on the device in FP64 (one block per normalised line) and derives the operands
 * of the selected precision.  Requires a quadrature.  Errors: ASSN_ERR_ARG, ASSN_ERR_STATE. */
int assn_set_artificial_scattering(assn_problem* p, double sigma_as, double eps, int kernel_kind,
                                   int normalisation);

/* Copy the FP64 K (row q, column p: K[q*Q + p]) to the host.  Syncs. */
int assn_get_kernel_matrix(assn_problem* p, double* K_host);

/* State.  psi[ny][nx][Q] host FP64, copied (converted to FP32 unless the precision is FP64).
 * set_state syncs before returning; get_state syncs. */
int assn_set_state(assn_problem* p, const double* psi_host);
int assn_get_state(assn_problem* p, double* psi_host);

/* FP32 state copies for FP32/BF16/BF16X3 problems: psi[ny][nx][Q] host FP32 (pinned host memory
 * gives full copy bandwidth).  set_state_f32 is asynchronous on the problem's stream: the
 * caller keeps psi alive and unchanged until the stream has passed the copy.  get_state_f32
 * syncs.  ASSN_ERR_UNSUPPORTED on an FP64 problem. */
int assn_set_state_f32(assn_problem* p, const float* psi_host);
int assn_get_state_f32(assn_problem* p, float* psi_host);

/* Line-source initial state (Sec. 4.1), computed on the device:
 * psi_q(x) = max{floor, exp(-|x|^2/(4 delta)) / (4 pi delta)} at cell centres for every q. */
int assn_init_line_source(assn_problem* p, double delta, double floor_value);

/* Scheme of later assn_step calls (an assn_scheme).  ASSN_ERR_ARG for an unknown scheme;
 * batches and assn_step_device take ASSN_SCHEME_EULER_UPWIND only (ASSN_ERR_UNSUPPORTED). */
int assn_set_scheme(assn_problem* p, int scheme);
int assn_get_scheme(const assn_problem* p, int* scheme);

/* Parameters of the implicit scheme (defaults in parentheses): the source iteration stops when
 * ||psi^{l+1} - psi^l||_2 < si_eps (1 - T) / T, T = max_cells dt sigma_as / (1 + dt (sigma_a +
 * sigma_s + sigma_as)) (1e-4), or after max_si iterations (1000), and for FP32 problems also when the
 * difference stops decreasing (the rounding floor of the state); GMRES on the scalar flux, restarted
 * every `restart` iterations (30), stops at relative residual gmres_tol (1.5e-8; for FP32 problems
 * not below 2^-20, the rounding level of FP32 source iterations) or after max_gmres iterations
 * (500).  Errors: ASSN_ERR_ARG for negative tolerances, restart outside 1..200 or limits < 1. */
int assn_set_implicit_params(assn_problem* p, double si_eps, double gmres_tol, int restart, int max_si,
                             int max_gmres);

/* Totals since the problem was created: source iterations, GMRES iterations, transport sweeps of
 * the implicit scheme (any pointer may be NULL). */
int assn_implicit_stats(const assn_problem* p, int64_t* source_iterations, int64_t* gmres_iterations,
                        int64_t* sweeps);

/* Exactly `iterations` source iterations (Alg. 1) of the implicit scheme at step size dt, for
 * (L - dt sigma_as K) psi = dt R: psi^{l+1} = L^{-1} dt (sigma_as K psi^l + R) from psi^0 = psi0.
 * R, psi0, psi_out: host [ny][nx][Q] FP64 (computed in the problem's precision).  One iteration
 * from any psi0 with sigma_as = 0 is one transport sweep.  Requires quadrature, cross sections and
 * K; ASSN_ERR_UNSUPPORTED for BF16 / BF16X3 problems. */
int assn_implicit_source_iteration(assn_problem* p, double dt, const double* R, const double* psi0,
                                   int iterations, double* psi_out);

/* Largest admissible dt for the problem's scheme.  Forward Euler: the explicit step keeps every
 * coefficient of the update non-negative (positivity): dt * (max_q [(|Omega_x,q| + |Omega_y,q|)/h
 * + sigma_as (1 - K_qq)] + max_cells [sigma_a + sigma_s]) <= 1.  Heun + minmod: every
 * forward-Euler stage keeps the coefficients non-negative (minmod bounds the transport factor by
 * 3/2): dt * (max_q [3/2 (|Omega_x,q| + |Omega_y,q|)/h + sigma_as (1 - K_qq)] + max_cells [sigma_a +
 * sigma_s]) <= 1.  K_qq is taken from the operator as stored (rounded in BF16 / BF16X3).
 * Implicit: infinity (no restriction).  Requires quadrature, cross sections and K. */
int assn_max_stable_dt(assn_problem* p, double* dt_out);

/* Advance nsteps explicit steps of size dt on the problem's stream (asynchronous; the
 * state buffers ping-pong on the device).  Errors: ASSN_ERR_STATE if quadrature, cross
 * sections or K are missing; ASSN_ERR_UNSTABLE if dt exceeds assn_max_stable_dt by more
 * than 1e-12 relative; ASSN_ERR_CUDA on a launch failure; ASSN_ERR_TIMEOUT if a bounded
 * device-side wait in the tensor-core kernel gave up (reported by a later syncing call). */
int assn_step(assn_problem* p, int nsteps, double dt);

/* Same step, with the ordinate state supplied and returned by the caller in device memory
 * laid out as the problem's own buffers ([ny][nx][Qpad] of FP32, or FP64 for ASSN_FP64;
 * Qpad from assn_layout).  psi_in_dev and psi_out_dev must not overlap.  Asynchronous, on the
 * problem's stream.  Where the problem's steps run on the paired-SM kernel (variant 2) and
 * psi_in_dev is 16-byte aligned, the step runs there (bitwise equal to assn_step); other tensor-core
 * problems run the one-tile-per-CTA kernel (variant 1). */
int assn_step_device(assn_problem* p, const void* psi_in_dev, void* psi_out_dev, double dt);

/* One call from host data to host result: upload psi0 (FP32 [ny][nx][Q] host; pinned memory gives
 * full copy bandwidth), take nsteps steps of size dt on the device, and return the scalar flux
 * [ny][nx] in FP64.  Syncs.  FP32/BF16/BF16X3 problems only (ASSN_ERR_UNSUPPORTED on FP64). */
int assn_run_f32(assn_problem* p, const float* psi0_host, int nsteps, double dt, double* phi_host);

/* Tensor-core kernel and tiling (BF16 / BF16X3 problems).  variant -1 (the initial value):
 * automatic, variant 2 where it applies, else variant 0.  variant 0: persistent warp-specialised
 * kernel, one CTA per SM, TMA-fed rings and two TMEM accumulator buffers; variant 1: one tile per
 * CTA (simpler, slower); variant 2: paired-SM kernel, a cluster of two CTAs sharing each M = 256
 * contraction (cta_group::2) over 2D tiles of 16 x 8 (512 ordinates) or 16 x 16 cells (256),
 * forward Euler in BF16 with 193..256 or 449..512 ordinates (else ASSN_ERR_UNSUPPORTED at the next
 * step; tile_cells is fixed by the ordinate count).  tile_cells: cells per tile (32, 64, 128 or 256;
 * 0 = automatic).  stages: ring depth (2..8; 0 = automatic).  Takes effect at the next step; the
 * results do not depend on these choices.  ASSN_ERR_UNSUPPORTED at the next step if the
 * combination does not fit the SM. */
int assn_set_tiling(assn_problem* p, int tile_cells, int stages, int variant);

/* Rings of the persistent kernels (variants 0 and 2; BF16 / BF16X3 problems): depths of the staging
 * ring (FP32 flux chunks fed by TMA), the operand ring (BF16 chunks written by the converter warps)
 * and the kernel-matrix ring (2..8 each; 0 = automatic), and the ordinate blocks of 128 that one
 * kernel-matrix request brings (1, 2, 4, 8; 0 = automatic; variant 0 only; variant 2 reads it as
 * 64-ordinate chunks per stage, 1 or 2).  Variant 2 with kernel_matrix = 0 keeps the kernel matrix
 * resident in shared memory where its distinct [128 x 64] blocks fit (all of them at 256 ordinates;
 * at 512, the 8 distinct blocks per SM of an azimuth-major product quadrature), found by reading G
 * back once when the step is planned (a sync; not done while the stream is being captured), and
 * get_rings then reports kernel_matrix = 0.  Results do not depend on these choices.  Selects
 * variant 0 unless variant 2 was set explicitly.  get_rings reports the resolved values (any pointer
 * may be NULL); ASSN_ERR_UNSUPPORTED at the next step / get if the rings do not fit shared memory. */
int assn_set_rings(assn_problem* p, int staging, int operand, int kernel_matrix, int blocks_per_request);
int assn_get_rings(assn_problem* p, int* staging, int* operand, int* kernel_matrix, int* blocks_per_request);

/* The tiling the next step will use (resolving automatic choices): tile cells, ring stages,
 * tensor-memory columns and dynamic shared memory per CTA.  Any output pointer may be NULL. */
int assn_get_tiling(assn_problem* p, int* tile_cells, int* stages, int* tmem_cols, int64_t* smem_bytes);

/* The tensor-core variant (0, 1 or 2) the next step of p runs, resolving the automatic choice.
 * Requires quadrature, cross sections and K (else ASSN_ERR_STATE); ASSN_ERR_UNSUPPORTED for the
 * CUDA-core precisions. */
int assn_get_variant(assn_problem* p, int* variant);

/* Device layout of the state: *Qpad = padded ordinate stride, *elem_bytes = 4 or 8. */
int assn_layout(const assn_problem* p, int* Qpad, int* elem_bytes);

/* Device pointer to the current state buffer ([ny][nx][Qpad]); valid until the next
 * assn_step / set_state / destroy. */
int assn_state_device(assn_problem* p, void** psi_dev);

/* Scalar flux Phi = sum_q w_q psi_q per cell (Eq. for Phi, Sec. 2.2), [ny][nx].
 * assn_scalar_flux copies FP64 to the host and syncs; assn_scalar_flux_device writes FP32
 * to a caller-owned device buffer, asynchronously. */
int assn_scalar_flux(assn_problem* p, double* phi_host);
int assn_scalar_flux_device(assn_problem* p, float* phi_dev);

/* Total particle number h^2 sum_cells sum_q w_q psi_q, accumulated in FP64.  Syncs. */
int assn_mass(assn_problem* p, double* mass_out);

/* Check the state for NaN/Inf: ASSN_OK or ASSN_ERR_NONFINITE.  Syncs. */
int assn_check_finite(assn_problem* p);

/* Out-of-bounds write check (a debugging aid; the method has no counterpart).  Each of the two
 * state buffers sits between two 4096-byte guard regions filled with 0xA5 when the state is
 * allocated.  Writes *guard_bytes_changed = the guard bytes that no longer hold 0xA5, and
 * *padding_nonzero = the padded ordinates (Q <= q < Qpad, both buffers) whose bits are not all
 * zero; both are 0 while every kernel has kept to its cells and ordinates.  Syncs.
 * Errors: ASSN_ERR_ARG on NULL, ASSN_ERR_STATE before a quadrature is set. */
int assn_check_guards(assn_problem* p, int64_t* guard_bytes_changed, int64_t* padding_nonzero);

/* ---- Batches: several problems stepped by one persistent launch per step.
 * The members may differ in grid size, quadrature (ordinate count), kernel width eps, cross
 * sections and dt; they share the device and one tensor-core precision (ASSN_BF16 or
 * ASSN_BF16X3; ASSN_TF32 or ASSN_BF16X2 when every member has 193..256 or 449..512 ordinates and
 * the grouping is per class, so that each runs on the paired-SM kernel) and one explicit scheme (assn_set_scheme: forward-Euler upwind, or the paper's Heun +
 * minmod of Sec. 3.1).  Each launch applies the same explicit step as assn_step (Sec. 3.2, forward
 * Euler of the as-S_N equations; for Heun + minmod one of the two stages of a Heun step, so a step
 * is two launches) to every member that still has steps left; a member's step count is
 * kept on the device, so members finish at their own counts within one run.  After
 * assn_batch_run each member is exactly as if assn_step(p, nsteps, dt) had been called on it,
 * bitwise.  With one class per padded ordinate count (the default grouping) a member whose steps run
 * on the paired-SM kernel (variant 2, automatic or set) is stepped by its own launches of that
 * kernel inside the batch's sequence (and graph); the other members run the persistent one-CTA
 * kernel, one launch per class and step, and equal assn_step with tiling variant 0 at the class's
 * tile width.  Members stay owned by the caller and must outlive their membership; while in a
 * batch they are stepped only through it.
 *
 * create:     stream = a cudaStream_t or NULL (library stream).  Errors: ASSN_ERR_CUDA / OOM.
 * add:        add p, to be advanced nsteps >= 0 steps of size dt per run.  Checks p is complete
 *             and dt admissible (as assn_step).  Errors: ASSN_ERR_ARG (NULL, duplicate, other
 *             device, mixed precision or scheme, more than 1024 members), ASSN_ERR_UNSUPPORTED (not a
 *             tensor-core precision, a TF32 / BF16X2 member without a paired-SM form, the implicit
 *             scheme), or p's own error
 *             (ASSN_ERR_STATE, ASSN_ERR_UNSTABLE).
 * set_steps:  change a member's nsteps / dt for later runs.
 * remove:     drop a member (syncs the batch stream).
 * set_tiling: tile cells (0, 32, 64, 128, 256) and ring depth (0 or 2..8) for all members.
 * autotune:   per class, time one launch of every candidate tiling (tile widths x ring shapes) on the
 *             members' current states (outputs go to scratch buffers, no state changes; syncs) and
 *             apply the fastest; the outputs describe the class with the most ordinates (*stages =
 *             its kernel-matrix ring depth), *ms_per_launch sums the classes.  With
 *             use_cache != 0 a previous result for the same precision and multiset of
 *             (cells, padded Q) is reused without timing (*ms_per_launch = -1 then).
 * Members are grouped into classes by padded ordinate count (Q rounded up to a multiple of 64):
 * each class has its own persistent launch per step and its own tile width (wide tiles for few
 * ordinates), so a step of the batch is one launch per class.
 * run:        enqueue, for each class, max nsteps of its members launches (twice that for Heun +
 *             minmod) on the batch stream
 *             (ordered after each member's stream; members' streams wait for the run).
 *             use_graph != 0 captures them once as a CUDA graph and replays it while the
 *             membership, tiling, dt and the classes' max nsteps stay the same.  Asynchronous.
 * sync:       wait for the batch stream; ASSN_ERR_TIMEOUT if a bounded device wait gave up.
 * info:       members, tile cells and stages of the class with the most ordinates, tiles per step
 *             summed over classes, launches issued (outputs may be NULL).
 * classes / class_info: number of classes; for class k (0 = most ordinates) its padded ordinate
 *             count, members, tile cells, stages and tiles per launch.
 * last_error: message of the last failure on b (b == NULL: last failed create on this thread). */
typedef struct assn_batch assn_batch;
int assn_batch_create(assn_batch** out, void* stream);
int assn_batch_destroy(assn_batch* b);
int assn_batch_add(assn_batch* b, assn_problem* p, int nsteps, double dt);
int assn_batch_set_steps(assn_batch* b, assn_problem* p, int nsteps, double dt);
int assn_batch_remove(assn_batch* b, assn_problem* p);
int assn_batch_set_tiling(assn_batch* b, int tile_cells, int stages);
/* Grouping of the members into launches: one_launch = 0 (default) one class, and one persistent
 * launch per step, for each padded ordinate count, each at the tile width that suits it;
 * one_launch = 1 every member in a single class, so each step (Heun: stage) of the whole batch is
 * one launch, with ordinate strides read per member and the tile width of the largest ordinate
 * count (every member on the one-CTA kernel).  Results of one-CTA members are the same either way
 * (bitwise, at equal tile widths).  ASSN_ERR_ARG for other values. */
int assn_batch_set_grouping(assn_batch* b, int one_launch);
int assn_batch_autotune(assn_batch* b, int use_cache, int* tile_cells, int* stages, double* ms_per_launch);
int assn_batch_run(assn_batch* b, int use_graph);
int assn_batch_sync(assn_batch* b);
int assn_batch_info(assn_batch* b, int* members, int* tile_cells, int* stages, int* total_tiles,
                    int64_t* launches);
int assn_batch_classes(assn_batch* b, int* nclass);
int assn_batch_class_info(assn_batch* b, int k, int* ordinate_stride, int* members, int* tile_cells, int* stages,
                          int* tiles);
const char* assn_batch_last_error(const assn_batch* b);

/* Autotune one problem's tiling for step size dt the same way (no state change; syncs) and apply
 * it (tile width and rings, as assn_set_tiling + assn_set_rings would); *stages receives the
 * kernel-matrix ring depth.  Outputs may be NULL. */
int assn_autotune(assn_problem* p, double dt, int use_cache, int* tile_cells, int* stages, double* ms_per_step);

/* ---- Serving: a request loop over whole solves (continuous batching).
 * A server owns one host thread that does all device work.  Requests (one complete as-S_N solve
 * each: grid, product quadrature, eps, cross sections, initial state, nsteps steps of size dt)
 * wait in arrival order and are admitted while fewer than max_active solves are on the device
 * and the estimated device memory of the admitted solves (assn_footprint_bytes) stays within
 * the budget; an admitted solve keeps its flux state on the device until it finishes.  The loop
 * advances all admitted solves together, chunk_steps steps at a time, with one persistent launch
 * per step (the batch path, optionally as CUDA graphs); requests that arrive meanwhile join at
 * the next chunk, and finished solves return the scalar flux Phi = sum_q w_q psi_q (FP64 on the
 * host, [ny][nx]) and free their memory.  A solve's result does not depend on which other solves
 * share its launches (each is bitwise equal to assn_step on the same problem with its default
 * tiling).
 *
 * Thread safety: submit, wait and stats may be called from any host threads concurrently;
 * assn_server_last_error returns the message of the calling thread's last failed server call. */
typedef enum {
    ASSN_INIT_LINE_SOURCE = 0,   /* assn_init_line_source(delta, floor_value) (Sec. 4.1)   */
    ASSN_INIT_ZERO = 1,          /* psi = 0                                                 */
    ASSN_INIT_STATE = 2          /* psi0: [ny][nx][Q] host FP32, copied at submit            */
} assn_init_kind;

typedef struct {
    int nx, ny;                          /* grid (square cells, as assn_create)               */
    double x0, x1, y0, y1;
    int n_polar, n_azim;                 /* product quadrature, Q = n_polar * n_azim <= 1024 */
    double sigma_as, eps;                /* artificial scattering (assn_set_artificial_scattering) */
    int kernel_kind, normalisation;
    const double* sigma_a;               /* [ny][nx] host, copied at submit                  */
    const double* sigma_s;
    const double* q;
    int init_kind;                       /* an assn_init_kind                                 */
    double delta, floor_value;           /* ASSN_INIT_LINE_SOURCE parameters                  */
    const float* psi0;                   /* ASSN_INIT_STATE state                             */
    int nsteps;                          /* steps of size dt (checked against the positivity  */
    double dt;                           /* bound at admission: the request then fails)       */
} assn_request;

typedef struct {
    int64_t submitted, completed, failed, active, queued, max_active_seen, launches;
    double p50_latency_s, p99_latency_s, mean_latency_s;   /* submit -> result, completed solves */
    double busy_s;                       /* host time spent in chunks with solves on the device */
    double wall_s;                       /* first submit -> last completion                   */
    double updates;                      /* cell-ordinate updates of completed solves         */
    double updates_per_s;                /* updates / wall_s                                   */
    int64_t budget_bytes, peak_bytes;    /* footprint budget and the largest admitted total   */
} assn_server_stats;

typedef struct assn_server assn_server;

/* Estimated device memory of one problem (state ping-pong, cell constants, K and its operands,
 * staging), rounded up to 2 MiB.  ASSN_ERR_ARG on invalid sizes. */
int assn_footprint_bytes(int nx, int ny, int Q, int precision, size_t* bytes);

/* precision: ASSN_BF16 or ASSN_BF16X3.  hbm_budget_bytes: admission budget (0 = 85% of the
 * device memory free at creation).  max_active: 1..1024 solves on the device at once.
 * chunk_steps >= 1: steps per admission round.  use_graph: replay chunks as CUDA graphs. */
int assn_server_create(assn_server** out, int precision, size_t hbm_budget_bytes, int max_active,
                       int chunk_steps, int use_graph);
/* Queue a request (inputs copied); *id receives its handle.  ASSN_ERR_ARG on an invalid request,
 * ASSN_ERR_OOM if its footprint exceeds the whole budget, ASSN_ERR_STATE while stopping. */
int assn_server_submit(assn_server* s, const assn_request* r, int64_t* id);
/* Wait for request id (timeout_s < 0: no limit), then release it: phi_host[ny*nx] receives the
 * scalar flux (may be NULL), *latency_s the submit-to-result time, *queue_s the time before
 * admission.  Returns the request's status (e.g. ASSN_ERR_UNSTABLE for an inadmissible dt),
 * ASSN_ERR_TIMEOUT if not finished in time (the request stays pending), ASSN_ERR_ARG for an
 * unknown id. */
int assn_server_wait(assn_server* s, int64_t id, double timeout_s, double* phi_host, double* latency_s,
                     double* queue_s);

/* Cancel request `id`.  A request still queued leaves the queue at once; one already on the device
 * is retired at the loop's next chunk boundary (its memory freed; a solve that reaches its last step
 * in the chunk running when the call is made completes normally instead).  assn_server_wait then
 * returns ASSN_ERR_CANCELLED for it, and the statistics count it as failed.  The other requests'
 * results are unaffected (each equals its own solve alone).  Errors: ASSN_ERR_ARG for an unknown id,
 * ASSN_ERR_STATE if the request has already finished. */
int assn_server_cancel(assn_server* s, int64_t id);

int assn_server_get_stats(assn_server* s, assn_server_stats* out);
/* Finish every queued and admitted request, stop the loop and free the server.  Results not
 * collected by assn_server_wait are dropped. */
int assn_server_destroy(assn_server* s);
const char* assn_server_last_error(void);

/* ---- Allocation-free total mass (the paper has no counterpart; this serves library users).
 * Some callers cannot allocate device memory during a call: real-time loops whose latency budget
 * rules out allocator calls (cudaMalloc may block and synchronise the device), and hosts that run
 * the library inside a memory pool they manage and account for themselves, handing it only the
 * buffers they own.  The paper has no counterpart; this is a service of the library.
 * assn_mass_noalloc computes h^2 sum_cells sum_q w_q psi_q of a
 * caller-owned device state without allocating anything: its partial sums go to a fixed
 * file-scope device array of ASSN_NOALLOC_MASS_MAX_BLOCKS doubles (128 KB), one per 256 cells,
 * which every device that loads the library holds until process exit.
 *   psi_dev    [ncell][Qp] state on the current device, FP32 (elem_bytes 4) or FP64 (8)
 *   w_dev      [Qp] FP64 quadrature weights on the device (0 on padded ordinates)
 *   mass_dev   one FP64 result on the device, written asynchronously on `stream`
 * Errors: ASSN_ERR_ARG for NULL pointers, elem_bytes not 4 or 8, ncell > ASSN_NOALLOC_MASS_MAX_CELLS
 * or Qp > ASSN_MAX_Q; ASSN_ERR_CUDA if the launch fails (message in assn_noalloc_last_error()).
 * The first call on a device looks up the scratch array's device address (with that device
 * current); later calls on that device reuse it.  Every call shares the scratch array and
 * overwrites it completely before reading it; calls whose work overlaps on one device race, so
 * serialise them (same stream, or events). */
#define ASSN_NOALLOC_MASS_CELLS_PER_BLOCK 256
#define ASSN_NOALLOC_MASS_MAX_BLOCKS 16384
#define ASSN_NOALLOC_MASS_MAX_CELLS (ASSN_NOALLOC_MASS_CELLS_PER_BLOCK * ASSN_NOALLOC_MASS_MAX_BLOCKS)
int assn_mass_noalloc(const void* psi_dev, int elem_bytes, const double* w_dev, int ncell, int Qp,
                      double h, double* mass_dev, void* stream);
const char* assn_noalloc_last_error(void);

/* Self-test of the failure path of the tensor-core kernels on the current device: launches one
 * block whose bounded wait on an mbarrier that nothing completes gives up after limit_us
 * microseconds (1 .. 1e6), records the event in a device flag and returns; the host reads the flag.
 * Returns ASSN_ERR_TIMEOUT when the wait gave up as designed (the CUDA context stays usable),
 * ASSN_ERR_ARG for a limit out of range, ASSN_ERR_CUDA / ASSN_ERR_OOM if the check itself failed. */
int assn_selftest_wait_timeout(int limit_us);

/* Message of the last failure on p (never NULL; "" when none).  With p == NULL, the last
 * failure of assn_create on this thread. */
const char* assn_last_error(const assn_problem* p);

/* Static name of a status code. */
const char* assn_status_string(int status);

/* Number of kernel launches this problem has issued so far (for launch accounting). */
int64_t assn_launch_count(const assn_problem* p);

int assn_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ASSN_H */

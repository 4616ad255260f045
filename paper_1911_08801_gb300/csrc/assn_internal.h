// Internal definitions shared by the translation units of libassn (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/assn.h"

namespace assn {

// Per-ordinate constants of one step (transport part depends on dt).
//   nux = dt * Omega_x / h, nuy = dt * Omega_y / h   (signed: the sign picks the upwind side)
//   w   = quadrature weight (0 on padded ordinates)
//   e   = out-scattering rate of the artificial generator: 1 - K_qq evaluated from the
//         rounded off-diagonal operand so that the chosen normalisation's invariant holds
//         exactly for the operand the contraction actually uses.
struct OrdF { float nux, nuy, w, e; };
struct OrdD { double nux, nuy, w, e; };

// Per-cell constants: sigma_t = sigma_a + sigma_s, sigma_s / sum_q w_q, q, unused.
struct CellF { float sig_t, sig_s_over_wsum, q, pad; };
struct CellD { double sig_t, sig_s_over_wsum, q, pad; };

// Arguments of one fused step launch.
template <typename T, typename OrdT, typename CellT>
struct StepArgs {
    const T* psi;        // [ny][nx][Qp], time level n
    T* psi_out;          // [ny][nx][Qp], time level n+1
    const OrdT* ord;     // [Qp]
    const CellT* cell;   // [ny][nx]
    const T* KT;         // SIMT paths: [Qp][Qp], KT[p*Qp + q] = K_qp for p != q, 0 on the diagonal
    int nx, ny, Q, Qp;
    T dt, dt_sigma_as;
};

// Tensor-core operands of the BF16 and TF32 paths.
struct TcOperands {
    __nv_bfloat16* G_hi = nullptr;   // [Mp][Qp] row q, column p: off-diagonal K rounded to BF16
    __nv_bfloat16* G_lo = nullptr;   // [Mp][Qp] residual K - G_hi rounded to BF16 (BF16X3 only)
    float* G32 = nullptr;            // [Mp][Qp] off-diagonal K rounded to TF32 (ASSN_TF32 only)
    int Mp = 0;                      // Q rounded up to 128 (the MMA M dimension)
};

// FP32 -> TF32 (sign, exponent, 10 significand bits): round to nearest, ties away from zero, by
// adding half a unit of the last kept bit to the magnitude and clearing the 13 bits below it (an
// overflowing magnitude carries into the exponent, which is the correctly rounded result).  Finite
// inputs; the word is what the contraction reads, its low 13 bits zero.
__device__ __forceinline__ uint32_t tf32_bits(float v) { return (__float_as_uint(v) + 0x1000u) & 0xffffe000u; }
__device__ __forceinline__ float tf32_round(float v) { return __uint_as_float(tf32_bits(v)); }

// Launchers (each returns cudaSuccess or the launch error).
cudaError_t launch_build_K(const double* omega, const double* w, int Q, double eps, int kind,
                           int norm, double* K64, cudaStream_t s);
cudaError_t launch_derive_simt_f64(const double* K64, const double* w, int Q, int Qp, int norm,
                                   double* KT, double* e, cudaStream_t s);
cudaError_t launch_derive_simt_f32(const double* K64, const double* w, int Q, int Qp, int norm,
                                   float* KT, double* e, cudaStream_t s);
cudaError_t launch_derive_tc(const double* K64, const double* w, int Q, int Qp, int Mp, int norm,
                             bool split, __nv_bfloat16* G_hi, __nv_bfloat16* G_lo, double* e,
                             cudaStream_t s);
// The TF32 operand: G32[q][p] = tf32_round((float) K_qp) off the diagonal, zero elsewhere, and the
// generator diagonal e from those values.
cudaError_t launch_derive_tf32(const double* K64, const double* w, int Q, int Qp, int Mp, int norm, float* G32,
                               double* e, cudaStream_t s);

cudaError_t launch_step_simt_f64(const StepArgs<double, OrdD, CellD>& a, cudaStream_t s);
cudaError_t launch_step_simt_f32(const StepArgs<float, OrdF, CellF>& a, cudaStream_t s);
// One stage of Heun's method with minmod-limited second-order upwind transport (CUDA cores):
// psi_out = alpha keep + beta (psi + dt L(psi)); keep may be psi_out itself (each element is read
// before it is written by the same thread) and is not read when alpha == 0.
cudaError_t launch_stage_simt_f64(const StepArgs<double, OrdD, CellD>& a, const double* keep, double alpha,
                                  double beta, cudaStream_t s);
cudaError_t launch_stage_simt_f32(const StepArgs<float, OrdF, CellF>& a, const float* keep, float alpha,
                                  float beta, cudaStream_t s);

// Tensor-core step.  Returns cudaErrorNotSupported for shapes the kernel does not cover.
struct TcPlan;
cudaError_t tc_plan_create(TcPlan** plan, const __nv_bfloat16* G_hi, const __nv_bfloat16* G_lo,
                           int Q, int Qp, int Mp, int nx, int ny, bool split, int want_nt, int want_stages);
void tc_plan_describe(const TcPlan* plan, int* tile_cells, int* stages, int* tmem_cols, size_t* smem);
void tc_plan_destroy(TcPlan* plan);
cudaError_t launch_step_tc(TcPlan* plan, const StepArgs<float, OrdF, CellF>& a, const float* w,
                           unsigned int* err_flag, cudaStream_t s);

// Persistent warp-specialised tensor-core step (the default tensor-core kernel), for one problem
// or a batch.  Each problem's flux buffer parity and activity come from a device step counter that
// the launch advances for the problems it stepped.
struct Tc2Problem {
    const float* buf[2];            // the problem's two FP32 flux buffers [ncell][Qp]
    const OrdF* ord;                // [Qp] per-ordinate constants for dt
    const CellF* cell;              // [ncell]
    const float* w;                 // [Qp]
    const __nv_bfloat16* G_hi;      // [Mp][Qp]
    const __nv_bfloat16* G_lo;      // [Mp][Qp] (BF16X3) or null
    int* counter;                   // device step counter
    int target;                     // stepped while counter < target
    int nx, ny, Q, Qp, Mp;
    float dt, dt_sigma_as;
};
// Ring request of the persistent kernel: staging (FP32 flux chunks), operand (BF16 B chunks) and
// kernel-matrix ring depths, and ordinate blocks per kernel-matrix request; 0 = automatic.
struct TcRings {
    int SS = 0, SB = 0, SA = 0, MPR = 0;
};
struct Tc2Plan;
cudaError_t tc2_plan_create(Tc2Plan** plan, const Tc2Problem* probs, int nprob, bool split, int want_nt,
                            TcRings rings);
void tc2_plan_destroy(Tc2Plan* plan);
void tc2_plan_describe(const Tc2Plan* plan, int* tile_cells, int* stages, int* tmem_cols, size_t* smem);
TcRings tc2_plan_rings(const Tc2Plan* plan);
int tc2_plan_total_tiles(const Tc2Plan* plan);
// New step targets (one per problem, in plan order) for later launches on `s`.
cudaError_t tc2_plan_set_targets(Tc2Plan* plan, const int* targets, cudaStream_t s);
// parity0 >= 0 (one-problem plans launched by the host step by step): problem 0's counter parity
// at launch, so the flux is read from buffer parity0 and written to parity0 ^ 1; parity0 < 0:
// every parity comes from the device counters (batches, CUDA graphs).
cudaError_t launch_step_tc2(Tc2Plan* plan, unsigned int* err_flag, int parity0, cudaStream_t s);
// One Heun stage with minmod-limited second-order transport.  parity0 >= 0 (one-problem plan): reads
// buffer parity0, writes alpha keep + beta (psi + dt L(psi)) to buffer parity0 ^ 1 (keep may be that
// buffer; not read when alpha == 0).  parity0 < 0 (any plan): every problem's buffers and stage come
// from its device counter (stage 2 when the counter's parity differs from its target's, keeping psi^n
// from the buffer it writes); keep, alpha and beta are ignored.
cudaError_t launch_heun_stage_tc2(Tc2Plan* plan, unsigned int* err_flag, int parity0, const float* keep, float alpha,
                                  float beta, cudaStream_t s);

// Paired-SM tensor-core step (variant 2): one problem, forward Euler or a Heun stage, BF16, BF16X3
// or TF32, padded ordinate count 256 or 512 (equal to the kernel-matrix rows).  A cluster of two CTAs
// shares each M = 256 MMA; the flux buffers and G are bound at plan creation, dt at launch.
struct Tc3Plan;
bool tc3_supported(int Q, int Qp, int Mp, bool split);
// precision: ASSN_BF16 (ops.G_hi), ASSN_BF16X3 (ops.G_hi and ops.G_lo: the split contraction
// hi x hi + hi x lo + lo x hi) or ASSN_TF32 (ops.G32); else cudaErrorInvalidValue.  With no
// kernel-matrix ring requested (want.SA == 0) and BF16, G is read back on `stream` (which syncs;
// skipped while the stream is being captured) to find its distinct blocks, which stay resident if
// they fit.
cudaError_t tc3_plan_create(Tc3Plan** plan, const float* buf0, const float* buf1, const TcOperands& ops,
                            int precision, int Q, int Qp, int Mp, int nx, int ny, TcRings want, cudaStream_t stream);
void tc3_plan_destroy(Tc3Plan* plan);
// MPR = 64-ordinate chunks per stage; SA = kernel-matrix ring depth, 0 when the matrix is resident
TcRings tc3_plan_rings(const Tc3Plan* plan);
// tile cells, kernel-matrix ring depth, CTA pairs launched, dynamic shared memory per CTA
void tc3_plan_describe(const Tc3Plan* plan, int* tile_cells, int* stages, int* pairs, size_t* smem);
// Reads buffer `parity`, writes buffer parity ^ 1.
cudaError_t launch_step_tc3(const Tc3Plan* plan, int parity, const OrdF* ord, const CellF* cell, const float* w,
                            float dt, float dt_sigma_as, unsigned int* err_flag, cudaStream_t s);
// The forward-Euler step of launch_step_tc3 between caller-owned buffers of the plan's layout
// ([ny][nx][Qp] FP32; in 16-byte aligned for the tensor copies, else cudaErrorInvalidValue).
cudaError_t launch_step_tc3_buffers(const Tc3Plan* p, const float* in, float* out, const OrdF* ord,
                                    const CellF* cell, const float* w, float dt, float dt_sigma_as,
                                    unsigned int* err_flag, cudaStream_t s);
// One Heun stage (Sec. 3.1) on the paired-SM kernel: reads buffer `parity`, writes buffer parity ^ 1
// = alpha keep + beta (in + dt L(in)) with the minmod-limited second-order upwind transport.
cudaError_t launch_heun_stage_tc3(const Tc3Plan* p, int parity, const OrdF* ord, const CellF* cell, const float* w,
                                  float dt, float dt_sigma_as, const float* keep, float alpha, float beta,
                                  unsigned int* err_flag, cudaStream_t s);

template <typename T>
cudaError_t launch_scalar_flux(const T* psi, const T* w, int ncell, int Qp, float* out_f,
                               double* out_d, cudaStream_t s);
template <typename T>
cudaError_t launch_mass_partials(const T* psi, const T* w, int ncell, int Qp, double* partials,
                                 int nblocks, cudaStream_t s);
cudaError_t launch_reduce_partials(const double* partials, int n, double* out, cudaStream_t s);
template <typename T>
cudaError_t launch_check_finite(const T* psi, size_t n, unsigned int* flag, cudaStream_t s);
template <typename T>
cudaError_t launch_padding_nonzero(const T* psi, size_t ncell, int Q, int Qp, unsigned long long* count,
                                   cudaStream_t s);
template <typename T>
cudaError_t launch_init_line_source(T* psi, int nx, int ny, int Q, int Qp, double x0, double y0,
                                    double h, double delta, double floor_value, cudaStream_t s);
template <typename T>
cudaError_t launch_pack_state(const double* src, T* dst, size_t ncell, int Q, int Qp, cudaStream_t s);
template <typename T>
cudaError_t launch_unpack_state(const T* src, double* dst, size_t ncell, int Q, int Qp, cudaStream_t s);

constexpr int kMassBlocks = 1024;

}  // namespace assn

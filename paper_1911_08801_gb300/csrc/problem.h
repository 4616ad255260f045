// Problem object shared by the host-side translation units of libassn (not part of the ABI).
#pragma once

#include <string>
#include <vector>

#include "assn_internal.h"

namespace assn {
struct ImplicitWork;
}

struct assn_problem {
    int dev = 0;
    int nx = 0, ny = 0;
    double x0 = 0, x1 = 0, y0 = 0, y1 = 0, h = 0;
    int precision = ASSN_FP32;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    int Q = 0, Qp = 0;
    std::vector<double> omega, w;   // host copies, [Q*3], [Q]
    double wsum = 0;
    bool have_quad = false;

    std::vector<double> sa, ss, src;
    bool have_xs = false;

    double sigma_as = 0, eps = 0;
    int kind = 0, norm = 0;
    bool have_K = false;
    std::vector<double> e;          // generator diagonal per ordinate

    // device memory
    double* d_omega = nullptr;
    double* d_w64 = nullptr;
    float* d_w32 = nullptr;
    double* d_K64 = nullptr;
    double* d_KT64 = nullptr;
    float* d_KT32 = nullptr;
    assn::TcOperands tc;
    assn::TcPlan* plan = nullptr;      // one-tile-per-CTA tensor-core kernel (variant 1)
    assn::Tc2Plan* plan2 = nullptr;    // persistent warp-specialised kernel (variant 0, default)
    assn::Tc3Plan* plan3 = nullptr;    // paired-SM kernel (variant 2)
    int variant = -1;                  // -1: automatic (2 where it applies, else 0)
    double* d_e = nullptr;
    void* d_ord = nullptr;
    double ord_dt = -1.0;
    void* d_cell = nullptr;
    void* d_psi[2] = {nullptr, nullptr};
    // each state buffer sits between two guard regions of kStateGuard bytes holding kGuardByte (the
    // allocation starts at d_psi_raw[b]); assn_check_guards reads them back
    unsigned char* d_psi_raw[2] = {nullptr, nullptr};
    int cur = 0;
    double* d_partials = nullptr;
    double* d_scalar = nullptr;
    unsigned int* d_flags = nullptr;   // [0] finite check, [1] tensor-core timeout
    double* d_stage = nullptr;
    size_t stage_elems = 0;

    int scheme = 0;                     // an assn_scheme
    int want_nt = 0, want_stages = 0;   // tensor-core tiling request (0 = automatic)
    assn::TcRings want_rings;           // persistent kernel's rings (zero fields automatic)
    int* d_counter = nullptr;           // device step counter of the persistent tensor-core kernel
    int counter_host = 0;               // last value written to / advanced on d_counter
    double plan2_dt = -1.0;             // dt the persistent plan was built for
    assn::ImplicitWork* impl = nullptr; // implicit scheme's work space and parameters (lazy)

    std::string err;
    int64_t launches = 0;

    size_t ncell() const { return (size_t)nx * ny; }
    size_t elem() const { return precision == ASSN_FP64 ? 8 : 4; }
    bool tensor() const {
        return precision == ASSN_BF16 || precision == ASSN_BF16X3 || precision == ASSN_TF32 || precision == ASSN_BF16X2;
    }
    // precisions with a paired-SM form only (no one-CTA or tile-per-CTA kernel)
    bool paired_only() const { return precision == ASSN_TF32 || precision == ASSN_BF16X2; }
};

namespace assn {

// Frees the implicit scheme's work space (NULL is a no-op).
void implicit_free(ImplicitWork* W);
// nsteps implicit sweeping-Krylov steps of size dt (FP64 / FP32 problems).
int implicit_steps(assn_problem* p, int nsteps, double dt);

// Set p's error message; returns status.
int problem_fail(assn_problem* p, int status, const char* msg);
// Checks that p is complete and dt admissible, uploads the per-ordinate constants for dt.
int problem_prepare(assn_problem* p, double dt);
// Reads and clears the device-wait timeout flag of p (synchronises p's stream).
int problem_check_flags(assn_problem* p);
// Description of p for the persistent tensor-core kernel: buffers, constants, step counter,
// stepped while the counter is below target.
Tc2Problem problem_tc2(const assn_problem* p, double dt, int target);
// True when p's steps run on the paired-SM kernel (the variant its own steps resolve to is 2).
bool problem_paired(const assn_problem* p);
// True when p's ordinate count has a paired-SM form (193..256 or 449..512 ordinates).
bool problem_pair_supported(const assn_problem* p);
// Creates p's paired-SM plan if missing (reads G back once: not while a stream is being captured).
int problem_pair_plan(assn_problem* p, double dt);
// Enqueues one launch of p's paired-SM kernel on stream s at step size dt: a forward-Euler step, or
// a Heun stage (stage 0: psi* from buffer `parity`; stage 1: psi^{n+1} into buffer parity ^ 1 from
// psi* in buffer `parity`, keeping psi^n there).  Errors go to err_flag.
cudaError_t problem_pair_launch(assn_problem* p, double dt, int parity, int heun_stage, unsigned int* err_flag,
                                cudaStream_t s);

}  // namespace assn

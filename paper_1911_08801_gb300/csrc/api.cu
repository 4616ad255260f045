// Host side of libassn: problem object, argument checks, device memory, dispatch.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "problem.h"
#include "trace.h"

using namespace assn;

namespace {

thread_local std::string g_create_error;

int fail(assn_problem* p, int status, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(assn_problem* p, int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (p) p->err = buf; else g_create_error = buf;
    return status;
}

#define CK(p, call)                                                                                    \
    do {                                                                                               \
        cudaError_t _e = (call);                                                                       \
        if (_e != cudaSuccess)                                                                         \
            return fail((p), _e == cudaErrorMemoryAllocation ? ASSN_ERR_OOM : ASSN_ERR_CUDA, "%s: %s", \
                        #call, cudaGetErrorString(_e));                                                \
    } while (0)

template <typename T>
void dfree(T*& ptr) {
    if (ptr) cudaFree((void*)ptr);
    ptr = nullptr;
}

int set_device(assn_problem* p) {
    CK(p, cudaSetDevice(p->dev));
    return ASSN_OK;
}

// Gauss-Legendre nodes and weights on [-1,1] by Newton iteration on P_n with the three-term
// recurrence, starting from the Chebyshev-like guess cos(pi (i + 3/4)/(n + 1/2)).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
    x.assign(n, 0.0);
    wt.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        wt[i] = wt[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

void free_operands(assn_problem* p) {
    dfree(p->d_K64);
    dfree(p->d_KT64);
    dfree(p->d_KT32);
    dfree(p->tc.G_hi);
    dfree(p->tc.G_lo);
    dfree(p->tc.G32);
    dfree(p->d_e);
    if (p->plan) tc_plan_destroy(p->plan);
    p->plan = nullptr;
    if (p->plan2) tc2_plan_destroy(p->plan2);
    p->plan2 = nullptr;
    if (p->plan3) tc3_plan_destroy(p->plan3);
    p->plan3 = nullptr;
    p->have_K = false;
}

int ensure_stage(assn_problem* p, size_t elems) {
    if (p->stage_elems >= elems) return ASSN_OK;
    dfree(p->d_stage);
    p->stage_elems = 0;
    CK(p, cudaMalloc(&p->d_stage, elems * sizeof(double)));
    p->stage_elems = elems;
    return ASSN_OK;
}

constexpr size_t kStateGuard = 4096;        // bytes before and after each state buffer
constexpr unsigned char kGuardByte = 0xA5;

int alloc_state(assn_problem* p) {
    const size_t bytes = p->ncell() * p->Qp * p->elem();
    for (int b = 0; b < 2; ++b) {
        dfree(p->d_psi_raw[b]);
        p->d_psi[b] = nullptr;
        CK(p, cudaMalloc(&p->d_psi_raw[b], bytes + 2 * kStateGuard));
        p->d_psi[b] = p->d_psi_raw[b] + kStateGuard;
        CK(p, cudaMemsetAsync(p->d_psi_raw[b], kGuardByte, kStateGuard, p->stream));
        CK(p, cudaMemsetAsync(p->d_psi_raw[b] + kStateGuard + bytes, kGuardByte, kStateGuard, p->stream));
        CK(p, cudaMemsetAsync(p->d_psi[b], 0, bytes, p->stream));
    }
    p->cur = 0;
    return ASSN_OK;
}

int check_flags(assn_problem* p) {
    unsigned int f[2] = {0, 0};
    CK(p, cudaMemcpyAsync(f, p->d_flags, sizeof f, cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    if (f[1]) {
        CK(p, cudaMemsetAsync(p->d_flags + 1, 0, sizeof(unsigned int), p->stream));
        return fail(p, ASSN_ERR_TIMEOUT, "a bounded device wait gave up (flag 0x%x)%s", f[1],
                    (f[1] & 0x80000000u) ? "; work in flight did not drain, treat the CUDA context as suspect" : "");
    }
    return ASSN_OK;
}

// Per-ordinate constants for step size dt.
int upload_ord(assn_problem* p, double dt) {
    if (p->ord_dt == dt && p->d_ord) return ASSN_OK;
    const int Qp = p->Qp;
    if (!p->d_ord) {
        CK(p, cudaMalloc(&p->d_ord, sizeof(OrdD) * Qp));
    }
    if (p->precision == ASSN_FP64) {
        std::vector<OrdD> o(Qp, OrdD{0, 0, 0, 0});
        for (int q = 0; q < p->Q; ++q)
            o[q] = OrdD{dt * p->omega[3 * q] / p->h, dt * p->omega[3 * q + 1] / p->h, p->w[q], p->e[q]};
        CK(p, cudaMemcpyAsync(p->d_ord, o.data(), sizeof(OrdD) * Qp, cudaMemcpyHostToDevice, p->stream));
        CK(p, cudaStreamSynchronize(p->stream));
    } else {
        std::vector<OrdF> o(Qp, OrdF{0, 0, 0, 0});
        for (int q = 0; q < p->Q; ++q)
            o[q] = OrdF{(float)(dt * p->omega[3 * q] / p->h), (float)(dt * p->omega[3 * q + 1] / p->h),
                        (float)p->w[q], (float)p->e[q]};
        CK(p, cudaMemcpyAsync(p->d_ord, o.data(), sizeof(OrdF) * Qp, cudaMemcpyHostToDevice, p->stream));
        CK(p, cudaStreamSynchronize(p->stream));
    }
    p->ord_dt = dt;
    return ASSN_OK;
}

// Largest dt keeping the coefficient of psi_q in its own update non-negative (all other
// coefficients are non-negative): 1 - dt (|Omega_x| + |Omega_y|)/h - dt sigma_as e_q
// - dt (sigma_a + sigma_s) >= 0, maximised over ordinates and cells separately.
double max_stable_dt(const assn_problem* p) {
    if (p->scheme == ASSN_SCHEME_IMPLICIT) return INFINITY;   // implicit Euler: no step restriction
    if (p->scheme == ASSN_SCHEME_HEUN_MINMOD) {
        // Each forward-Euler stage of Heun's method stays a non-negative combination of old values:
        // with minmod slopes the upwind flux difference along an axis is (psi_i - psi_{i-1}) times a
        // factor in [1/2, 3/2], so the transport term takes at most 3/2 (|Omega_x| + |Omega_y|) dt / h
        // of psi_q.
        double vmax = 0, smax = 0;
        for (int q = 0; q < p->Q; ++q)
            vmax = std::max(vmax, 1.5 * (fabs(p->omega[3 * q]) + fabs(p->omega[3 * q + 1])) / p->h +
                                      p->sigma_as * p->e[q]);
        for (size_t c = 0; c < p->ncell(); ++c) smax = std::max(smax, p->sa[c] + p->ss[c]);
        const double rate = vmax + smax;
        return rate > 0 ? 1.0 / rate : INFINITY;
    }
    double vmax = 0;
    for (int q = 0; q < p->Q; ++q)
        vmax = std::max(vmax, (fabs(p->omega[3 * q]) + fabs(p->omega[3 * q + 1])) / p->h + p->sigma_as * p->e[q]);
    double smax = 0;
    for (size_t c = 0; c < p->ncell(); ++c) smax = std::max(smax, p->sa[c] + p->ss[c]);
    const double rate = vmax + smax;
    return rate > 0 ? 1.0 / rate : INFINITY;
}

int ready(assn_problem* p) {
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    if (!p->have_xs) return fail(p, ASSN_ERR_STATE, "no cross sections set");
    if (!p->have_K) return fail(p, ASSN_ERR_STATE, "artificial scattering (K) not set");
    return ASSN_OK;
}

int install_quadrature(assn_problem* p, int Q, const double* omega, const double* w) {
    free_operands(p);
    dfree(p->d_omega);
    dfree(p->d_w64);
    dfree(p->d_w32);
    dfree(p->d_ord);
    p->ord_dt = -1;
    p->Q = Q;
    p->Qp = (Q + 63) / 64 * 64;
    p->omega.assign(omega, omega + 3 * Q);
    p->w.assign(w, w + Q);
    p->wsum = 0;
    for (int q = 0; q < Q; ++q) p->wsum += w[q];
    std::vector<double> wp(p->Qp, 0.0);
    std::vector<float> wf(p->Qp, 0.0f);
    for (int q = 0; q < Q; ++q) { wp[q] = w[q]; wf[q] = (float)w[q]; }
    CK(p, cudaMalloc(&p->d_omega, sizeof(double) * 3 * Q));
    CK(p, cudaMalloc(&p->d_w64, sizeof(double) * p->Qp));
    CK(p, cudaMalloc(&p->d_w32, sizeof(float) * p->Qp));
    CK(p, cudaMemcpyAsync(p->d_omega, omega, sizeof(double) * 3 * Q, cudaMemcpyHostToDevice, p->stream));
    CK(p, cudaMemcpyAsync(p->d_w64, wp.data(), sizeof(double) * p->Qp, cudaMemcpyHostToDevice, p->stream));
    CK(p, cudaMemcpyAsync(p->d_w32, wf.data(), sizeof(float) * p->Qp, cudaMemcpyHostToDevice, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    int r = alloc_state(p);
    if (r) return r;
    p->have_quad = true;
    if (p->have_xs) {
        // per-cell constant sigma_s / sum w depends on the quadrature
        std::vector<double> sa = p->sa, ss = p->ss, src = p->src;
        r = assn_set_cross_sections(p, sa.data(), ss.data(), src.data());
        if (r) return r;
    }
    return ASSN_OK;
}

}  // namespace

namespace assn {

int problem_fail(assn_problem* p, int status, const char* msg) { return fail(p, status, "%s", msg); }

int problem_prepare(assn_problem* p, double dt);   // defined after the step entry points

int problem_check_flags(assn_problem* p) { return check_flags(p); }

Tc2Problem problem_tc2(const assn_problem* p, double dt, int target) {
    Tc2Problem d;
    d.buf[0] = (const float*)p->d_psi[0];
    d.buf[1] = (const float*)p->d_psi[1];
    d.ord = (const OrdF*)p->d_ord;
    d.cell = (const CellF*)p->d_cell;
    d.w = p->d_w32;
    d.G_hi = p->tc.G_hi;
    d.G_lo = p->tc.G_lo;
    d.counter = p->d_counter;
    d.target = target;
    d.nx = p->nx;
    d.ny = p->ny;
    d.Q = p->Q;
    d.Qp = p->Qp;
    d.Mp = p->tc.Mp;
    d.dt = (float)dt;
    d.dt_sigma_as = (float)(dt * p->sigma_as);
    return d;
}

}  // namespace assn

extern "C" {

int assn_abi_version(void) { return ASSN_ABI_VERSION; }

const char* assn_status_string(int s) {
    switch (s) {
        case ASSN_OK: return "ASSN_OK";
        case ASSN_ERR_ARG: return "ASSN_ERR_ARG";
        case ASSN_ERR_OOM: return "ASSN_ERR_OOM";
        case ASSN_ERR_CUDA: return "ASSN_ERR_CUDA";
        case ASSN_ERR_UNSTABLE: return "ASSN_ERR_UNSTABLE";
        case ASSN_ERR_NONFINITE: return "ASSN_ERR_NONFINITE";
        case ASSN_ERR_TIMEOUT: return "ASSN_ERR_TIMEOUT";
        case ASSN_ERR_STATE: return "ASSN_ERR_STATE";
        case ASSN_ERR_UNSUPPORTED: return "ASSN_ERR_UNSUPPORTED";
        case ASSN_ERR_CANCELLED: return "ASSN_ERR_CANCELLED";
        default: return "ASSN_ERR_UNKNOWN";
    }
}

const char* assn_last_error(const assn_problem* p) { return p ? p->err.c_str() : g_create_error.c_str(); }

int64_t assn_launch_count(const assn_problem* p) { return p ? p->launches : 0; }

int assn_create(assn_problem** out, int nx, int ny, double x0, double x1, double y0, double y1, int precision,
                void* stream) {
    if (!out) return fail(nullptr, ASSN_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nx > ASSN_MAX_SIDE || ny > ASSN_MAX_SIDE)
        return fail(nullptr, ASSN_ERR_ARG, "grid %d x %d out of range [1, %d]", nx, ny, ASSN_MAX_SIDE);
    if (!(x1 > x0) || !(y1 > y0)) return fail(nullptr, ASSN_ERR_ARG, "empty domain");
    const double hx = (x1 - x0) / nx, hy = (y1 - y0) / ny;
    if (fabs(hx - hy) > 1e-12 * hx) return fail(nullptr, ASSN_ERR_ARG, "cells must be square (hx=%g, hy=%g)", hx, hy);
    if (precision < ASSN_FP64 || precision > ASSN_BF16X2) return fail(nullptr, ASSN_ERR_ARG, "unknown precision %d", precision);
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return fail(nullptr, ASSN_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ce));
    assn_problem* p = new (std::nothrow) assn_problem();
    if (!p) return fail(nullptr, ASSN_ERR_OOM, "host allocation failed");
    p->dev = dev;
    p->nx = nx; p->ny = ny; p->x0 = x0; p->x1 = x1; p->y0 = y0; p->y1 = y1; p->h = hx;
    p->precision = precision;
    if (stream) {
        p->stream = (cudaStream_t)stream;
    } else {
        ce = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) { delete p; return fail(nullptr, ASSN_ERR_CUDA, "stream: %s", cudaGetErrorString(ce)); }
        p->own_stream = true;
    }
    int r = ASSN_OK;
    if ((ce = cudaMalloc(&p->d_cell, sizeof(CellD) * p->ncell())) != cudaSuccess ||
        (ce = cudaMalloc(&p->d_partials, sizeof(double) * kMassBlocks)) != cudaSuccess ||
        (ce = cudaMalloc(&p->d_scalar, sizeof(double))) != cudaSuccess ||
        (ce = cudaMalloc(&p->d_flags, 2 * sizeof(unsigned int))) != cudaSuccess ||
        (ce = cudaMalloc(&p->d_counter, sizeof(int))) != cudaSuccess ||
        (ce = cudaMemsetAsync(p->d_counter, 0, sizeof(int), p->stream)) != cudaSuccess ||
        (ce = cudaMemsetAsync(p->d_flags, 0, 2 * sizeof(unsigned int), p->stream)) != cudaSuccess) {
        r = fail(nullptr, ce == cudaErrorMemoryAllocation ? ASSN_ERR_OOM : ASSN_ERR_CUDA, "create: %s",
                 cudaGetErrorString(ce));
        assn_destroy(p);
        return r;
    }
    *out = p;
    return ASSN_OK;
}

int assn_destroy(assn_problem* p) {
    if (!p) return ASSN_OK;
    cudaSetDevice(p->dev);
    if (p->stream) cudaStreamSynchronize(p->stream);
    free_operands(p);
    dfree(p->d_omega); dfree(p->d_w64); dfree(p->d_w32); dfree(p->d_ord); dfree(p->d_cell);
    dfree(p->d_psi_raw[0]); dfree(p->d_psi_raw[1]); dfree(p->d_partials); dfree(p->d_scalar); dfree(p->d_flags);
    dfree(p->d_counter);
    dfree(p->d_stage);
    assn::implicit_free(p->impl);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    delete p;
    return ASSN_OK;
}

int assn_set_quadrature(assn_problem* p, int Q, const double* omega, const double* w) {
    if (!p) return ASSN_ERR_ARG;
    if (!omega || !w) return fail(p, ASSN_ERR_ARG, "omega or w is NULL");
    if (Q < 1 || Q > ASSN_MAX_Q) return fail(p, ASSN_ERR_ARG, "Q = %d out of range [1, %d]", Q, ASSN_MAX_Q);
    for (int q = 0; q < Q; ++q) {
        const double n = sqrt(omega[3 * q] * omega[3 * q] + omega[3 * q + 1] * omega[3 * q + 1] +
                              omega[3 * q + 2] * omega[3 * q + 2]);
        if (!(fabs(n - 1.0) <= 1e-9)) return fail(p, ASSN_ERR_ARG, "ordinate %d is not a unit vector", q);
        if (!(w[q] > 0) || !isfinite(w[q])) return fail(p, ASSN_ERR_ARG, "weight %d is not positive", q);
    }
    int r = set_device(p);
    if (r) return r;
    return install_quadrature(p, Q, omega, w);
}

int assn_set_product_quadrature(assn_problem* p, int n_polar, int n_azim) {
    if (!p) return ASSN_ERR_ARG;
    if (n_polar < 1 || n_azim < 1 || (long)n_polar * n_azim > ASSN_MAX_Q)
        return fail(p, ASSN_ERR_ARG, "product quadrature %d x %d out of range", n_polar, n_azim);
    std::vector<double> mu, wg;
    gauss_legendre(n_polar, mu, wg);
    const int Q = n_polar * n_azim;
    std::vector<double> om(3 * Q), w(Q);
    // azimuth-major numbering q = k n_polar + i: a rotation by 2 pi / n_azim about the z axis maps
    // ordinate q to q + n_polar, so the kernel matrix repeats along its block diagonals
    for (int i = 0; i < n_polar; ++i) {
        const double st = sqrt(std::max(0.0, 1.0 - mu[i] * mu[i]));
        for (int k = 0; k < n_azim; ++k) {
            const double phi = (k + 0.5) * 2.0 * M_PI / n_azim;
            const int q = k * n_polar + i;
            om[3 * q] = st * cos(phi);
            om[3 * q + 1] = st * sin(phi);
            om[3 * q + 2] = mu[i];
            w[q] = wg[i] * 2.0 * M_PI / n_azim;
        }
    }
    return assn_set_quadrature(p, Q, om.data(), w.data());
}

int assn_get_quadrature(const assn_problem* p, int* Q_out, double* omega, double* w) {
    if (!p) return ASSN_ERR_ARG;
    if (!p->have_quad) return ASSN_ERR_STATE;
    if (Q_out) *Q_out = p->Q;
    if (omega) memcpy(omega, p->omega.data(), sizeof(double) * 3 * p->Q);
    if (w) memcpy(w, p->w.data(), sizeof(double) * p->Q);
    return ASSN_OK;
}

int assn_set_cross_sections(assn_problem* p, const double* sigma_a, const double* sigma_s, const double* q) {
    if (!p) return ASSN_ERR_ARG;
    if (!sigma_a || !sigma_s || !q) return fail(p, ASSN_ERR_ARG, "cross section array is NULL");
    const size_t n = p->ncell();
    for (size_t c = 0; c < n; ++c) {
        if (!(sigma_a[c] >= 0) || !(sigma_s[c] >= 0) || !isfinite(sigma_a[c]) || !isfinite(sigma_s[c]) ||
            !isfinite(q[c]))
            return fail(p, ASSN_ERR_ARG, "cell %zu: invalid cross section or source", c);
    }
    int r = set_device(p);
    if (r) return r;
    if (p->sa.data() != sigma_a) p->sa.assign(sigma_a, sigma_a + n);
    if (p->ss.data() != sigma_s) p->ss.assign(sigma_s, sigma_s + n);
    if (p->src.data() != q) p->src.assign(q, q + n);
    const double inv_wsum = p->wsum > 0 ? 1.0 / p->wsum : 1.0 / (4.0 * M_PI);
    if (p->precision == ASSN_FP64) {
        std::vector<CellD> cl(n);
        for (size_t c = 0; c < n; ++c) cl[c] = CellD{sigma_a[c] + sigma_s[c], sigma_s[c] * inv_wsum, q[c], 0.0};
        CK(p, cudaMemcpyAsync(p->d_cell, cl.data(), sizeof(CellD) * n, cudaMemcpyHostToDevice, p->stream));
        CK(p, cudaStreamSynchronize(p->stream));
    } else {
        std::vector<CellF> cl(n);
        for (size_t c = 0; c < n; ++c)
            cl[c] = CellF{(float)(sigma_a[c] + sigma_s[c]), (float)(sigma_s[c] * inv_wsum), (float)q[c], 0.0f};
        CK(p, cudaMemcpyAsync(p->d_cell, cl.data(), sizeof(CellF) * n, cudaMemcpyHostToDevice, p->stream));
        CK(p, cudaStreamSynchronize(p->stream));
    }
    p->have_xs = true;
    return ASSN_OK;
}

int assn_set_artificial_scattering(assn_problem* p, double sigma_as, double eps, int kernel_kind, int normalisation) {
    if (!p) return ASSN_ERR_ARG;
    if (!(sigma_as >= 0) || !isfinite(sigma_as)) return fail(p, ASSN_ERR_ARG, "sigma_as must be >= 0");
    if (!(eps > 0) || !isfinite(eps)) return fail(p, ASSN_ERR_ARG, "eps must be > 0");
    if (kernel_kind != ASSN_KERNEL_GAUSS && kernel_kind != ASSN_KERNEL_EXP)
        return fail(p, ASSN_ERR_ARG, "unknown kernel kind %d", kernel_kind);
    if (normalisation != ASSN_NORM_COLUMN && normalisation != ASSN_NORM_ROW)
        return fail(p, ASSN_ERR_ARG, "unknown normalisation %d", normalisation);
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "set a quadrature first");
    int r = set_device(p);
    if (r) return r;
    free_operands(p);
    const int Q = p->Q, Qp = p->Qp;
    CK(p, cudaMalloc(&p->d_K64, sizeof(double) * Q * Q));
    CK(p, cudaMalloc(&p->d_e, sizeof(double) * Q));
    CK(p, launch_build_K(p->d_omega, p->d_w64, Q, eps, kernel_kind, normalisation, p->d_K64, p->stream));
    p->launches++;
    if (p->precision == ASSN_FP64) {
        CK(p, cudaMalloc(&p->d_KT64, sizeof(double) * Qp * Qp));
        CK(p, launch_derive_simt_f64(p->d_K64, p->d_w64, Q, Qp, normalisation, p->d_KT64, p->d_e, p->stream));
    } else if (p->precision == ASSN_FP32) {
        CK(p, cudaMalloc(&p->d_KT32, sizeof(float) * Qp * Qp));
        CK(p, launch_derive_simt_f32(p->d_K64, p->d_w64, Q, Qp, normalisation, p->d_KT32, p->d_e, p->stream));
    } else if (p->precision == ASSN_TF32) {
        p->tc.Mp = (Q + 127) / 128 * 128;
        CK(p, cudaMalloc(&p->tc.G32, sizeof(float) * (size_t)p->tc.Mp * Qp));
        CK(p, launch_derive_tf32(p->d_K64, p->d_w64, Q, Qp, p->tc.Mp, normalisation, p->tc.G32, p->d_e, p->stream));
    } else {
        const bool split = p->precision == ASSN_BF16X3 || p->precision == ASSN_BF16X2;   // G hi + lo
        p->tc.Mp = (Q + 127) / 128 * 128;
        CK(p, cudaMalloc(&p->tc.G_hi, sizeof(__nv_bfloat16) * (size_t)p->tc.Mp * Qp));
        if (split) CK(p, cudaMalloc(&p->tc.G_lo, sizeof(__nv_bfloat16) * (size_t)p->tc.Mp * Qp));
        CK(p, launch_derive_tc(p->d_K64, p->d_w64, Q, Qp, p->tc.Mp, normalisation, split, p->tc.G_hi, p->tc.G_lo,
                               p->d_e, p->stream));
    }
    p->launches++;
    p->e.assign(Q, 0.0);
    CK(p, cudaMemcpyAsync(p->e.data(), p->d_e, sizeof(double) * Q, cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    p->sigma_as = sigma_as;
    p->eps = eps;
    p->kind = kernel_kind;
    p->norm = normalisation;
    p->ord_dt = -1;
    p->have_K = true;
    return ASSN_OK;
}

int assn_get_kernel_matrix(assn_problem* p, double* K_host) {
    if (!p || !K_host) return ASSN_ERR_ARG;
    if (!p->have_K) return fail(p, ASSN_ERR_STATE, "K not built");
    CK(p, cudaMemcpyAsync(K_host, p->d_K64, sizeof(double) * p->Q * p->Q, cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    return ASSN_OK;
}

int assn_layout(const assn_problem* p, int* Qpad, int* elem_bytes) {
    if (!p) return ASSN_ERR_ARG;
    if (!p->have_quad) return ASSN_ERR_STATE;
    if (Qpad) *Qpad = p->Qp;
    if (elem_bytes) *elem_bytes = (int)p->elem();
    return ASSN_OK;
}

int assn_state_device(assn_problem* p, void** psi_dev) {
    if (!p || !psi_dev) return ASSN_ERR_ARG;
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    *psi_dev = p->d_psi[p->cur];
    return ASSN_OK;
}

int assn_set_state(assn_problem* p, const double* psi) {
    if (!p || !psi) return ASSN_ERR_ARG;
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    int r = set_device(p);
    if (r) return r;
    const size_t n = p->ncell();
    const size_t chunk_cells = std::max<size_t>(1, (8u << 20) / p->Q);   // 64 MB of FP64 per chunk
    r = ensure_stage(p, std::min(n, chunk_cells) * p->Q);
    if (r) return r;
    for (size_t c0 = 0; c0 < n; c0 += chunk_cells) {
        const size_t nc = std::min(chunk_cells, n - c0);
        CK(p, cudaMemcpyAsync(p->d_stage, psi + c0 * p->Q, sizeof(double) * nc * p->Q, cudaMemcpyHostToDevice,
                              p->stream));
        if (p->precision == ASSN_FP64)
            CK(p, launch_pack_state(p->d_stage, (double*)p->d_psi[p->cur] + c0 * p->Qp, nc, p->Q, p->Qp, p->stream));
        else
            CK(p, launch_pack_state(p->d_stage, (float*)p->d_psi[p->cur] + c0 * p->Qp, nc, p->Q, p->Qp, p->stream));
        p->launches++;
        CK(p, cudaStreamSynchronize(p->stream));
    }
    return ASSN_OK;
}

int assn_get_state(assn_problem* p, double* psi) {
    if (!p || !psi) return ASSN_ERR_ARG;
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    int r = set_device(p);
    if (r) return r;
    const size_t n = p->ncell();
    const size_t chunk_cells = std::max<size_t>(1, (8u << 20) / p->Q);
    r = ensure_stage(p, std::min(n, chunk_cells) * p->Q);
    if (r) return r;
    for (size_t c0 = 0; c0 < n; c0 += chunk_cells) {
        const size_t nc = std::min(chunk_cells, n - c0);
        if (p->precision == ASSN_FP64)
            CK(p, launch_unpack_state((const double*)p->d_psi[p->cur] + c0 * p->Qp, p->d_stage, nc, p->Q, p->Qp, p->stream));
        else
            CK(p, launch_unpack_state((const float*)p->d_psi[p->cur] + c0 * p->Qp, p->d_stage, nc, p->Q, p->Qp, p->stream));
        p->launches++;
        CK(p, cudaMemcpyAsync(psi + c0 * p->Q, p->d_stage, sizeof(double) * nc * p->Q, cudaMemcpyDeviceToHost,
                              p->stream));
        CK(p, cudaStreamSynchronize(p->stream));
    }
    return check_flags(p);
}

int assn_set_state_f32(assn_problem* p, const float* psi) {
    if (!p || !psi) return ASSN_ERR_ARG;
    assn::TraceRange tr("assn_set_state_f32");
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    if (p->precision == ASSN_FP64) return fail(p, ASSN_ERR_UNSUPPORTED, "FP32 state copy on an FP64 problem");
    int r = set_device(p);
    if (r) return r;
    if (p->Q == p->Qp)   // the layouts agree: one contiguous copy (a row per cell runs slower)
        CK(p, cudaMemcpyAsync(p->d_psi[p->cur], psi, sizeof(float) * p->Qp * p->ncell(), cudaMemcpyHostToDevice,
                              p->stream));
    else
        CK(p, cudaMemcpy2DAsync(p->d_psi[p->cur], sizeof(float) * p->Qp, psi, sizeof(float) * p->Q,
                                sizeof(float) * p->Q, p->ncell(), cudaMemcpyHostToDevice, p->stream));
    return ASSN_OK;
}

int assn_get_state_f32(assn_problem* p, float* psi) {
    if (!p || !psi) return ASSN_ERR_ARG;
    assn::TraceRange tr("assn_get_state_f32");
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    if (p->precision == ASSN_FP64) return fail(p, ASSN_ERR_UNSUPPORTED, "FP32 state copy on an FP64 problem");
    int r = set_device(p);
    if (r) return r;
    if (p->Q == p->Qp)
        CK(p, cudaMemcpyAsync(psi, p->d_psi[p->cur], sizeof(float) * p->Qp * p->ncell(), cudaMemcpyDeviceToHost,
                              p->stream));
    else
        CK(p, cudaMemcpy2DAsync(psi, sizeof(float) * p->Q, p->d_psi[p->cur], sizeof(float) * p->Qp,
                                sizeof(float) * p->Q, p->ncell(), cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    return check_flags(p);
}

int assn_init_line_source(assn_problem* p, double delta, double floor_value) {
    if (!p) return ASSN_ERR_ARG;
    if (!(delta > 0)) return fail(p, ASSN_ERR_ARG, "delta must be > 0");
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    int r = set_device(p);
    if (r) return r;
    if (p->precision == ASSN_FP64)
        CK(p, launch_init_line_source((double*)p->d_psi[p->cur], p->nx, p->ny, p->Q, p->Qp, p->x0, p->y0, p->h, delta,
                                      floor_value, p->stream));
    else
        CK(p, launch_init_line_source((float*)p->d_psi[p->cur], p->nx, p->ny, p->Q, p->Qp, p->x0, p->y0, p->h, delta,
                                      floor_value, p->stream));
    p->launches++;
    return ASSN_OK;
}

int assn_max_stable_dt(assn_problem* p, double* dt_out) {
    if (!p || !dt_out) return ASSN_ERR_ARG;
    int r = ready(p);
    if (r) return r;
    *dt_out = max_stable_dt(p);
    return ASSN_OK;
}

// The tensor-core kernel a step of p runs: the requested variant, or (automatic, -1) the paired-SM
// kernel where it applies (forward Euler or Heun, 193..256 or 449..512 ordinates), else variant 0.
// TF32 and BF16X2 have the paired-SM kernel only.
static int eff_variant(const assn_problem* p) {
    if (p->variant >= 0) return p->variant;
    if (p->paired_only()) return 2;
    return (p->scheme != ASSN_SCHEME_IMPLICIT &&
            tc3_supported(p->Q, p->Qp, p->tc.Mp, p->precision == ASSN_BF16X3)) ? 2 : 0;
}

}  // extern "C"

namespace assn {
bool problem_paired(const assn_problem* p) { return p->tensor() && eff_variant(p) == 2; }
bool problem_pair_supported(const assn_problem* p) {
    return p->tensor() && tc3_supported(p->Q, p->Qp, p->tc.Mp, p->precision != ASSN_BF16);
}

cudaError_t problem_pair_launch(assn_problem* p, double dt, int parity, int heun_stage, unsigned int* err_flag,
                                cudaStream_t s) {
    const float fdt = (float)dt, fdts = (float)(dt * p->sigma_as);
    if (heun_stage < 0)
        return launch_step_tc3(p->plan3, parity, (const OrdF*)p->d_ord, (const CellF*)p->d_cell, p->d_w32, fdt, fdts,
                               err_flag, s);
    if (heun_stage == 0)
        return launch_heun_stage_tc3(p->plan3, parity, (const OrdF*)p->d_ord, (const CellF*)p->d_cell, p->d_w32, fdt,
                                     fdts, nullptr, 0.0f, 1.0f, err_flag, s);
    return launch_heun_stage_tc3(p->plan3, parity, (const OrdF*)p->d_ord, (const CellF*)p->d_cell, p->d_w32, fdt, fdts,
                                 (const float*)p->d_psi[parity ^ 1], 0.5f, 0.5f, err_flag, s);
}
}  // namespace assn

extern "C" {

static int step_once(assn_problem* p, const void* in, void* out, double dt) {
    if (p->precision == ASSN_FP64) {
        StepArgs<double, OrdD, CellD> a{(const double*)in, (double*)out, (const OrdD*)p->d_ord,
                                        (const CellD*)p->d_cell, p->d_KT64, p->nx, p->ny, p->Q, p->Qp, dt,
                                        dt * p->sigma_as};
        CK(p, launch_step_simt_f64(a, p->stream));
    } else {
        StepArgs<float, OrdF, CellF> a{(const float*)in, (float*)out, (const OrdF*)p->d_ord,
                                       (const CellF*)p->d_cell, p->d_KT32, p->nx, p->ny, p->Q, p->Qp, (float)dt,
                                       (float)(dt * p->sigma_as)};
        if (p->precision == ASSN_FP32) {
            CK(p, launch_step_simt_f32(a, p->stream));
        } else {
            const bool own = in == p->d_psi[p->cur] && out == p->d_psi[p->cur ^ 1];
            cudaError_t e;
            const int v = eff_variant(p);
            if (v == 2 && own) {
                e = launch_step_tc3(p->plan3, p->cur, (const OrdF*)p->d_ord, (const CellF*)p->d_cell, p->d_w32,
                                    (float)dt, (float)(dt * p->sigma_as), p->d_flags + 1, p->stream);
            } else if (v == 0 && own) {
                // the persistent kernel takes its buffer parity from the device step counter
                if ((p->counter_host & 1) != p->cur) {
                    p->counter_host = p->cur;
                    CK(p, cudaMemcpyAsync(p->d_counter, &p->counter_host, sizeof(int), cudaMemcpyHostToDevice,
                                          p->stream));
                }
                e = launch_step_tc2(p->plan2, p->d_flags + 1, p->cur, p->stream);
                p->counter_host += 1;
            } else {
                e = launch_step_tc(p->plan, a, p->d_w32, p->d_flags + 1, p->stream);
            }
            if (e == cudaErrorNotSupported) return fail(p, ASSN_ERR_UNSUPPORTED, "tensor-core step: shape not supported");
            CK(p, e);
        }
    }
    p->launches++;
    return ASSN_OK;
}

static int ensure_plan(assn_problem* p, double dt, bool need_v1) {
    cudaError_t e = cudaSuccess;
    const int v = eff_variant(p);
    if (p->paired_only() && (v != 2 || need_v1))
        return fail(p, ASSN_ERR_UNSUPPORTED,
                    "TF32 and BF16X2 run on the paired-SM kernel only (tiling variant 2, its own flux buffers or a "
                    "16-byte aligned input)");
    if ((v == 1 || need_v1) && !p->plan)
        e = tc_plan_create(&p->plan, p->tc.G_hi, p->tc.G_lo, p->Q, p->Qp, p->tc.Mp, p->nx, p->ny,
                           p->precision == ASSN_BF16X3, p->want_nt, p->want_stages);
    if (e == cudaSuccess && v == 0 && (!p->plan2 || p->plan2_dt != dt)) {
        if (p->plan2) tc2_plan_destroy(p->plan2);
        p->plan2 = nullptr;
        const Tc2Problem d = problem_tc2(p, dt, 0x7fffffff);
        e = tc2_plan_create(&p->plan2, &d, 1, p->precision == ASSN_BF16X3, p->want_nt, p->want_rings);
        if (e == cudaSuccess) p->plan2_dt = dt;
    }
    if (e == cudaSuccess && v == 2 && !p->plan3) {
        if (!tc3_supported(p->Q, p->Qp, p->tc.Mp, p->precision == ASSN_BF16X3))
            return fail(p, ASSN_ERR_UNSUPPORTED,
                        "paired-SM step (variant 2): 193..256 or 449..512 ordinates only (Q = %d)", p->Q);
        e = tc3_plan_create(&p->plan3, (const float*)p->d_psi[0], (const float*)p->d_psi[1], p->tc, p->precision,
                            p->Q, p->Qp, p->tc.Mp, p->nx, p->ny, p->want_rings, p->stream);
    }
    if (e == cudaErrorNotSupported)
        return fail(p, ASSN_ERR_UNSUPPORTED, "tensor-core step: Q = %d with tile %d / stages %d not supported", p->Q,
                    p->want_nt, p->want_stages);
    CK(p, e);
    return ASSN_OK;
}

}  // extern "C"

namespace assn {
int problem_pair_plan(assn_problem* p, double dt) { return ensure_plan(p, dt, false); }
}  // namespace assn

extern "C" {

static int prepare_step(assn_problem* p, double dt) {
    int r = assn::problem_prepare(p, dt);
    if (r) return r;
    if (p->tensor()) {
        r = ensure_plan(p, dt, false);
        if (r) return r;
    }
    return ASSN_OK;
}

}  // extern "C"

int assn::problem_prepare(assn_problem* p, double dt) {
    int r = ready(p);
    if (r) return r;
    if (!(dt > 0) || !isfinite(dt)) return fail(p, ASSN_ERR_ARG, "dt must be > 0");
    const double dmax = max_stable_dt(p);
    if (dt > dmax * (1.0 + 1e-12))
        return fail(p, ASSN_ERR_UNSTABLE, "dt = %.17g exceeds the positivity bound %.17g", dt, dmax);
    r = set_device(p);
    if (r) return r;
    return upload_ord(p, dt);
}

extern "C" {

int assn_set_scheme(assn_problem* p, int scheme) {
    if (!p) return ASSN_ERR_ARG;
    if (scheme != ASSN_SCHEME_EULER_UPWIND && scheme != ASSN_SCHEME_HEUN_MINMOD && scheme != ASSN_SCHEME_IMPLICIT)
        return fail(p, ASSN_ERR_ARG, "unknown scheme %d", scheme);
    if (scheme == ASSN_SCHEME_IMPLICIT && p->tensor())
        return fail(p, ASSN_ERR_UNSUPPORTED, "the implicit scheme runs in FP64 or FP32 (CUDA cores)");
    p->scheme = scheme;
    return ASSN_OK;
}

int assn_get_scheme(const assn_problem* p, int* scheme) {
    if (!p || !scheme) return ASSN_ERR_ARG;
    *scheme = p->scheme;
    return ASSN_OK;
}

// One Heun step (two stages); the state stays in buffer cur.
static int heun_step(assn_problem* p, double dt) {
    void* a = p->d_psi[p->cur];
    void* b = p->d_psi[p->cur ^ 1];
    if (p->tensor() && eff_variant(p) == 2) {
        // paired-SM kernel: stage 1 reads a and writes b; stage 2 reads b and writes a, keeping psi^n
        // from a (each element is read there before it is overwritten, by the same thread)
        const float fdt = (float)dt, fdts = (float)(dt * p->sigma_as);
        cudaError_t e = launch_heun_stage_tc3(p->plan3, p->cur, (const OrdF*)p->d_ord, (const CellF*)p->d_cell,
                                              p->d_w32, fdt, fdts, nullptr, 0.0f, 1.0f, p->d_flags + 1, p->stream);
        if (e == cudaSuccess)
            e = launch_heun_stage_tc3(p->plan3, p->cur ^ 1, (const OrdF*)p->d_ord, (const CellF*)p->d_cell, p->d_w32,
                                      fdt, fdts, (const float*)a, 0.5f, 0.5f, p->d_flags + 1, p->stream);
        CK(p, e);
        p->launches += 2;
        return ASSN_OK;
    }
    if (p->tensor()) {
        // persistent kernel: the device step counter's parity selects the flux buffer, and each
        // launch advances it, so stage 1 reads a and writes b, stage 2 reads b and writes a
        if ((p->counter_host & 1) != p->cur) {
            p->counter_host = p->cur;
            CK(p, cudaMemcpyAsync(p->d_counter, &p->counter_host, sizeof(int), cudaMemcpyHostToDevice, p->stream));
        }
        cudaError_t e = launch_heun_stage_tc2(p->plan2, p->d_flags + 1, p->cur, nullptr, 0.0f, 1.0f, p->stream);
        if (e == cudaSuccess)
            e = launch_heun_stage_tc2(p->plan2, p->d_flags + 1, p->cur ^ 1, (const float*)a, 0.5f, 0.5f, p->stream);
        CK(p, e);
        p->counter_host += 2;
        p->launches += 2;
        return ASSN_OK;
    }
    if (p->precision == ASSN_FP64) {
        StepArgs<double, OrdD, CellD> s1{(const double*)a, (double*)b, (const OrdD*)p->d_ord, (const CellD*)p->d_cell,
                                         p->d_KT64, p->nx, p->ny, p->Q, p->Qp, dt, dt * p->sigma_as};
        CK(p, launch_stage_simt_f64(s1, nullptr, 0.0, 1.0, p->stream));
        StepArgs<double, OrdD, CellD> s2 = s1;
        s2.psi = (const double*)b;
        s2.psi_out = (double*)a;
        CK(p, launch_stage_simt_f64(s2, (const double*)a, 0.5, 0.5, p->stream));
    } else {
        StepArgs<float, OrdF, CellF> s1{(const float*)a, (float*)b, (const OrdF*)p->d_ord, (const CellF*)p->d_cell,
                                        p->d_KT32, p->nx, p->ny, p->Q, p->Qp, (float)dt, (float)(dt * p->sigma_as)};
        CK(p, launch_stage_simt_f32(s1, nullptr, 0.0f, 1.0f, p->stream));
        StepArgs<float, OrdF, CellF> s2 = s1;
        s2.psi = (const float*)b;
        s2.psi_out = (float*)a;
        CK(p, launch_stage_simt_f32(s2, (const float*)a, 0.5f, 0.5f, p->stream));
    }
    p->launches += 2;
    return ASSN_OK;
}

int assn_step(assn_problem* p, int nsteps, double dt) {
    if (!p) return ASSN_ERR_ARG;
    assn::TraceRange tr("assn_step");
    if (nsteps < 0) return fail(p, ASSN_ERR_ARG, "nsteps < 0");
    if (p->scheme == ASSN_SCHEME_IMPLICIT) return assn::implicit_steps(p, nsteps, dt);
    if (p->scheme == ASSN_SCHEME_HEUN_MINMOD) {
        int r = assn::problem_prepare(p, dt);
        if (r) return r;
        if (p->tensor()) {
            if (eff_variant(p) == 1)
                return fail(p, ASSN_ERR_UNSUPPORTED,
                            "the Heun + minmod scheme runs on the persistent kernels (variants 0 and 2)");
            r = ensure_plan(p, dt, false);
            if (r) return r;
        }
        for (int n = 0; n < nsteps; ++n) {
            r = heun_step(p, dt);
            if (r) return r;
        }
        return ASSN_OK;
    }
    int r = prepare_step(p, dt);
    if (r) return r;
    for (int n = 0; n < nsteps; ++n) {
        r = step_once(p, p->d_psi[p->cur], p->d_psi[p->cur ^ 1], dt);
        if (r) return r;
        p->cur ^= 1;
    }
    return ASSN_OK;
}

int assn_step_device(assn_problem* p, const void* psi_in_dev, void* psi_out_dev, double dt) {
    if (!p || !psi_in_dev || !psi_out_dev) return ASSN_ERR_ARG;
    if (p->scheme != ASSN_SCHEME_EULER_UPWIND)
        return fail(p, ASSN_ERR_UNSUPPORTED, "assn_step_device takes the forward-Euler upwind step only");
    if (psi_in_dev == psi_out_dev) return fail(p, ASSN_ERR_ARG, "input and output buffers must differ");
    int r = prepare_step(p, dt);
    if (r) return r;
    if (p->tensor() && eff_variant(p) == 2 && !((uintptr_t)psi_in_dev & 15u) && !((uintptr_t)psi_out_dev & 3u)) {
        // the paired-SM kernel, with a tensor map of the caller's input
        r = ensure_plan(p, dt, false);
        if (r) return r;
        CK(p, launch_step_tc3_buffers(p->plan3, (const float*)psi_in_dev, (float*)psi_out_dev, (const OrdF*)p->d_ord,
                                      (const CellF*)p->d_cell, p->d_w32, (float)dt, (float)(dt * p->sigma_as),
                                      p->d_flags + 1, p->stream));
        p->launches++;
        return ASSN_OK;
    }
    if (p->tensor()) {   // other caller-owned buffers run on the one-tile-per-CTA kernel
        r = ensure_plan(p, dt, true);
        if (r) return r;
    }
    return step_once(p, psi_in_dev, psi_out_dev, dt);
}

int assn_set_tiling(assn_problem* p, int tile_cells, int stages, int variant) {
    if (!p) return ASSN_ERR_ARG;
    if (tile_cells != 0 && tile_cells != 32 && tile_cells != 64 && tile_cells != 128 && tile_cells != 256)
        return fail(p, ASSN_ERR_ARG, "tile_cells must be 0, 32, 64, 128 or 256");
    if (stages != 0 && (stages < 2 || stages > 8)) return fail(p, ASSN_ERR_ARG, "stages must be 0 or 2..8");
    if (variant < -1 || variant > 2) return fail(p, ASSN_ERR_ARG, "variant must be -1 (automatic), 0, 1 or 2");
    if (p->paired_only() && (variant == 0 || variant == 1))
        return fail(p, ASSN_ERR_UNSUPPORTED, "TF32 and BF16X2 run on the paired-SM kernel only (variant -1 or 2)");
    p->want_nt = tile_cells;
    p->want_stages = stages;
    p->want_rings = TcRings{stages, stages, stages, 0};
    p->variant = variant;
    if (p->plan) tc_plan_destroy(p->plan);
    p->plan = nullptr;
    if (p->plan2) tc2_plan_destroy(p->plan2);
    p->plan2 = nullptr;
    if (p->plan3) tc3_plan_destroy(p->plan3);
    p->plan3 = nullptr;
    return ASSN_OK;
}

int assn_set_rings(assn_problem* p, int staging, int operand, int kernel_matrix, int blocks_per_request) {
    if (!p) return ASSN_ERR_ARG;
    auto bad = [](int v) { return v != 0 && (v < 2 || v > 8); };
    if (bad(staging) || bad(operand) || bad(kernel_matrix))
        return fail(p, ASSN_ERR_ARG, "ring depths must be 0 or 2..8");
    if (blocks_per_request != 0 && blocks_per_request != 1 && blocks_per_request != 2 && blocks_per_request != 4 &&
        blocks_per_request != 8)
        return fail(p, ASSN_ERR_ARG, "blocks_per_request must be 0, 1, 2, 4 or 8");
    p->want_rings = TcRings{staging, operand, kernel_matrix, blocks_per_request};
    if (p->variant != 2) p->variant = p->paired_only() ? 2 : 0;
    if (p->plan2) tc2_plan_destroy(p->plan2);
    p->plan2 = nullptr;
    if (p->plan3) tc3_plan_destroy(p->plan3);
    p->plan3 = nullptr;
    return ASSN_OK;
}

int assn_get_rings(assn_problem* p, int* staging, int* operand, int* kernel_matrix, int* blocks_per_request) {
    if (!p) return ASSN_ERR_ARG;
    if (!p->tensor()) return fail(p, ASSN_ERR_UNSUPPORTED, "rings apply to the tensor-core precisions");
    int r = ready(p);
    if (r) return r;
    r = set_device(p);
    if (r) return r;
    const int v = p->variant;
    const bool pair = eff_variant(p) == 2;
    if (!pair) p->variant = 0;
    r = ensure_plan(p, p->plan2_dt > 0 ? p->plan2_dt : 1.0, false);
    p->variant = v;
    if (r) return r;
    const TcRings g = pair ? tc3_plan_rings(p->plan3) : tc2_plan_rings(p->plan2);
    if (staging) *staging = g.SS;
    if (operand) *operand = g.SB;
    if (kernel_matrix) *kernel_matrix = g.SA;
    if (blocks_per_request) *blocks_per_request = g.MPR;
    return ASSN_OK;
}

int assn_get_tiling(assn_problem* p, int* tile_cells, int* stages, int* tmem_cols, int64_t* smem_bytes) {
    if (!p) return ASSN_ERR_ARG;
    if (!p->tensor()) return fail(p, ASSN_ERR_UNSUPPORTED, "tiling applies to the tensor-core precisions");
    int r = ready(p);
    if (r) return r;
    r = set_device(p);
    if (r) return r;
    r = ensure_plan(p, p->plan2_dt > 0 ? p->plan2_dt : 1.0, false);
    if (r) return r;
    size_t sm = 0;
    const int v = eff_variant(p);
    if (v == 1) {
        tc_plan_describe(p->plan, tile_cells, stages, tmem_cols, &sm);
    } else if (v == 2) {
        tc3_plan_describe(p->plan3, tile_cells, stages, nullptr, &sm);
        if (tmem_cols) *tmem_cols = 512;
    } else {
        tc2_plan_describe(p->plan2, tile_cells, stages, tmem_cols, &sm);
    }
    if (smem_bytes) *smem_bytes = (int64_t)sm;
    return ASSN_OK;
}

int assn_get_variant(assn_problem* p, int* variant) {
    if (!p || !variant) return ASSN_ERR_ARG;
    if (!p->tensor()) return fail(p, ASSN_ERR_UNSUPPORTED, "variants apply to the tensor-core precisions");
    int r = ready(p);
    if (r) return r;
    *variant = eff_variant(p);
    return ASSN_OK;
}

int assn_run_f32(assn_problem* p, const float* psi0_host, int nsteps, double dt, double* phi_host) {
    if (!p || !psi0_host || !phi_host) return ASSN_ERR_ARG;
    assn::TraceRange tr("assn_run_f32");
    if (nsteps < 0) return fail(p, ASSN_ERR_ARG, "nsteps < 0");
    int r = prepare_step(p, dt);
    if (r) return r;
    r = assn_set_state_f32(p, psi0_host);
    if (r) return r;
    r = assn_step(p, nsteps, dt);
    if (r) return r;
    return assn_scalar_flux(p, phi_host);
}

int assn_scalar_flux(assn_problem* p, double* phi_host) {
    if (!p || !phi_host) return ASSN_ERR_ARG;
    assn::TraceRange tr("assn_scalar_flux");
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    int r = set_device(p);
    if (r) return r;
    r = ensure_stage(p, p->ncell());
    if (r) return r;
    if (p->precision == ASSN_FP64)
        CK(p, launch_scalar_flux((const double*)p->d_psi[p->cur], p->d_w64, (int)p->ncell(), p->Qp, nullptr, p->d_stage, p->stream));
    else
        CK(p, launch_scalar_flux((const float*)p->d_psi[p->cur], p->d_w32, (int)p->ncell(), p->Qp, nullptr, p->d_stage, p->stream));
    p->launches++;
    CK(p, cudaMemcpyAsync(phi_host, p->d_stage, sizeof(double) * p->ncell(), cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    return check_flags(p);
}

int assn_scalar_flux_device(assn_problem* p, float* phi_dev) {
    if (!p || !phi_dev) return ASSN_ERR_ARG;
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    int r = set_device(p);
    if (r) return r;
    if (p->precision == ASSN_FP64)
        CK(p, launch_scalar_flux((const double*)p->d_psi[p->cur], p->d_w64, (int)p->ncell(), p->Qp, phi_dev, nullptr, p->stream));
    else
        CK(p, launch_scalar_flux((const float*)p->d_psi[p->cur], p->d_w32, (int)p->ncell(), p->Qp, phi_dev, nullptr, p->stream));
    p->launches++;
    return ASSN_OK;
}

int assn_mass(assn_problem* p, double* mass_out) {
    if (!p || !mass_out) return ASSN_ERR_ARG;
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    int r = set_device(p);
    if (r) return r;
    if (p->precision == ASSN_FP64)
        CK(p, launch_mass_partials((const double*)p->d_psi[p->cur], p->d_w64, (int)p->ncell(), p->Qp, p->d_partials, kMassBlocks, p->stream));
    else
        CK(p, launch_mass_partials((const float*)p->d_psi[p->cur], p->d_w32, (int)p->ncell(), p->Qp, p->d_partials, kMassBlocks, p->stream));
    CK(p, launch_reduce_partials(p->d_partials, kMassBlocks, p->d_scalar, p->stream));
    p->launches += 2;
    double m = 0;
    CK(p, cudaMemcpyAsync(&m, p->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    *mass_out = m * p->h * p->h;
    return check_flags(p);
}

int assn_check_finite(assn_problem* p) {
    if (!p) return ASSN_ERR_ARG;
    if (!p->have_quad) return fail(p, ASSN_ERR_STATE, "no quadrature set");
    int r = set_device(p);
    if (r) return r;
    CK(p, cudaMemsetAsync(p->d_flags, 0, sizeof(unsigned int), p->stream));
    const size_t n = p->ncell() * p->Qp;
    if (p->precision == ASSN_FP64)
        CK(p, launch_check_finite((const double*)p->d_psi[p->cur], n, p->d_flags, p->stream));
    else
        CK(p, launch_check_finite((const float*)p->d_psi[p->cur], n, p->d_flags, p->stream));
    p->launches++;
    unsigned int f = 0;
    CK(p, cudaMemcpyAsync(&f, p->d_flags, sizeof f, cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    if (f) return fail(p, ASSN_ERR_NONFINITE, "state holds NaN or Inf");
    return check_flags(p);
}

int assn_check_guards(assn_problem* p, int64_t* guard_bytes_changed, int64_t* padding_nonzero) {
    if (!p || !guard_bytes_changed || !padding_nonzero) return ASSN_ERR_ARG;
    if (!p->d_psi_raw[0]) return fail(p, ASSN_ERR_STATE, "no state allocated");
    int r = set_device(p);
    if (r) return r;
    const size_t bytes = p->ncell() * p->Qp * p->elem();
    std::vector<unsigned char> g(4 * kStateGuard);
    unsigned long long* d_count = reinterpret_cast<unsigned long long*>(p->d_partials);   // scratch
    CK(p, cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), p->stream));
    for (int b = 0; b < 2; ++b) {
        CK(p, cudaMemcpyAsync(g.data() + (2 * b) * kStateGuard, p->d_psi_raw[b], kStateGuard, cudaMemcpyDeviceToHost,
                              p->stream));
        CK(p, cudaMemcpyAsync(g.data() + (2 * b + 1) * kStateGuard, p->d_psi_raw[b] + kStateGuard + bytes, kStateGuard,
                              cudaMemcpyDeviceToHost, p->stream));
        if (p->precision == ASSN_FP64)
            CK(p, launch_padding_nonzero((const double*)p->d_psi[b], p->ncell(), p->Q, p->Qp, d_count, p->stream));
        else
            CK(p, launch_padding_nonzero((const float*)p->d_psi[b], p->ncell(), p->Q, p->Qp, d_count, p->stream));
        p->launches++;
    }
    unsigned long long nz = 0;
    CK(p, cudaMemcpyAsync(&nz, d_count, sizeof nz, cudaMemcpyDeviceToHost, p->stream));
    CK(p, cudaStreamSynchronize(p->stream));
    int64_t bad = 0;
    for (unsigned char c : g) bad += c != kGuardByte;
    *guard_bytes_changed = bad;
    *padding_nonzero = (int64_t)nz;
    return check_flags(p);
}

}  // extern "C"

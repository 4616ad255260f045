// Artificial-scattering matrix K built on the device in FP64, and the operands each
// precision's contraction consumes.
//
// K follows Sec. 2.3 (kernel s_eps(mu) ~ exp(-(1-mu)^2/eps^2)) and Sec. 3.2 (discrete gain
// sum_p w_p c s_qp psi_p with a normalisation factor c).  The constant prefactor of s_eps
// cancels in either normalisation and is not evaluated.
#include "assn_internal.h"

namespace assn {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; every thread gets the result.  blockDim.x is a multiple of 32, <= 1024.
__device__ double block_sum(double v) {
    __shared__ double red[32];
    __shared__ double total;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double t = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) total = t;
    }
    __syncthreads();
    double r = total;
    __syncthreads();
    return r;
}

__device__ __forceinline__ double kernel_value(const double* omega, int a, int b, double inv_eps2,
                                               int kind) {
    double mu = omega[3 * a] * omega[3 * b] + omega[3 * a + 1] * omega[3 * b + 1] +
                omega[3 * a + 2] * omega[3 * b + 2];
    mu = fmin(1.0, fmax(-1.0, mu));
    const double d = 1.0 - mu;
    return kind == ASSN_KERNEL_GAUSS ? exp(-d * d * inv_eps2) : exp(-d * inv_eps2);
}

// One block per normalised line l: the column p = l (COLUMN) or the row q = l (ROW).
// K is row-major [Q][Q]: K[q*Q + p].
__global__ void build_K_kernel(const double* __restrict__ omega, const double* __restrict__ w, int Q,
                               double inv_eps2, int kind, int norm, double* __restrict__ K) {
    const int l = blockIdx.x;
    double part = 0.0;
    for (int m = threadIdx.x; m < Q; m += blockDim.x) part += w[m] * kernel_value(omega, l, m, inv_eps2, kind);
    const double c = 1.0 / block_sum(part);
    for (int m = threadIdx.x; m < Q; m += blockDim.x) {
        const double s = kernel_value(omega, l, m, inv_eps2, kind);
        if (norm == ASSN_NORM_COLUMN)
            K[(size_t)m * Q + l] = w[l] * c * s;   // K_{m l} = w_l c_l s_{ml}
        else
            K[(size_t)l * Q + m] = w[m] * c * s;   // K_{l m} = w_m c_l s_{lm}
    }
}

// Rounds K_qp (q != p) to the operand type and accumulates the generator diagonal e from the
// rounded values: COLUMN: e_p = sum_{q != p} w_q G_qp / w_p (weighted column sums of K - I are
// zero); ROW: e_q = sum_{p != q} G_qp (rows of K - I sum to zero).  One block per line.
template <typename Store>
__global__ void derive_kernel(const double* __restrict__ K, const double* __restrict__ w, int Q, int norm,
                              Store store, double* __restrict__ e) {
    const int l = blockIdx.x;
    double part = 0.0;
    for (int m = threadIdx.x; m < Q; m += blockDim.x) {
        if (m == l) continue;
        const int q = norm == ASSN_NORM_COLUMN ? m : l;
        const int p = norm == ASSN_NORM_COLUMN ? l : m;
        const double g = store(q, p, K[(size_t)q * Q + p]);    // value actually stored
        part += norm == ASSN_NORM_COLUMN ? w[q] * g : g;
    }
    const double s = block_sum(part);
    if (threadIdx.x == 0) e[l] = norm == ASSN_NORM_COLUMN ? s / w[l] : s;
}

struct StoreF64 {
    double* KT; int Qp;
    __device__ double operator()(int q, int p, double v) const { KT[(size_t)p * Qp + q] = v; return v; }
};
struct StoreF32 {
    float* KT; int Qp;
    __device__ double operator()(int q, int p, double v) const {
        const float f = (float)v;
        KT[(size_t)p * Qp + q] = f;
        return (double)f;
    }
};
struct StoreBF16 {
    __nv_bfloat16* hi; __nv_bfloat16* lo; int Qp;
    __device__ double operator()(int q, int p, double v) const {
        const __nv_bfloat16 h = __double2bfloat16(v);
        double g = (double)__bfloat162float(h);
        hi[(size_t)q * Qp + p] = h;
        if (lo) {
            const __nv_bfloat16 r = __double2bfloat16(v - g);
            lo[(size_t)q * Qp + p] = r;
            g += (double)__bfloat162float(r);
        }
        return g;
    }
};

struct StoreTF32 {
    float* G; int Qp;
    __device__ double operator()(int q, int p, double v) const {
        const float t = tf32_round((float)v);
        G[(size_t)q * Qp + p] = t;
        return (double)t;
    }
};

int line_threads(int Q) { return Q >= 256 ? 256 : (Q >= 128 ? 128 : 64); }

}  // namespace

cudaError_t launch_build_K(const double* omega, const double* w, int Q, double eps, int kind, int norm,
                           double* K64, cudaStream_t s) {
    const double inv = kind == ASSN_KERNEL_GAUSS ? 1.0 / (eps * eps) : 1.0 / (eps * eps);
    build_K_kernel<<<Q, line_threads(Q), 0, s>>>(omega, w, Q, inv, kind, norm, K64);
    return cudaGetLastError();
}

cudaError_t launch_derive_simt_f64(const double* K64, const double* w, int Q, int Qp, int norm, double* KT,
                                   double* e, cudaStream_t s) {
    cudaError_t r = cudaMemsetAsync(KT, 0, sizeof(double) * (size_t)Qp * Qp, s);
    if (r != cudaSuccess) return r;
    derive_kernel<<<Q, line_threads(Q), 0, s>>>(K64, w, Q, norm, StoreF64{KT, Qp}, e);
    return cudaGetLastError();
}

cudaError_t launch_derive_simt_f32(const double* K64, const double* w, int Q, int Qp, int norm, float* KT,
                                   double* e, cudaStream_t s) {
    cudaError_t r = cudaMemsetAsync(KT, 0, sizeof(float) * (size_t)Qp * Qp, s);
    if (r != cudaSuccess) return r;
    derive_kernel<<<Q, line_threads(Q), 0, s>>>(K64, w, Q, norm, StoreF32{KT, Qp}, e);
    return cudaGetLastError();
}

cudaError_t launch_derive_tc(const double* K64, const double* w, int Q, int Qp, int Mp, int norm, bool split,
                             __nv_bfloat16* G_hi, __nv_bfloat16* G_lo, double* e, cudaStream_t s) {
    cudaError_t r = cudaMemsetAsync(G_hi, 0, sizeof(__nv_bfloat16) * (size_t)Mp * Qp, s);
    if (r == cudaSuccess && split) r = cudaMemsetAsync(G_lo, 0, sizeof(__nv_bfloat16) * (size_t)Mp * Qp, s);
    if (r != cudaSuccess) return r;
    derive_kernel<<<Q, line_threads(Q), 0, s>>>(K64, w, Q, norm, StoreBF16{G_hi, split ? G_lo : nullptr, Qp}, e);
    return cudaGetLastError();
}

cudaError_t launch_derive_tf32(const double* K64, const double* w, int Q, int Qp, int Mp, int norm, float* G32,
                               double* e, cudaStream_t s) {
    cudaError_t r = cudaMemsetAsync(G32, 0, sizeof(float) * (size_t)Mp * Qp, s);
    if (r != cudaSuccess) return r;
    derive_kernel<<<Q, line_threads(Q), 0, s>>>(K64, w, Q, norm, StoreTF32{G32, Qp}, e);
    return cudaGetLastError();
}

}  // namespace assn

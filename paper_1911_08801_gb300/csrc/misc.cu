// Diagnostics and state utilities: scalar flux, total mass, finite check, line-source
// initial state, host-layout <-> device-layout conversion.
#include "assn_internal.h"

namespace assn {
namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Phi_c = sum_q w_q psi_q(c): one warp per cell, FP64 accumulation.
template <typename T>
__global__ void scalar_flux_kernel(const T* __restrict__ psi, const T* __restrict__ w, int ncell, int Qp,
                                   float* out_f, double* out_d) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < ncell; c += gridDim.x * wpb) {
        double s = 0.0;
        const T* row = psi + (size_t)c * Qp;
        for (int q = lane; q < Qp; q += 32) s += (double)w[q] * (double)row[q];
        s = warp_sum(s);
        if (lane == 0) {
            if (out_f) out_f[c] = (float)s;
            if (out_d) out_d[c] = s;
        }
    }
}

// Per-block partial sums of sum_c sum_q w_q psi_q(c) into partials[blockIdx.x] (scratch).
template <typename T>
__global__ void mass_partials_kernel(const T* __restrict__ psi, const T* __restrict__ w, int ncell, int Qp,
                                     double* __restrict__ partials) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    double s = 0.0;
    for (int c = blockIdx.x * wpb + wid; c < ncell; c += gridDim.x * wpb) {
        const T* row = psi + (size_t)c * Qp;
        for (int q = lane; q < Qp; q += 32) s += (double)w[q] * (double)row[q];
    }
    s = warp_sum(s);
    if (lane == 0) red[wid] = s;
    __syncthreads();
    if (wid == 0) {
        double t = lane < wpb ? red[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) partials[blockIdx.x] = t;
    }
}

__global__ void reduce_partials_kernel(const double* __restrict__ partials, int n, double* out) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    s = warp_sum(s);
    if (lane == 0) red[wid] = s;
    __syncthreads();
    if (wid == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) *out = t;
    }
}

template <typename T>
__global__ void check_finite_kernel(const T* __restrict__ psi, size_t n, unsigned int* flag) {
    bool bad = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        bad |= !isfinite((double)psi[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// psi_q(x) = max{floor, exp(-|x|^2/(4 delta))/(4 pi delta)} at cell centres (Sec. 4.1).
template <typename T>
__global__ void init_line_source_kernel(T* __restrict__ psi, int nx, int ny, int Q, int Qp, double x0,
                                        double y0, double h, double delta, double floor_value) {
    const size_t n = (size_t)nx * ny * Qp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(i % Qp);
        const size_t c = i / Qp;
        const int ix = (int)(c % nx), jy = (int)(c / nx);
        const double x = x0 + (ix + 0.5) * h, y = y0 + (jy + 0.5) * h;
        const double v = exp(-(x * x + y * y) / (4.0 * delta)) / (4.0 * 3.14159265358979323846 * delta);
        psi[i] = q < Q ? (T)fmax(floor_value, v) : T(0);
    }
}

template <typename T>
__global__ void pack_kernel(const double* __restrict__ src, T* __restrict__ dst, size_t ncell, int Q, int Qp) {
    const size_t n = ncell * Qp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(i % Qp);
        const size_t c = i / Qp;
        dst[i] = q < Q ? (T)src[c * Q + q] : T(0);
    }
}

template <typename T>
__global__ void unpack_kernel(const T* __restrict__ src, double* __restrict__ dst, size_t ncell, int Q, int Qp) {
    const size_t n = ncell * Q;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(i % Q);
        const size_t c = i / Q;
        dst[i] = (double)src[c * Qp + q];
    }
}

int grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

template <typename T>
cudaError_t launch_scalar_flux(const T* psi, const T* w, int ncell, int Qp, float* out_f, double* out_d,
                               cudaStream_t s) {
    scalar_flux_kernel<T><<<grid_for((size_t)ncell * 32, 256), 256, 0, s>>>(psi, w, ncell, Qp, out_f, out_d);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mass_partials(const T* psi, const T* w, int ncell, int Qp, double* partials, int nblocks,
                                 cudaStream_t s) {
    mass_partials_kernel<T><<<nblocks, 256, 0, s>>>(psi, w, ncell, Qp, partials);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partials, int n, double* out, cudaStream_t s) {
    reduce_partials_kernel<<<1, 1024, 0, s>>>(partials, n, out);
    return cudaGetLastError();
}

template <typename T>
__device__ __forceinline__ bool bits_nonzero(T v);
template <>
__device__ __forceinline__ bool bits_nonzero<float>(float v) { return __float_as_uint(v) != 0u; }
template <>
__device__ __forceinline__ bool bits_nonzero<double>(double v) { return __double_as_longlong(v) != 0ll; }

// Counts the padded ordinates (Q <= q < Qp) of a state buffer whose bits are not all zero.
template <typename T>
__global__ void padding_nonzero_kernel(const T* psi, size_t ncell, int Q, int Qp, unsigned long long* count) {
    const int pad = Qp - Q;
    const size_t n = ncell * (size_t)pad;
    unsigned long long local = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t c = i / (size_t)pad;
        const int q = Q + (int)(i - c * (size_t)pad);
        if (bits_nonzero<T>(psi[c * (size_t)Qp + q])) ++local;
    }
    if (local) atomicAdd(count, local);
}

template <typename T>
cudaError_t launch_padding_nonzero(const T* psi, size_t ncell, int Q, int Qp, unsigned long long* count,
                                   cudaStream_t s) {
    if (Qp <= Q || ncell == 0) return cudaSuccess;
    padding_nonzero_kernel<T><<<grid_for(ncell * (size_t)(Qp - Q), 256), 256, 0, s>>>(psi, ncell, Q, Qp, count);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_check_finite(const T* psi, size_t n, unsigned int* flag, cudaStream_t s) {
    check_finite_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(psi, n, flag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_line_source(T* psi, int nx, int ny, int Q, int Qp, double x0, double y0, double h,
                                    double delta, double floor_value, cudaStream_t s) {
    init_line_source_kernel<T><<<grid_for((size_t)nx * ny * Qp, 256), 256, 0, s>>>(psi, nx, ny, Q, Qp, x0, y0, h,
                                                                                  delta, floor_value);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack_state(const double* src, T* dst, size_t ncell, int Q, int Qp, cudaStream_t s) {
    pack_kernel<T><<<grid_for(ncell * Qp, 256), 256, 0, s>>>(src, dst, ncell, Q, Qp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack_state(const T* src, double* dst, size_t ncell, int Q, int Qp, cudaStream_t s) {
    unpack_kernel<T><<<grid_for(ncell * Q, 256), 256, 0, s>>>(src, dst, ncell, Q, Qp);
    return cudaGetLastError();
}

#define ASSN_INSTANTIATE(T)                                                                                   \
    template cudaError_t launch_scalar_flux<T>(const T*, const T*, int, int, float*, double*, cudaStream_t);  \
    template cudaError_t launch_mass_partials<T>(const T*, const T*, int, int, double*, int, cudaStream_t);   \
    template cudaError_t launch_check_finite<T>(const T*, size_t, unsigned int*, cudaStream_t);              \
    template cudaError_t launch_padding_nonzero<T>(const T*, size_t, int, int, unsigned long long*, cudaStream_t); \
    template cudaError_t launch_init_line_source<T>(T*, int, int, int, int, double, double, double, double,   \
                                                    double, cudaStream_t);                                    \
    template cudaError_t launch_pack_state<T>(const double*, T*, size_t, int, int, cudaStream_t);            \
    template cudaError_t launch_unpack_state<T>(const T*, double*, size_t, int, int, cudaStream_t);
ASSN_INSTANTIATE(float)
ASSN_INSTANTIATE(double)

}  // namespace assn

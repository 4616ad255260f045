// Fused as-S_N step on CUDA cores, FP64 (the plain FP64 GPU path) and FP32.
//
// One block owns a tile of TN consecutive cells of one grid row plus their two x-neighbours
// and all Qp ordinates, staged in shared memory.  Threads own ordinates: thread q forms
//   Y_q(c) = sum_{p != q} K_qp psi_p(c)                     (artificial in-scattering, Sec. 3.2)
// for the TN cells of the tile, then applies upwind transport, collision, isotropic scattering
// and the source to produce psi^{n+1} (Sec. 3.1-3.2, forward Euler).
#include "assn_internal.h"

namespace assn {
namespace {

template <typename T> struct Q4 { T x, y, z, w; };
__device__ __forceinline__ Q4<float> load4(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Q4<double> load4(const double* p) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    return {a.x, a.y, b.x, b.y};
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, typename OrdT, typename CellT, int TN>
__global__ void __launch_bounds__(256)
step_simt_kernel(const StepArgs<T, OrdT, CellT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Qp = a.Qp, nx = a.nx;
    T* ps = reinterpret_cast<T*>(smem_raw);   // [(TN+2)][Qp], slot s <-> cell x0 - 1 + s
    T* phi = ps + (size_t)(TN + 2) * Qp;      // [TN]
    const int j = blockIdx.y;
    const int x0 = blockIdx.x * TN;
    const int nt = min(TN, nx - x0);
    const size_t row = (size_t)j * nx;

    for (int idx = threadIdx.x; idx < (TN + 2) * Qp; idx += blockDim.x) {
        const int sl = idx / Qp, q = idx - sl * Qp;
        const int x = x0 - 1 + sl;
        ps[idx] = (x >= 0 && x < nx) ? a.psi[(row + x) * Qp + q] : T(0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int c = warp; c < nt; c += nwarps) {
        T s = 0;
        for (int q = lane; q < Qp; q += 32) s += a.ord[q].w * ps[(size_t)(c + 1) * Qp + q];
        s = warp_sum(s);
        if (lane == 0) phi[c] = s;
    }
    __syncthreads();

    for (int q = threadIdx.x; q < Qp; q += blockDim.x) {
        if (q >= a.Q) {   // padded ordinates stay zero
            for (int c = 0; c < nt; ++c) a.psi_out[(row + x0 + c) * Qp + q] = T(0);
            continue;
        }
        T acc[TN];
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[c] = 0;
        for (int p = 0; p < Qp; p += 4) {
            const T k0 = a.KT[(size_t)(p + 0) * Qp + q];
            const T k1 = a.KT[(size_t)(p + 1) * Qp + q];
            const T k2 = a.KT[(size_t)(p + 2) * Qp + q];
            const T k3 = a.KT[(size_t)(p + 3) * Qp + q];
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const Q4<T> v = load4(ps + (size_t)(c + 1) * Qp + p);
                acc[c] += k0 * v.x + k1 * v.y + k2 * v.z + k3 * v.w;
            }
        }
        const OrdT o = a.ord[q];
        const T ax = o.nux > 0 ? o.nux : -o.nux;
        const T ay = o.nuy > 0 ? o.nuy : -o.nuy;
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            if (c >= nt) break;
            const int x = x0 + c;
            const T self = ps[(size_t)(c + 1) * Qp + q];
            const T upx = o.nux > 0 ? ps[(size_t)c * Qp + q] : (o.nux < 0 ? ps[(size_t)(c + 2) * Qp + q] : T(0));
            T upy = 0;
            if (o.nuy > 0 && j > 0) upy = a.psi[(row - nx + x) * Qp + q];
            else if (o.nuy < 0 && j + 1 < a.ny) upy = a.psi[(row + nx + x) * Qp + q];
            const CellT cl = a.cell[row + x];
            const T out = self - ax * (self - upx) - ay * (self - upy) - a.dt * cl.sig_t * self +
                          a.dt * (cl.sig_s_over_wsum * phi[c] + cl.q) +
                          a.dt_sigma_as * (acc[c] - o.e * self);
            a.psi_out[(row + x) * Qp + q] = out;
        }
    }
}

template <typename T>
__device__ __forceinline__ T minmod(T a, T b) {
    return a * b > T(0) ? (fabs(a) < fabs(b) ? a : b) : T(0);
}

// Flux difference F_{i+1/2} - F_{i-1/2} (in units of the face value) of the limited upwind scheme
// for one ordinate along one axis, from the values at i-2 .. i+2 (zero beyond the domain):
// nu > 0 takes face values psi_i + D_i / 2 (D = minmod of the one-sided differences); nu < 0
// takes psi_{i+1} - D_{i+1} / 2.
template <typename T>
__device__ __forceinline__ T limited_difference(T nu, T m2, T m1, T c0, T p1, T p2) {
    if (nu > T(0)) {
        const T fp = c0 + T(0.5) * minmod(c0 - m1, p1 - c0);
        const T fm = m1 + T(0.5) * minmod(m1 - m2, c0 - m1);
        return fp - fm;
    }
    if (nu < T(0)) {
        const T fp = p1 - T(0.5) * minmod(p1 - c0, p2 - p1);
        const T fm = c0 - T(0.5) * minmod(c0 - m1, p1 - c0);
        return fp - fm;
    }
    return T(0);
}

// Heun stage on CUDA cores (the paper's explicit scheme, Sec. 3.1; Sec. 3.2 operator).  Tile of TN
// cells of one row plus two x-neighbours on each side in shared memory; threads own ordinates.
template <typename T, typename OrdT, typename CellT, int TN>
__global__ void __launch_bounds__(256)
stage_simt_kernel(const StepArgs<T, OrdT, CellT> a, const T* keep, T alpha, T beta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Qp = a.Qp, nx = a.nx, ny = a.ny;
    T* ps = reinterpret_cast<T*>(smem_raw);   // [(TN+4)][Qp], slot s <-> cell x0 - 2 + s
    T* phi = ps + (size_t)(TN + 4) * Qp;      // [TN]
    const int j = blockIdx.y;
    const int x0 = blockIdx.x * TN;
    const int nt = min(TN, nx - x0);
    const size_t row = (size_t)j * nx;

    for (int idx = threadIdx.x; idx < (TN + 4) * Qp; idx += blockDim.x) {
        const int sl = idx / Qp, q = idx - sl * Qp;
        const int x = x0 - 2 + sl;
        ps[idx] = (x >= 0 && x < nx) ? a.psi[(row + x) * Qp + q] : T(0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int c = warp; c < nt; c += nwarps) {
        T s = 0;
        for (int q = lane; q < Qp; q += 32) s += a.ord[q].w * ps[(size_t)(c + 2) * Qp + q];
        s = warp_sum(s);
        if (lane == 0) phi[c] = s;
    }
    __syncthreads();

    for (int q = threadIdx.x; q < Qp; q += blockDim.x) {
        if (q >= a.Q) {
            for (int c = 0; c < nt; ++c) a.psi_out[(row + x0 + c) * Qp + q] = T(0);
            continue;
        }
        T acc[TN];
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[c] = 0;
        for (int p = 0; p < Qp; p += 4) {
            const T k0 = a.KT[(size_t)(p + 0) * Qp + q];
            const T k1 = a.KT[(size_t)(p + 1) * Qp + q];
            const T k2 = a.KT[(size_t)(p + 2) * Qp + q];
            const T k3 = a.KT[(size_t)(p + 3) * Qp + q];
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const Q4<T> v = load4(ps + (size_t)(c + 2) * Qp + p);
                acc[c] += k0 * v.x + k1 * v.y + k2 * v.z + k3 * v.w;
            }
        }
        const OrdT o = a.ord[q];
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            if (c >= nt) break;
            const int x = x0 + c;
            const T* col = ps + (size_t)(c + 2) * Qp + q;
            const T self = col[0];
            const T tx = limited_difference<T>(o.nux, col[-2 * Qp], col[-Qp], self, col[Qp], col[2 * Qp]);
            T ym2 = 0, ym1 = 0, yp1 = 0, yp2 = 0;
            if (o.nuy != T(0)) {
                const T* g = a.psi + (row + x) * Qp + q;
                const size_t sy = (size_t)nx * Qp;
                if (j >= 2) ym2 = g[-2 * (long)sy];
                if (j >= 1) ym1 = g[-(long)sy];
                if (j + 1 < ny) yp1 = g[sy];
                if (j + 2 < ny) yp2 = g[2 * sy];
            }
            const T ty = limited_difference<T>(o.nuy, ym2, ym1, self, yp1, yp2);
            const CellT cl = a.cell[row + x];
            const T adv = self - o.nux * tx - o.nuy * ty - a.dt * cl.sig_t * self +
                          a.dt * (cl.sig_s_over_wsum * phi[c] + cl.q) + a.dt_sigma_as * (acc[c] - o.e * self);
            T out = beta * adv;
            if (alpha != T(0)) out += alpha * keep[(row + x) * Qp + q];
            a.psi_out[(row + x) * Qp + q] = out;
        }
    }
}

template <typename T, typename OrdT, typename CellT, int TN>
cudaError_t launch_stage(const StepArgs<T, OrdT, CellT>& a, const T* keep, T alpha, T beta, cudaStream_t s) {
    const size_t smem = sizeof(T) * ((size_t)(TN + 4) * a.Qp + TN);
    auto kern = stage_simt_kernel<T, OrdT, CellT, TN>;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r != cudaSuccess) return r;
    dim3 grid((a.nx + TN - 1) / TN, a.ny);
    kern<<<grid, 256, smem, s>>>(a, keep, alpha, beta);
    return cudaGetLastError();
}

template <typename T, typename OrdT, typename CellT, int TN>
cudaError_t launch_simt(const StepArgs<T, OrdT, CellT>& a, cudaStream_t s) {
    const size_t smem = sizeof(T) * ((size_t)(TN + 2) * a.Qp + TN);
    auto kern = step_simt_kernel<T, OrdT, CellT, TN>;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (r != cudaSuccess) return r;
    dim3 grid((a.nx + TN - 1) / TN, a.ny);
    kern<<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_simt_f64(const StepArgs<double, OrdD, CellD>& a, cudaStream_t s) {
    return launch_simt<double, OrdD, CellD, 8>(a, s);
}

cudaError_t launch_step_simt_f32(const StepArgs<float, OrdF, CellF>& a, cudaStream_t s) {
    return launch_simt<float, OrdF, CellF, 16>(a, s);
}

cudaError_t launch_stage_simt_f64(const StepArgs<double, OrdD, CellD>& a, const double* keep, double alpha,
                                  double beta, cudaStream_t s) {
    return launch_stage<double, OrdD, CellD, 8>(a, keep, alpha, beta, s);
}

cudaError_t launch_stage_simt_f32(const StepArgs<float, OrdF, CellF>& a, const float* keep, float alpha,
                                  float beta, cudaStream_t s) {
    return launch_stage<float, OrdF, CellF, 16>(a, keep, alpha, beta, s);
}

}  // namespace assn

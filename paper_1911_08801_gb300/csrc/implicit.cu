// Implicit as-S_N time step (Sec. 3.4-3.5, Alg. 1-3): implicit Euler with the second-order upwind
// stencil without limiter, solved by the sweeping-Krylov method on CUDA cores (FP64 and FP32 state).
//
// With lx = |Omega_x| dt / h, ly = |Omega_y| dt / h and sigma_tot = sigma_a + sigma_s + sigma_as, the
// streaming operator times dt is
//   (L psi)_c = lx (3/2 psi_c - 2 psi_{c-x} + 1/2 psi_{c-2x}) + ly (...) + (1 + dt sigma_tot) psi_c
// (c-x, c-2x the upwind neighbours, zero outside the grid), and a step solves
//   L psi - dt (sigma_s Phi / sum w + sigma_as K psi) = dt q + psi_old.
//
//   source iteration (Alg. 1)   psi^{l+1} = L^{-1} S,  S = dt (sigma_as K psi^l + R), until
//                               ||psi^{l+1} - psi^l||_2 < eps (1 - T) / T (FP32 state: also when the
//                               difference stops falling, the rounding floor of the state)
//   GMRES (Alg. 2-3)            on the scalar flux phi (isotropic physical scattering: one moment);
//                               FP32 state: relative tolerance not below 2^-20
//
// Kernels: si_source_kernel forms S (the artificial in-scattering contraction on CUDA cores, the
// layout of the explicit CUDA-core step: a tile of cells of one row in shared memory, threads own
// ordinates); the sweeps invert L: one block per chunk of up to kChunk ordinates of one quadrant
// (sign of Omega_x, Omega_y), which walks the anti-diagonals of the grid in the upwind order of that
// quadrant -- every cell needs only its two upwind neighbours in x and y, which lie on the two
// previous anti-diagonals -- with a block barrier between anti-diagonals.  sweep_rows_kernel (grids
// up to 2048 rows) gives every row its own thread, so x-neighbours stay in registers and y-neighbours
// come from a ring of anti-diagonals in shared memory, and it also sums the convergence norm;
// sweep_kernel (any grid) reads all neighbours back from memory.  One ordinate per block, so a sweep
// spreads over up to Q SMs and each block's barrier joins few warps.  GMRES runs on the host over device
// vectors of one value per cell.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "assn.h"
#include "problem.h"
#include "trace.h"

namespace assn {

struct ImplicitWork {
    void* buf[3] = {nullptr, nullptr, nullptr};   // two iterates and the sweep source, [ncell][Qp]
    void* rtmp[2] = {nullptr, nullptr};           // caller right-hand side and start (diagnostic entry)
    size_t buf_bytes = 0;                         // size of each of buf / rtmp
    int* d_chunks = nullptr;                      // [nchunks][kChunk] ordinates, -1 padding
    int nchunks = 0;
    std::vector<int> chunk_quads;                 // quadrant of every ordinate the table was built for
    double* V = nullptr;                          // GMRES basis, (restart + 1) x ncell
    double* vec = nullptr;                        // x, b, w, t: 4 x ncell
    int restart_alloc = 0;
    double* d_part = nullptr;                     // reduction partials
    double* d_red = nullptr;                      // reduction results
    double* h_red = nullptr;                      // pinned host copy of one result
    double si_eps = 1e-4, gmres_tol = 1.5e-8;
    double lip_dt = -1.0, lip = 0.0;              // the source iteration's T for one dt
    int restart = 30, max_si = 1000, max_gmres = 500;
    long long si_total = 0, gmres_total = 0, sweeps_total = 0;
    int last_si_converged = 1, last_gmres_converged = 1;
};

namespace {

constexpr int kChunk = 1;          // ordinates per sweep block (one: the ordinates spread over the SMs)
constexpr int kSweepThreads = 256; // general sweep kernel
constexpr int kRowBlock = 512;     // row-per-thread sweep kernel: at most this many threads per block
constexpr int kTN = 8;             // cells per source-kernel tile
constexpr int kRedBlocks = 304;    // reduction partials (2 per SM)
constexpr int kPartMax = ASSN_MAX_Q;   // partial sums held: reductions and one per sweep block

int blocks_for(size_t n, int threads) {
    const size_t b = (n + threads - 1) / threads;
    return (int)std::min<size_t>(std::max<size_t>(b, 1), 1u << 20);
}

// ------------------------------------------------------------------------------------- kernels
template <typename T> struct Vec4 { T x, y, z, w; };
__device__ __forceinline__ Vec4<float> load_vec4(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Vec4<double> load_vec4(const double* p) {
    const double2 u = *reinterpret_cast<const double2*>(p);
    const double2 v = *reinterpret_cast<const double2*>(p + 2);
    return {u.x, u.y, v.x, v.y};
}

template <typename T, typename OrdT, typename CellT>
struct SourceArgs {
    const T* psi;            // iterate psi^l [ncell][Qp]
    T* S;                    // out: dt (sigma_as K psi + R) [ncell][Qp]
    const T* KT;             // off-diagonal K transposed: KT[p * Qp + q] = G_qp
    const OrdT* ord;         // per ordinate: e (generator diagonal, K_qq = 1 - e)
    const CellT* cell;
    const double* phi;       // nullable: R += sigma_s phi / sum w
    const T* old;            // nullable: R += old / dt
    const T* rarr;           // nullable: R += rarr
    int withq;               // R += q
    int nx, ny, Q, Qp;
    T dt, sigma_as;
};

template <typename T, typename OrdT, typename CellT>
__global__ void __launch_bounds__(256) si_source_kernel(const SourceArgs<T, OrdT, CellT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* ps = reinterpret_cast<T*>(smem_raw);     // [kTN][Qp]
    const int Qp = a.Qp, nx = a.nx;
    const int j = blockIdx.y, x0 = blockIdx.x * kTN;
    const int nt = min(kTN, nx - x0);
    const size_t row = (size_t)j * nx;
    for (int idx = threadIdx.x; idx < kTN * Qp; idx += blockDim.x) {
        const int c = idx / Qp;
        ps[idx] = c < nt ? a.psi[(row + x0) * Qp + idx] : T(0);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < a.Q; q += blockDim.x) {
        T acc[kTN];
#pragma unroll
        for (int c = 0; c < kTN; ++c) acc[c] = 0;
        if (a.sigma_as != T(0)) {
            // four ordinates p at a time: one 16-byte (FP32) or two (FP64) shared loads per cell
            for (int p = 0; p < Qp; p += 4) {
                const T k0 = a.KT[(size_t)(p + 0) * Qp + q], k1 = a.KT[(size_t)(p + 1) * Qp + q];
                const T k2 = a.KT[(size_t)(p + 2) * Qp + q], k3 = a.KT[(size_t)(p + 3) * Qp + q];
#pragma unroll
                for (int c = 0; c < kTN; ++c) {
                    const Vec4<T> v = load_vec4(ps + c * Qp + p);
                    acc[c] += k0 * v.x + k1 * v.y + k2 * v.z + k3 * v.w;
                }
            }
        }
        const T kqq = T(1) - a.ord[q].e;
#pragma unroll
        for (int c = 0; c < kTN; ++c) {
            if (c >= nt) break;
            const size_t cell = row + x0 + c;
            const size_t idx = cell * Qp + q;
            const CellT cl = a.cell[cell];
            T r = a.withq ? (T)cl.q : T(0);
            if (a.phi) r += (T)cl.sig_s_over_wsum * (T)a.phi[cell];
            if (a.rarr) r += a.rarr[idx];
            T s = a.dt * (a.sigma_as * (acc[c] + kqq * ps[c * Qp + q]) + r);
            if (a.old) s += a.old[idx];
            a.S[idx] = s;
        }
    }
}

template <typename T, typename OrdT, typename CellT>
struct SweepArgs {
    const T* S;              // [ncell][Qp]
    T* out;                  // [ncell][Qp] (only real ordinates written)
    const OrdT* ord;         // nux = dt Omega_x / h, nuy = dt Omega_y / h
    const CellT* cell;       // sig_t = sigma_a + sigma_s
    const int* chunks;       // [nchunks][kChunk]
    const T* prev;           // nullable: the previous iterate, for sum (out - prev)^2
    double* part;            // [nchunks] per-block sums of (out - prev)^2 (when prev is set)
    int nx, ny, Qp;
    T dt, sigma_as;
};

template <typename T, typename OrdT, typename CellT>
__global__ void __launch_bounds__(kSweepThreads) sweep_kernel(const SweepArgs<T, OrdT, CellT> a) {
    const int k = threadIdx.x % kChunk, slot = threadIdx.x / kChunk;
    constexpr int nslot = kSweepThreads / kChunk;
    const int* ch = a.chunks + blockIdx.x * kChunk;
    const int q = ch[k];
    const OrdT o0 = a.ord[ch[0]];
    const int sx = o0.nux >= 0 ? 1 : -1, sy = o0.nuy >= 0 ? 1 : -1;   // the chunk's quadrant
    T ax = 0, ay = 0;
    if (q >= 0) {
        const OrdT o = a.ord[q];
        ax = o.nux >= 0 ? (T)o.nux : -(T)o.nux;
        ay = o.nuy >= 0 ? (T)o.nuy : -(T)o.nuy;
    }
    const T lead = T(1.5) * (ax + ay) + T(1);
    const int nx = a.nx, ny = a.ny, Qp = a.Qp;
    const ptrdiff_t dx = (ptrdiff_t)sx * Qp, dy = (ptrdiff_t)sy * nx * Qp;
    for (int d = 0; d < nx + ny - 1; ++d) {
        if (q >= 0) {
            const int b0 = max(0, d - (nx - 1)), b1 = min(d, ny - 1);
            for (int b = b0 + slot; b <= b1; b += nslot) {
                const int u = d - b;                                   // upwind-ordered column
                const int i = sx > 0 ? u : nx - 1 - u, jj = sy > 0 ? b : ny - 1 - b;
                const size_t c = (size_t)jj * nx + i;
                const ptrdiff_t idx = (ptrdiff_t)(c * Qp + q);
                const T x1 = u >= 1 ? a.out[idx - dx] : T(0);
                const T x2 = u >= 2 ? a.out[idx - 2 * dx] : T(0);
                const T y1 = b >= 1 ? a.out[idx - dy] : T(0);
                const T y2 = b >= 2 ? a.out[idx - 2 * dy] : T(0);
                const T den = lead + a.dt * ((T)a.cell[c].sig_t + a.sigma_as);
                a.out[idx] = (a.S[idx] + ax * (T(2) * x1 - T(0.5) * x2) + ay * (T(2) * y1 - T(0.5) * y2)) / den;
            }
        }
        __syncthreads();
    }
}

// The sweep with one thread per (row of the grid, ordinate), RPT rows per thread: in the upwind-ordered
// frame row b reaches anti-diagonal d at column u = d - b, so a thread meets its row's cells in order
// and keeps their two upwind x-neighbours in registers; the y-neighbours, computed one and two
// anti-diagonals earlier by the threads of rows b - 1 and b - 2, come from a three-deep ring of
// anti-diagonals in shared memory.  The source term and stencil diagonal of a thread's cells are
// loaded three anti-diagonals before their use.  With prev set, the block also sums (out - prev)^2.
template <typename T, typename OrdT, typename CellT, int RPT>
__global__ void __launch_bounds__(kRowBlock) sweep_rows_kernel(const SweepArgs<T, OrdT, CellT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kRowBlock / 32];
    const int nx = a.nx, ny = a.ny, Qp = a.Qp;
    T* ring = reinterpret_cast<T*>(smem_raw);                          // [3][ny][kChunk]
    const int k = threadIdx.x % kChunk, rt = threadIdx.x / kChunk;
    const int nrow = blockDim.x / kChunk;                               // rows handled at once
    const int* ch = a.chunks + blockIdx.x * kChunk;
    const int q = ch[k];
    const OrdT o0 = a.ord[ch[0]];
    const int sx = o0.nux >= 0 ? 1 : -1, sy = o0.nuy >= 0 ? 1 : -1;   // the chunk's quadrant
    T ax = 0, ay = 0;
    if (q >= 0) {
        const OrdT o = a.ord[q];
        ax = o.nux >= 0 ? (T)o.nux : -(T)o.nux;
        ay = o.nuy >= 0 ? (T)o.nuy : -(T)o.nuy;
    }
    const T lead = T(1.5) * (ax + ay) + T(1);
    // Per row: the x-neighbours in registers, and four sets of the cell of anti-diagonals d .. d + 3
    // (index, source term, sigma_a + sigma_s, previous iterate): set d % 4 is loaded when anti-diagonal
    // d - 4 is done, three anti-diagonals before its use.  The loop is unrolled by four so the sets
    // stay in registers.
    using Set = struct {
        T sn[RPT], sg[RPT], pv[RPT];
        ptrdiff_t ix[RPT];
    };
    T x1[RPT], x2[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) x1[r] = x2[r] = T(0);
    Set s0, s1, s2, s3;
    double d2 = 0;
    auto fetch = [&](int d, Set& z) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int b = rt + r * nrow, u = d - b;
            z.ix[r] = -1;
            z.sn[r] = z.pv[r] = z.sg[r] = T(0);
            if (q >= 0 && b < ny && u >= 0 && u < nx) {
                const int i = sx > 0 ? u : nx - 1 - u, jj = sy > 0 ? b : ny - 1 - b;
                const size_t c = (size_t)jj * nx + i;
                z.ix[r] = (ptrdiff_t)(c * Qp + q);
                z.sn[r] = a.S[z.ix[r]];
                z.sg[r] = (T)a.cell[c].sig_t;        // only loaded here: used three anti-diagonals later
                if (a.prev) z.pv[r] = a.prev[z.ix[r]];
            }
        }
    };
    const int nd = nx + ny - 1;
    int cs = 0;                                                         // ring slot of anti-diagonal d
    // one anti-diagonal with the cells of set z, then z takes anti-diagonal d + 4
    auto step = [&](int d, Set& z) {
        const int r1 = cs == 0 ? 2 : cs - 1, r2 = cs == 2 ? 0 : cs + 1;  // slots of d - 1, d - 2
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (z.ix[r] < 0) continue;
            const int b = rt + r * nrow;
            const T y1 = b >= 1 ? ring[((size_t)r1 * ny + b - 1) * kChunk + k] : T(0);
            const T y2 = b >= 2 ? ring[((size_t)r2 * ny + b - 2) * kChunk + k] : T(0);
            const T den = lead + a.dt * (z.sg[r] + a.sigma_as);
            const T v = (z.sn[r] + ax * (T(2) * x1[r] - T(0.5) * x2[r]) + ay * (T(2) * y1 - T(0.5) * y2)) / den;
            a.out[z.ix[r]] = v;
            ring[((size_t)cs * ny + b) * kChunk + k] = v;
            if (a.prev) {
                const double e = (double)v - (double)z.pv[r];
                d2 += e * e;
            }
            x2[r] = x1[r];
            x1[r] = v;
        }
        fetch(d + 4, z);
        __syncthreads();
        cs = cs == 2 ? 0 : cs + 1;
    };
    fetch(0, s0);
    fetch(1, s1);
    fetch(2, s2);
    fetch(3, s3);
    for (int d = 0; d < nd; d += 4) {                                   // d < nd is uniform in the block
        step(d, s0);
        if (d + 1 < nd) step(d + 1, s1);
        if (d + 2 < nd) step(d + 2, s2);
        if (d + 3 < nd) step(d + 3, s3);
    }
    if (a.prev) {
        for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d2;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            a.part[blockIdx.x] = t;
        }
    }
}

// sum over all elements of (x - y)^2: per-block partials
template <typename T>
__global__ void __launch_bounds__(256) sqdiff_partials(const T* x, const T* y, size_t n, double* part) {
    __shared__ double sh[256];
    double s = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double d = (double)x[i] - (double)y[i];
        s += d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) dot_partials(const double* x, const double* y, size_t n, double* part) {
    __shared__ double sh[256];
    double s = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        s += x[i] * y[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) finish_sum(const double* part, int n, double* out) {
    __shared__ double sh[256];
    double s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// y = alpha x + beta y
__global__ void __launch_bounds__(256) axpby(double alpha, const double* x, double beta, double* y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = alpha * x[i] + beta * y[i];
}

// y = alpha x (y's old contents are not read)
__global__ void __launch_bounds__(256) scale_copy(double alpha, const double* x, double* y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = alpha * x[i];
}

// ------------------------------------------------------------------------------------- host side
template <typename T> struct Types;
template <> struct Types<double> { using Ord = OrdD; using Cell = CellD; };
template <> struct Types<float> { using Ord = OrdF; using Cell = CellF; };

#define ICK(p, call)                                                                                 \
    do {                                                                                             \
        cudaError_t _e = (call);                                                                     \
        if (_e != cudaSuccess)                                                                       \
            return problem_fail((p), _e == cudaErrorMemoryAllocation ? ASSN_ERR_OOM : ASSN_ERR_CUDA,  \
                                cudaGetErrorString(_e));                                             \
    } while (0)

int ensure_work(assn_problem* p) {
    if (!p->impl) p->impl = new ImplicitWork();
    ImplicitWork* W = p->impl;
    const size_t ncell = p->ncell(), n = ncell * p->Qp;
    if (W->buf_bytes != n * p->elem()) {             // first use, or the quadrature changed Qp
        ICK(p, cudaStreamSynchronize(p->stream));
        for (auto*& b : W->buf) {
            if (b) cudaFree(b);
            b = nullptr;
        }
        for (auto*& b : W->rtmp) {
            if (b) cudaFree(b);
            b = nullptr;
        }
        W->buf_bytes = 0;
        for (int b = 0; b < 3; ++b) {
            ICK(p, cudaMalloc(&W->buf[b], n * p->elem()));
            ICK(p, cudaMemsetAsync(W->buf[b], 0, n * p->elem(), p->stream));   // padded ordinates stay 0
        }
        W->buf_bytes = n * p->elem();
    }
    if (!W->vec) {
        ICK(p, cudaMalloc(&W->vec, 4 * ncell * sizeof(double)));
        ICK(p, cudaMalloc(&W->d_part, kPartMax * sizeof(double)));
        ICK(p, cudaMalloc(&W->d_red, sizeof(double)));
        ICK(p, cudaMallocHost(&W->h_red, sizeof(double)));
    }
    if (W->restart_alloc < W->restart) {
        if (W->V) cudaFree(W->V);
        W->V = nullptr;
        ICK(p, cudaMalloc(&W->V, (size_t)(W->restart + 1) * ncell * sizeof(double)));
        W->restart_alloc = W->restart;
    }
    // quadrant of each ordinate (a zero component counts as positive)
    std::vector<int> quads(p->Q);
    for (int q = 0; q < p->Q; ++q) quads[q] = (p->omega[3 * q] >= 0 ? 0 : 1) | (p->omega[3 * q + 1] >= 0 ? 0 : 2);
    if (quads != W->chunk_quads) {
        // ordinates grouped by quadrant, kChunk per block
        std::vector<int> table;
        for (int quad = 0; quad < 4; ++quad) {
            std::vector<int> sel;
            for (int q = 0; q < p->Q; ++q)
                if (quads[q] == quad) sel.push_back(q);
            for (size_t s = 0; s < sel.size(); s += kChunk)
                for (int k = 0; k < kChunk; ++k) table.push_back(s + k < sel.size() ? sel[s + k] : -1);
        }
        if (W->d_chunks) cudaFree(W->d_chunks);
        W->d_chunks = nullptr;
        ICK(p, cudaMalloc(&W->d_chunks, table.size() * sizeof(int)));
        ICK(p, cudaMemcpyAsync(W->d_chunks, table.data(), table.size() * sizeof(int), cudaMemcpyHostToDevice,
                               p->stream));
        ICK(p, cudaStreamSynchronize(p->stream));
        W->nchunks = (int)(table.size() / kChunk);
        W->chunk_quads = quads;
    }
    return ASSN_OK;
}

// The source iteration's contraction factor estimate T (artificial gain over the removal rate of a
// cell, at its largest), cached per dt.
double lipschitz(assn_problem* p, double dt) {
    ImplicitWork* W = p->impl;
    if (W->lip_dt != dt) {
        double t = 0;
        for (size_t c = 0; c < p->ncell(); ++c)
            t = std::max(t, dt * p->sigma_as / (1.0 + dt * (p->sa[c] + p->ss[c] + p->sigma_as)));
        W->lip = t;
        W->lip_dt = dt;
    }
    return W->lip;
}

int read_sum(assn_problem* p, double* out, int nparts = kRedBlocks) {
    ImplicitWork* W = p->impl;
    finish_sum<<<1, 256, 0, p->stream>>>(W->d_part, nparts, W->d_red);
    ICK(p, cudaGetLastError());
    ++p->launches;
    ICK(p, cudaMemcpyAsync(W->h_red, W->d_red, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    ICK(p, cudaStreamSynchronize(p->stream));
    *out = *W->h_red;
    return ASSN_OK;
}

int dot(assn_problem* p, const double* x, const double* y, double* out) {
    dot_partials<<<kRedBlocks, 256, 0, p->stream>>>(x, y, p->ncell(), p->impl->d_part);
    ICK(p, cudaGetLastError());
    ++p->launches;
    return read_sum(p, out);
}

int lincomb(assn_problem* p, double alpha, const double* x, double beta, double* y) {
    axpby<<<blocks_for(p->ncell(), 256), 256, 0, p->stream>>>(alpha, x, beta, y, p->ncell());
    ICK(p, cudaGetLastError());
    ++p->launches;
    return ASSN_OK;
}

int scale(assn_problem* p, double alpha, const double* x, double* y) {
    scale_copy<<<blocks_for(p->ncell(), 256), 256, 0, p->stream>>>(alpha, x, y, p->ncell());
    ICK(p, cudaGetLastError());
    ++p->launches;
    return ASSN_OK;
}

// Right-hand side of a source iteration: phi (scattering of a scalar flux), q, old / dt, rarr.
struct Rhs {
    const double* phi = nullptr;
    int withq = 0;
    bool old = false;
    const void* rarr = nullptr;
};

// Alg. 1 from psi0 (device, [ncell][Qp]); fixed > 0 runs exactly that many iterations.  *result is
// one of the work buffers.
template <typename T>
int source_iteration(assn_problem* p, double dt, const Rhs& R, const void* psi0, int fixed, const void** result) {
    using Ord = typename Types<T>::Ord;
    using Cell = typename Types<T>::Cell;
    ImplicitWork* W = p->impl;
    const double Tl = lipschitz(p, dt);
    const double tol = Tl > 0 ? W->si_eps * (1.0 - Tl) / Tl : 0.0;
    const T* KT = std::is_same<T, double>::value ? (const T*)p->d_KT64 : (const T*)(const void*)p->d_KT32;
    const void* cur = psi0;
    int out = 0, it = 0;
    const dim3 sgrid((p->nx + kTN - 1) / kTN, p->ny);
    const size_t smem = (size_t)kTN * p->Qp * sizeof(T);
    if (smem > 48 * 1024)
        ICK(p, cudaFuncSetAttribute(si_source_kernel<T, Ord, Cell>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    const size_t n = p->ncell() * p->Qp;
    // row-per-thread sweep (rows per thread RPT) where its ring of three anti-diagonals fits
    const int ny = p->ny;
    const int rpt = ny <= kRowBlock ? 1 : ny <= 2 * kRowBlock ? 2 : ny <= 4 * kRowBlock ? 4 : 0;
    const int row_threads = rpt ? ((ny + rpt - 1) / rpt * kChunk + 31) / 32 * 32 : 0;
    const size_t ring = (size_t)3 * ny * kChunk * sizeof(T);
    const bool rows = rpt > 0 && ring <= 200 * 1024;
    if (rows && ring > 48 * 1024) {
        auto set = [&](const void* f) { return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring); };
        cudaError_t e = rpt == 1 ? set((const void*)sweep_rows_kernel<T, Ord, Cell, 1>)
                      : rpt == 2 ? set((const void*)sweep_rows_kernel<T, Ord, Cell, 2>)
                                 : set((const void*)sweep_rows_kernel<T, Ord, Cell, 4>);
        ICK(p, e);
    }
    W->last_si_converged = 1;
    double prev_d2 = INFINITY;
    while (true) {
        SourceArgs<T, Ord, Cell> sa{(const T*)cur, (T*)W->buf[2], KT, (const Ord*)p->d_ord, (const Cell*)p->d_cell,
                                    R.phi, R.old ? (const T*)p->d_psi[p->cur] : nullptr, (const T*)R.rarr, R.withq,
                                    p->nx, p->ny, p->Q, p->Qp, (T)dt, (T)p->sigma_as};
        si_source_kernel<T, Ord, Cell><<<sgrid, std::min(256, (p->Q + 31) / 32 * 32), smem, p->stream>>>(sa);
        ICK(p, cudaGetLastError());
        const bool norm = fixed <= 0 && Tl > 0.0;                // the stopping rule needs the difference
        SweepArgs<T, Ord, Cell> sw{(const T*)W->buf[2], (T*)W->buf[out], (const Ord*)p->d_ord, (const Cell*)p->d_cell,
                                   W->d_chunks, rows && norm ? (const T*)cur : nullptr, W->d_part,
                                   p->nx, p->ny, p->Qp, (T)dt, (T)p->sigma_as};
        if (rows) {
            const dim3 g(W->nchunks), b(row_threads);
            if (rpt == 1) sweep_rows_kernel<T, Ord, Cell, 1><<<g, b, ring, p->stream>>>(sw);
            else if (rpt == 2) sweep_rows_kernel<T, Ord, Cell, 2><<<g, b, ring, p->stream>>>(sw);
            else sweep_rows_kernel<T, Ord, Cell, 4><<<g, b, ring, p->stream>>>(sw);
        } else {
            sweep_kernel<T, Ord, Cell><<<W->nchunks, kSweepThreads, 0, p->stream>>>(sw);
        }
        ICK(p, cudaGetLastError());
        p->launches += 2;
        ++it;
        ++W->sweeps_total;
        const void* prev = cur;
        cur = W->buf[out];
        out ^= 1;
        if (fixed > 0) {
            if (it >= fixed) break;
            continue;
        }
        if (Tl == 0.0) break;                      // no artificial scattering: one sweep is exact
        int nparts = W->nchunks;
        if (!rows) {
            sqdiff_partials<T><<<kRedBlocks, 256, 0, p->stream>>>((const T*)cur, (const T*)prev, n, W->d_part);
            ICK(p, cudaGetLastError());
            ++p->launches;
            nparts = kRedBlocks;
        }
        double d2 = 0;
        int r = read_sum(p, &d2, nparts);
        if (r) return r;
        if (sqrt(d2) < tol) break;
        // FP32 state: once the difference stops falling the iterates only differ by rounding
        if (!std::is_same<T, double>::value && d2 >= prev_d2) break;
        prev_d2 = d2;
        if (it >= W->max_si) {
            W->last_si_converged = 0;
            break;
        }
    }
    W->si_total += it;
    *result = cur;
    return ASSN_OK;
}

template <typename T>
int moments(assn_problem* p, const void* psi, double* phi) {
    const T* w = std::is_same<T, double>::value ? (const T*)p->d_w64 : (const T*)(const void*)p->d_w32;
    ICK(p, launch_scalar_flux<T>((const T*)psi, w, (int)p->ncell(), p->Qp, nullptr, phi, p->stream));
    ++p->launches;
    return ASSN_OK;
}

// out = v - M SI(sigma_s O Sigma v): the operator A of the Krylov system (Alg. 2).
template <typename T>
int apply_A(assn_problem* p, double dt, const double* v, double* out) {
    Rhs R;
    R.phi = v;
    const void* psi = nullptr;
    int r = source_iteration<T>(p, dt, R, p->d_psi[p->cur], 0, &psi);
    if (r) return r;
    r = moments<T>(p, psi, out);
    if (r) return r;
    return lincomb(p, 1.0, v, -1.0, out);
}

// Restarted GMRES with modified Gram-Schmidt and Givens rotations: A x = b, x holds the start.
template <typename T>
int gmres(assn_problem* p, double dt, double* x, const double* b, int* iters) {
    ImplicitWork* W = p->impl;
    const int m = W->restart;
    const size_t n = p->ncell();
    double* wv = W->vec + 2 * n;
    double nb = 0;
    int r = dot(p, b, b, &nb);
    if (r) return r;
    nb = sqrt(nb);
    // FP32 state: the operator is evaluated through FP32 source iterations, so residuals below about
    // 2^-20 relative are rounding; the tolerance is not taken below that
    const double tol = std::is_same<T, double>::value ? W->gmres_tol : std::max(W->gmres_tol, 0x1p-20);
    *iters = 0;
    W->last_gmres_converged = 1;
    if (nb == 0.0) {
        ICK(p, cudaMemsetAsync(x, 0, n * sizeof(double), p->stream));
        return ASSN_OK;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    int total = 0;
    while (true) {
        double* v0 = W->V;
        if ((r = apply_A<T>(p, dt, x, v0))) return r;
        if ((r = lincomb(p, 1.0, b, -1.0, v0))) return r;          // v0 = b - A x
        double beta = 0;
        if ((r = dot(p, v0, v0, &beta))) return r;
        beta = sqrt(beta);
        if (beta <= tol * nb) break;
        if (total >= W->max_gmres) {
            W->last_gmres_converged = 0;
            break;
        }
        if ((r = scale(p, 1.0 / beta, v0, v0))) return r;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int kd = 0;
        for (int k = 0; k < m; ++k) {
            double* vk = W->V + (size_t)k * n;
            if ((r = apply_A<T>(p, dt, vk, wv))) return r;
            for (int i = 0; i <= k; ++i) {
                double hik = 0;
                if ((r = dot(p, W->V + (size_t)i * n, wv, &hik))) return r;
                Hij(i, k) = hik;
                if ((r = lincomb(p, -hik, W->V + (size_t)i * n, 1.0, wv))) return r;
            }
            double hk1 = 0;
            if ((r = dot(p, wv, wv, &hk1))) return r;
            hk1 = sqrt(hk1);
            Hij(k + 1, k) = hk1;
            for (int i = 0; i < k; ++i) {                              // earlier rotations
                const double t = cs[i] * Hij(i, k) + sn[i] * Hij(i + 1, k);
                Hij(i + 1, k) = -sn[i] * Hij(i, k) + cs[i] * Hij(i + 1, k);
                Hij(i, k) = t;
            }
            const double den = hypot(Hij(k, k), Hij(k + 1, k));
            cs[k] = den > 0 ? Hij(k, k) / den : 1.0;
            sn[k] = den > 0 ? Hij(k + 1, k) / den : 0.0;
            Hij(k, k) = den;
            Hij(k + 1, k) = 0.0;
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            ++total;
            kd = k + 1;
            if (hk1 > 0 && (r = scale(p, 1.0 / hk1, wv, W->V + (size_t)(k + 1) * n))) return r;
            if (fabs(g[k + 1]) <= tol * nb || hk1 == 0.0 || total >= W->max_gmres) break;
        }
        for (int i = kd - 1; i >= 0; --i) {                            // H y = g (upper triangular)
            double s = g[i];
            for (int j = i + 1; j < kd; ++j) s -= Hij(i, j) * y[j];
            y[i] = s / Hij(i, i);
        }
        for (int i = 0; i < kd; ++i)
            if ((r = lincomb(p, y[i], W->V + (size_t)i * n, 1.0, x))) return r;
        if (fabs(g[kd]) <= tol * nb) break;
        if (total >= W->max_gmres) {
            W->last_gmres_converged = 0;
            break;
        }
    }
    W->gmres_total += total;
    *iters = total;
    return ASSN_OK;
}

// One step of Alg. 3; x carries the scalar flux (the GMRES start) between the steps of one call.
template <typename T>
int implicit_step(assn_problem* p, double dt) {
    ImplicitWork* W = p->impl;
    const size_t n = p->ncell();
    double* x = W->vec;
    double* b = W->vec + n;
    Rhs base;
    base.withq = 1;
    base.old = true;
    const void* psi = nullptr;
    int r = source_iteration<T>(p, dt, base, p->d_psi[p->cur], 0, &psi);
    if (r) return r;
    if ((r = moments<T>(p, psi, b))) return r;
    int its = 0;
    if ((r = gmres<T>(p, dt, x, b, &its))) return r;
    Rhs fin = base;
    fin.phi = x;
    if ((r = source_iteration<T>(p, dt, fin, p->d_psi[p->cur], 0, &psi))) return r;
    ICK(p, cudaMemcpyAsync(p->d_psi[p->cur ^ 1], psi, n * p->Qp * p->elem(), cudaMemcpyDeviceToDevice, p->stream));
    p->cur ^= 1;
    return ASSN_OK;
}

}  // namespace

void implicit_free(ImplicitWork* W) {
    if (!W) return;
    for (auto* b : W->buf) if (b) cudaFree(b);
    for (auto* b : W->rtmp) if (b) cudaFree(b);
    if (W->d_chunks) cudaFree(W->d_chunks);
    if (W->V) cudaFree(W->V);
    if (W->vec) cudaFree(W->vec);
    if (W->d_part) cudaFree(W->d_part);
    if (W->d_red) cudaFree(W->d_red);
    if (W->h_red) cudaFreeHost(W->h_red);
    delete W;
}

int implicit_steps(assn_problem* p, int nsteps, double dt) {
    TraceRange tr("implicit steps");
    if (p->tensor())
        return problem_fail(p, ASSN_ERR_UNSUPPORTED, "the implicit scheme runs in FP64 or FP32 (CUDA cores)");
    int r = problem_prepare(p, dt);
    if (r) return r;
    if ((r = ensure_work(p))) return r;
    const bool f64 = p->precision == ASSN_FP64;
    // GMRES start of the first step: the scalar flux of the current state
    r = f64 ? moments<double>(p, p->d_psi[p->cur], p->impl->vec) : moments<float>(p, p->d_psi[p->cur], p->impl->vec);
    if (r) return r;
    for (int s = 0; s < nsteps; ++s) {
        r = f64 ? implicit_step<double>(p, dt) : implicit_step<float>(p, dt);
        if (r) return r;
    }
    return ASSN_OK;
}

}  // namespace assn

using namespace assn;

extern "C" int assn_set_implicit_params(assn_problem* p, double si_eps, double gmres_tol, int restart, int max_si,
                                        int max_gmres) {
    if (!p) return ASSN_ERR_ARG;
    if (!(si_eps >= 0) || !(gmres_tol >= 0) || restart < 1 || restart > 200 || max_si < 1 || max_gmres < 1)
        return problem_fail(p, ASSN_ERR_ARG, "implicit parameters out of range");
    if (!p->impl) p->impl = new ImplicitWork();
    p->impl->si_eps = si_eps;
    p->impl->gmres_tol = gmres_tol;
    p->impl->restart = restart;
    p->impl->max_si = max_si;
    p->impl->max_gmres = max_gmres;
    return ASSN_OK;
}

extern "C" int assn_implicit_stats(const assn_problem* p, int64_t* source_iterations, int64_t* gmres_iterations,
                                   int64_t* sweeps) {
    if (!p) return ASSN_ERR_ARG;
    const ImplicitWork* W = p->impl;
    if (source_iterations) *source_iterations = W ? W->si_total : 0;
    if (gmres_iterations) *gmres_iterations = W ? W->gmres_total : 0;
    if (sweeps) *sweeps = W ? W->sweeps_total : 0;
    return ASSN_OK;
}

extern "C" int assn_implicit_source_iteration(assn_problem* p, double dt, const double* R, const double* psi0,
                                              int iterations, double* psi_out) {
    if (!p || !R || !psi0 || !psi_out) return ASSN_ERR_ARG;
    if (iterations < 1) return problem_fail(p, ASSN_ERR_ARG, "iterations < 1");
    if (p->tensor())
        return problem_fail(p, ASSN_ERR_UNSUPPORTED, "the implicit scheme runs in FP64 or FP32 (CUDA cores)");
    int r = problem_prepare(p, dt);
    if (r) return r;
    if ((r = ensure_work(p))) return r;
    ImplicitWork* W = p->impl;
    const size_t ncell = p->ncell(), n = ncell * p->Qp;
    const bool f64 = p->precision == ASSN_FP64;
    for (int b = 0; b < 2; ++b)
        if (!W->rtmp[b]) ICK(p, cudaMalloc(&W->rtmp[b], n * p->elem()));   // freed with buf when Qp changes
    // pack [ncell][Q] FP64 host arrays into padded device arrays of the state type
    std::vector<double> pd(n, 0.0);
    std::vector<float> pf(f64 ? 0 : n, 0.0f);
    const double* src[2] = {R, psi0};
    for (int b = 0; b < 2; ++b) {
        for (size_t c = 0; c < ncell; ++c)
            for (int q = 0; q < p->Q; ++q) {
                const double v = src[b][c * p->Q + q];
                if (f64) pd[c * p->Qp + q] = v; else pf[c * p->Qp + q] = (float)v;
            }
        ICK(p, cudaMemcpyAsync(W->rtmp[b], f64 ? (const void*)pd.data() : (const void*)pf.data(), n * p->elem(),
                               cudaMemcpyHostToDevice, p->stream));
        ICK(p, cudaStreamSynchronize(p->stream));
    }
    Rhs rhs;
    rhs.rarr = W->rtmp[0];
    const void* out = nullptr;
    r = f64 ? source_iteration<double>(p, dt, rhs, W->rtmp[1], iterations, &out)
            : source_iteration<float>(p, dt, rhs, W->rtmp[1], iterations, &out);
    if (r) return r;
    ICK(p, cudaMemcpyAsync(f64 ? (void*)pd.data() : (void*)pf.data(), out, n * p->elem(), cudaMemcpyDeviceToHost,
                           p->stream));
    ICK(p, cudaStreamSynchronize(p->stream));
    for (size_t c = 0; c < ncell; ++c)
        for (int q = 0; q < p->Q; ++q)
            psi_out[c * p->Q + q] = f64 ? pd[c * p->Qp + q] : (double)pf[c * p->Qp + q];
    return ASSN_OK;
}

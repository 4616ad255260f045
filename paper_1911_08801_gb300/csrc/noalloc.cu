// Total particle number of a caller-owned device state, computed without allocating any memory.
//
// For callers that cannot allocate device memory during the call: real-time loops whose latency
// budget rules out allocator calls (cudaMalloc may block and synchronise the device), and hosts
// that run the library inside a memory pool they manage themselves.  The reduction's partial sums
// live in a fixed file-scope device array instead of an allocation; its device address is looked
// up once per device, on the first call there, and reused by later calls.
#include <cstdio>
#include <mutex>

#include "assn_internal.h"

namespace {

constexpr int kCellsPerBlock = ASSN_NOALLOC_MASS_CELLS_PER_BLOCK;
constexpr int kMaxBlocks = ASSN_NOALLOC_MASS_MAX_BLOCKS;
constexpr int kThreads = 256;

// One partial sum per block.  Held by every device that loads the library until process exit;
// shared by all calls, so calls whose work overlaps on a device race on it.
static __device__ __align__(256) double g_mass_scratch[kMaxBlocks];

template <typename T>
__global__ void mass_blocks_kernel(const T* __restrict__ psi, const double* __restrict__ w, int ncell, int Qp,
                                   double* __restrict__ partials) {
    __shared__ double red[kThreads / 32];
    const int c0 = blockIdx.x * kCellsPerBlock;
    const int c1 = min(ncell, c0 + kCellsPerBlock);
    double s = 0.0;
    const size_t n = (size_t)(c1 - c0) * Qp;
    const T* base = psi + (size_t)c0 * Qp;
    for (size_t i = threadIdx.x; i < n; i += kThreads) s += w[i % Qp] * (double)base[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) t += red[i];
        partials[blockIdx.x] = t;
    }
}

__global__ void mass_finish_kernel(const double* __restrict__ partials, int nblocks, double area, double* out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partials[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        *out = t * area;
    }
}

// Device address of the scratch array, looked up once per device (with that device current).
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mass_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

thread_local char g_err[256];

int fail(int status, const char* msg) {
    snprintf(g_err, sizeof g_err, "%s", msg);
    return status;
}

}  // namespace

extern "C" int assn_mass_noalloc(const void* psi_dev, int elem_bytes, const double* w_dev, int ncell, int Qp,
                                 double h, double* mass_dev, void* stream) {
    if (!psi_dev || !w_dev || !mass_dev) return fail(ASSN_ERR_ARG, "assn_mass_noalloc: NULL pointer");
    if (elem_bytes != 4 && elem_bytes != 8) return fail(ASSN_ERR_ARG, "assn_mass_noalloc: elem_bytes must be 4 or 8");
    if (ncell < 1 || Qp < 1) return fail(ASSN_ERR_ARG, "assn_mass_noalloc: ncell and Qp must be positive");
    if (ncell > ASSN_NOALLOC_MASS_MAX_CELLS)
        return fail(ASSN_ERR_ARG, "assn_mass_noalloc: ncell exceeds ASSN_NOALLOC_MASS_MAX_CELLS (scratch holds "
                                  "one partial sum per 256 cells, 16384 partial sums)");
    if (Qp > ASSN_MAX_Q) return fail(ASSN_ERR_ARG, "assn_mass_noalloc: Qp exceeds ASSN_MAX_Q");
    double* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return fail(ASSN_ERR_CUDA, cudaGetErrorString(e));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nblocks = (ncell + kCellsPerBlock - 1) / kCellsPerBlock;
    if (elem_bytes == 4)
        mass_blocks_kernel<float><<<nblocks, kThreads, 0, s>>>(static_cast<const float*>(psi_dev), w_dev, ncell, Qp,
                                                             scratch);
    else
        mass_blocks_kernel<double><<<nblocks, kThreads, 0, s>>>(static_cast<const double*>(psi_dev), w_dev, ncell,
                                                              Qp, scratch);
    mass_finish_kernel<<<1, 1024, 0, s>>>(scratch, nblocks, h * h, mass_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ASSN_ERR_CUDA, cudaGetErrorString(e));
    g_err[0] = 0;
    return ASSN_OK;
}

extern "C" const char* assn_noalloc_last_error(void) { return g_err; }

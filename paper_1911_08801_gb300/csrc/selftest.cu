// Self-test of the failure path shared by the tensor-core step kernels: a bounded mbarrier wait that
// nothing completes gives up after its limit, records the event in an error flag that the host
// reads, and the kernel returns normally, so the CUDA context stays usable.
#include "assn_internal.h"
#include "tc_ptx.h"

namespace {

using namespace assn::ptx;

__global__ void wait_timeout_kernel(unsigned int* err, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);   // one arrival expected; none is ever made
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait_for(&bar, 0u, &abort_flag, err, 0x8000u, limit_ns);
}

}  // namespace

extern "C" int assn_selftest_wait_timeout(int limit_us) {
    if (limit_us < 1 || limit_us > 1000000) return ASSN_ERR_ARG;
    unsigned int* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned int)) != cudaSuccess) return ASSN_ERR_OOM;
    unsigned int flag = 0;
    cudaError_t e = cudaMemset(d, 0, sizeof flag);
    if (e == cudaSuccess) {
        wait_timeout_kernel<<<1, 32>>>(d, (uint64_t)limit_us * 1000ull);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, d, sizeof flag, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return ASSN_ERR_CUDA;
    return flag == 0x8000u ? ASSN_ERR_TIMEOUT : ASSN_ERR_CUDA;
}

// fsp_selftest.cu -- a check of the bounded device waits (C ABI test hook).
//
// The TMA-staged passes wait on shared-memory barriers whose phases complete
// when their bulk copies land; every such wait gives up after a time limit,
// records FSP_ERR_TIMEOUT in a status word and lets the kernel return, so a
// lost copy cannot hang the GPU.  This hook runs that wait on a barrier that
// nothing will ever complete: one arrival announcing 16 bytes that are never
// copied, with no copy in flight, so the kernel exits cleanly once its wait
// gives up.  Nothing faults; the context stays usable.
#include "fsp_internal.h"
#include "fsp_tma.cuh"

namespace {

__global__ void k_wait_selftest(int *status, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        fsp::mbar_init(&bar, 1);
        fsp::mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) fsp::mbar_expect_tx(&bar, 16);   // 16 bytes that no copy will deliver
    const bool ok = fsp::mbar_wait(&bar, 0, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) fsp::record_status(status, FSP_ERR_TIMEOUT);
}

} // namespace

extern "C" int fsp_selftest_wait_timeout(double limit_seconds)
{
    if (!(limit_seconds > 0.0) || limit_seconds > 10.0) return fsp::record_error(FSP_ERR_INVALID);
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return fsp::record_error(FSP_ERR_NOMEM);
    int h = -1, rc = FSP_OK;
    if (cudaMemset(d, 0, sizeof(int)) != cudaSuccess) rc = FSP_ERR_CUDA;
    if (rc == FSP_OK) {
        k_wait_selftest<<<1, 32>>>(d, (unsigned long long)(limit_seconds * 1e9));
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = FSP_ERR_CUDA;
    }
    cudaFree(d);
    return fsp::record_error(rc == FSP_OK ? h : rc);
}

// Self-test of the bounded device-side waits: each kernel waits for
// something that never happens (an mbarrier phase nobody completes, a flag
// nobody sets) with a short budget, and must give up, record
// GBSW_ERR_TIMEOUT and return, leaving the context usable.
#include "common.cuh"
#include "tc.cuh"

namespace {

__global__ void selftest_mbar_kernel(long long budget, int *status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        gbsw::tc::mbar_init(&bar, 1);
        gbsw::tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !gbsw::tc::mbar_wait(&bar, 0, budget)) atomicCAS(status, gbsw::DEV_OK, gbsw::DEV_TIMEOUT);
}

__global__ void selftest_flag_kernel(const unsigned *flag, long long spins, int *status)
{
    if (threadIdx.x != 0) return;
    long long n = 0;
    while (atomicAdd((unsigned *)flag, 0u) == 0u) {
        if (++n > spins) {
            atomicCAS(status, gbsw::DEV_OK, gbsw::DEV_TIMEOUT);
            break;
        }
        __nanosleep(64);
    }
}

}  // namespace

extern "C" gbsw_status gbsw_selftest_wait(int which, long long budget)
{
    if (which < 0 || which > 1 || budget < 1 || budget > 1000000000LL) return GBSW_ERR_ARG;
    int *d = nullptr;  // [0] status, [1] flag (never set)
    GBSW_CUDA_TRY(cudaMalloc((void **)&d, 2 * sizeof(int)));
    int h = 0;
    cudaError_t e = cudaMemset(d, 0, 2 * sizeof(int));
    if (e == cudaSuccess) {
        if (which == 0) selftest_mbar_kernel<<<1, 32>>>(budget, d);
        else selftest_flag_kernel<<<1, 32>>>((const unsigned *)(d + 1), budget, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        gbsw::record_cuda_error(e, "gbsw_selftest_wait", __FILE__, __LINE__);
        return GBSW_ERR_CUDA;
    }
    return gbsw::dev_status_to_gbsw(h);
}

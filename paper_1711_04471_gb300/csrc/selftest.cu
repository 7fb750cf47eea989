// Self-tests.
// gbsw_selftest_wait: the bounded device-side waits.  Each kernel waits for
// something that never happens (an mbarrier phase nobody completes, a flag
// nobody sets) with a short budget, and must give up, record
// GBSW_ERR_TIMEOUT and return, leaving the context usable.
// gbsw_selftest_sor_division: the SOR sweep's division by the diagonal
// (sor_div) against the IEEE division x / d for every finite FP32 x.
// gbsw_measure_l2_copy: the copy bandwidth of buffers that stay in L2, the
// ceiling of a kernel whose working set stays in L2 between passes.
// gbsw_selftest_bounds: the index test of the bounds-checked debug build,
// given an index one past the end of a buffer (no access is made).
#include "common.cuh"
#include "poisson.cuh"
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

// Every 32-bit pattern once (grid-stride); out[0] counts mismatches with a
// normal x of magnitude at least 2^-100, out[1] the others; out[2] is the
// smallest mismatching pattern (0xffffffff if none).
__global__ void selftest_div_kernel(float d, float y, unsigned long long *out)
{
    unsigned long long bad_normal = 0, bad_tiny = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; b < (1ull << 32);
         b += stride) {
        const float x = __uint_as_float((unsigned)b);
        if (!isfinite(x)) continue;
        const float got = gbsw::sor_div(x, d, y);
        const float want = x / d;
        if (__float_as_uint(got) != __float_as_uint(want)) {
            if (fabsf(x) >= 0x1p-100f) ++bad_normal;
            else ++bad_tiny;
            atomicMin(&out[2], b);
        }
    }
    if (bad_normal) atomicAdd(&out[0], bad_normal);
    if (bad_tiny) atomicAdd(&out[1], bad_tiny);
}

// passes x (dst = src) over n float4 words, grid-stride, in one launch.
__global__ void __launch_bounds__(512) l2_copy_kernel(const float4 *__restrict__ src, float4 *__restrict__ dst,
                                                      long long n, int passes)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p)
        for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) dst[q] = src[q];
}

// The debug build's index test on index n of an n-element buffer: the
// test fails, counts the violation, and the access it guards is skipped.
__global__ void selftest_bounds_kernel(const float *buf, long long n, unsigned *count, float *out)
{
    if (threadIdx.x == 0) *out = gbsw::index_ok(n, n, count) ? buf[n] : 0.0f;
}

}  // namespace

extern "C" gbsw_status gbsw_selftest_bounds(void)
{
    unsigned *d = nullptr;  // [0] count, [1..] the guarded buffer and the result
    GBSW_CUDA_TRY(cudaMalloc((void **)&d, 8 * sizeof(unsigned)));
    unsigned h = 0;
    cudaError_t e = cudaMemset(d, 0, 8 * sizeof(unsigned));
    if (e == cudaSuccess) {
        selftest_bounds_kernel<<<1, 32>>>((const float *)(d + 1), 4, d, (float *)(d + 6));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        gbsw::record_cuda_error(e, "gbsw_selftest_bounds", __FILE__, __LINE__);
        return GBSW_ERR_CUDA;
    }
    return h == 1 ? GBSW_ERR_DEVICE_BOUNDS : GBSW_ERR_CUDA;
}

extern "C" gbsw_status gbsw_measure_l2_copy(long long bytes, int passes, double *gbs)
{
    if (bytes < (1 << 20) || bytes % 16 || passes < 1 || passes > 10000 || !gbs) return GBSW_ERR_ARG;
    float4 *buf = nullptr;
    GBSW_CUDA_TRY(cudaMalloc((void **)&buf, 2 * (size_t)bytes));
    const long long n = bytes / 16;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemset(buf, 0, 2 * (size_t)bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 0.0;
    const int grid = 2 * gbsw::sm_count();  // 2 x 512 threads per SM, one wave
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0);
        l2_copy_kernel<<<grid, 512>>>(buf, buf + n, n, passes);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && ms > 0.0f) {  // the first launch brings the buffers into L2
            const double r = 2.0 * (double)bytes * passes / (ms * 1e-3) / 1e9;
            if (r > best) best = r;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) {
        gbsw::record_cuda_error(e, "gbsw_measure_l2_copy", __FILE__, __LINE__);
        return GBSW_ERR_CUDA;
    }
    *gbs = best;
    return GBSW_OK;
}

extern "C" gbsw_status gbsw_selftest_sor_division(int d, unsigned long long *counts)
{
    if (d < 4 || d > 7 || !counts) return GBSW_ERR_ARG;
    const gbsw::SorDiag dg = gbsw::sor_diag();
    unsigned long long *dev = nullptr;
    GBSW_CUDA_TRY(cudaMalloc((void **)&dev, 3 * sizeof(unsigned long long)));
    unsigned long long init[3] = {0, 0, 0xffffffffull};
    cudaError_t e = cudaMemcpy(dev, init, sizeof(init), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        selftest_div_kernel<<<4 * gbsw::sm_count(), 256>>>(dg.d[d - 4], dg.y[d - 4], dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(counts, dev, sizeof(init), cudaMemcpyDeviceToHost);
    cudaFree(dev);
    if (e != cudaSuccess) {
        gbsw::record_cuda_error(e, "gbsw_selftest_sor_division", __FILE__, __LINE__);
        return GBSW_ERR_CUDA;
    }
    return GBSW_OK;
}

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

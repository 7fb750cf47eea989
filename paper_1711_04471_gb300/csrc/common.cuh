// Shared host/device helpers of the gbsw CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/gbsw.h"

namespace gbsw {

// Device status word values (first writer wins, see set_device_status).
enum : int { DEV_OK = 0, DEV_BOUNDS = 1, DEV_TIMEOUT = 2, DEV_NONFINITE = 3 };

__device__ __forceinline__ void set_device_status(int *status, int code)
{
    atomicCAS(status, DEV_OK, code);
}

inline gbsw_status dev_status_to_gbsw(int s)
{
    switch (s) {
    case DEV_OK: return GBSW_OK;
    case DEV_BOUNDS: return GBSW_ERR_DEVICE_BOUNDS;
    case DEV_TIMEOUT: return GBSW_ERR_TIMEOUT;
    case DEV_NONFINITE: return GBSW_ERR_NONFINITE;
    default: return GBSW_ERR_CUDA;
    }
}

// Bounds-checked debug build (compiled with -DGBSW_DEBUG_BOUNDS=1 into
// libgbsw_debug.so): the 2DSW and SOR kernels test every global index
// against the extent of its buffer before the access.  A failed test skips
// the access (a load gives 0) and counts the violation in a device word of
// its translation unit; gbsw_debug_bounds reads and clears the counts.
// The product build compiles the tests away.
#ifndef GBSW_DEBUG_BOUNDS
#define GBSW_DEBUG_BOUNDS 0
#endif

__device__ __forceinline__ bool index_ok(long long i, long long n, unsigned *count)
{
    if (i >= 0 && i < n) return true;
    atomicAdd(count, 1u);
    return false;
}

#if GBSW_DEBUG_BOUNDS
#define GBSW_INBOUNDS(i, n, count) ::gbsw::index_ok((long long)(i), (long long)(n), (count))
#else
#define GBSW_INBOUNDS(i, n, count) true
#endif

// Violation counts of the debug build, read and cleared (one function per
// translation unit that has checked kernels; 0 in the product build).
unsigned long long take_bounds_sw();
unsigned long long take_bounds_batch();
unsigned long long take_bounds_poisson();
unsigned long long take_bounds_les();
unsigned long long take_bounds_ws();

// Remember the last CUDA error text for diagnostics.
void record_cuda_error(cudaError_t e, const char *what, const char *file, int line);

#define GBSW_CUDA_TRY(expr)                                                   \
    do {                                                                      \
        cudaError_t _e = (expr);                                              \
        if (_e != cudaSuccess) {                                              \
            ::gbsw::record_cuda_error(_e, #expr, __FILE__, __LINE__);         \
            return _e == cudaErrorMemoryAllocation ? GBSW_ERR_OOM : GBSW_ERR_CUDA; \
        }                                                                     \
    } while (0)

#define GBSW_LAUNCH_CHECK()                                                   \
    do {                                                                      \
        cudaError_t _e = cudaGetLastError();                                  \
        if (_e != cudaSuccess) {                                              \
            ::gbsw::record_cuda_error(_e, "kernel launch", __FILE__, __LINE__); \
            return GBSW_ERR_CUDA;                                             \
        }                                                                     \
    } while (0)

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
inline size_t round_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// Number of SMs of the current device (cached per process).
int sm_count();

// Host-side fault injection for tests, from the GBSW_FAULT environment
// variable (read at each call): "alloc" makes the create calls return
// GBSW_ERR_OOM before any device allocation; "sync_timeout" gives the
// ensemble kernel's grid barrier a zero spin budget, so that its bounded
// wait gives up and the call reports GBSW_ERR_TIMEOUT.  No injection
// faults, traps or hangs a device.
bool fault_injected(const char *what);

// NVTX range over a host scope (shown by profilers that record NVTX; the
// header-only NVTX library makes it a no-op otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------------------
// Deterministic FP64 block reduction: every thread contributes one value;
// the warp tree (shuffle down by 16, 8, 4, 2, 1) and then a fixed-order
// tree over warps give a result that depends only on the launch shape.
// ---------------------------------------------------------------------------
template <int NWARPS>
__device__ __forceinline__ double block_sum_f64(double v, double *smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < NWARPS ? smem[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

template <int NWARPS>
__device__ __forceinline__ double block_min_f64(double v, double *smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double r = INFINITY;
    if (warp == 0) {
        r = lane < NWARPS ? smem[lane] : INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmin(r, __shfl_down_sync(0xffffffffu, r, o));
    }
    __syncthreads();
    return r;
}

}  // namespace gbsw

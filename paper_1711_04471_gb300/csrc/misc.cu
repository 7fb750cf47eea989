// Library-wide helpers: status strings, last-error text, device queries.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"

namespace gbsw {

static thread_local char g_last_error[512] = "";

void record_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 1;
    }
    return n;
}

bool fault_injected(const char *what)
{
    const char *v = getenv("GBSW_FAULT");
    return v && strcmp(v, what) == 0;
}

}  // namespace gbsw

extern "C" {

const char *gbsw_status_string(int status)
{
    switch (status) {
    case GBSW_OK: return "ok";
    case GBSW_ERR_ARG: return "invalid argument";
    case GBSW_ERR_CUDA: return "CUDA error";
    case GBSW_ERR_OOM: return "out of memory";
    case GBSW_ERR_CFL: return "CFL condition violated";
    case GBSW_ERR_NONFINITE: return "non-finite value in state";
    case GBSW_ERR_TIMEOUT: return "device-side wait timed out";
    case GBSW_ERR_DEVICE_BOUNDS: return "device index out of range";
    case GBSW_NOT_CONVERGED: return "not converged";
    default: return "unknown status";
    }
}

const char *gbsw_last_error(void) { return gbsw::g_last_error; }

int gbsw_version(void) { return 100; }

}  // extern "C"

// Out-of-range index counts of the bounds-checked debug build.
extern "C" gbsw_status gbsw_debug_bounds(long long *violations)
{
    if (!violations) return GBSW_ERR_ARG;
#if GBSW_DEBUG_BOUNDS
    GBSW_CUDA_TRY(cudaDeviceSynchronize());
    const unsigned long long n = gbsw::take_bounds_sw() + gbsw::take_bounds_batch() + gbsw::take_bounds_poisson() +
                                 gbsw::take_bounds_les() + gbsw::take_bounds_ws();
    *violations = (long long)n;
    return n ? GBSW_ERR_DEVICE_BOUNDS : GBSW_OK;
#else
    *violations = -1;  // the product build has no checks
    return GBSW_OK;
#endif
}

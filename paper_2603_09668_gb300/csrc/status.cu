// Error reporting of the C-ABI (dw_last_error, dw_version) and the mapping
// from device status bits to dw_status codes.
#include <stdarg.h>
#include <stdio.h>

#include "common.cuh"

namespace dw {

static thread_local char g_last_error[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
}

dw_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    if (e == cudaErrorMemoryAllocation) return DW_ERR_OOM;
    return DW_ERR_CUDA;
}

dw_status status_from_bits(int bits) {
    if (bits & ERRBIT_DOMAIN) {
        set_error("device: a particle's stencil left the grid");
        return DW_ERR_DOMAIN;
    }
    if (bits & ERRBIT_INVERTED) {
        set_error("device: inverted element (det F <= 0)");
        return DW_ERR_INVERTED;
    }
    if (bits & ERRBIT_NONFINITE) {
        set_error("device: non-finite value");
        return DW_ERR_NONFINITE;
    }
    if (bits & ERRBIT_TIMEOUT) {
        set_error("device: a bounded wait gave up");
        return DW_ERR_TIMEOUT;
    }
    return DW_OK;
}

}  // namespace dw

extern "C" const char *dw_last_error(void) { return dw::g_last_error; }

extern "C" const char *dw_version(void) { return "diffwind-gb300 0.1 (sm_103a)"; }

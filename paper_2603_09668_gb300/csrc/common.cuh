// Shared host/device helpers of libdiffwind: status handling, device error
// bits, launch helpers. Internal to the CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "diffwind.h"

namespace dw {

// Thread-local message for dw_last_error().
void set_error(const char *fmt, ...);
dw_status cuda_fail(cudaError_t e, const char *what);

// Bits of a handle's device status word (set with atomicOr, never cleared on
// the device). The host maps the lowest set bit to a dw_status.
enum : int {
    ERRBIT_NONFINITE = 1,
    ERRBIT_DOMAIN = 2,
    ERRBIT_TIMEOUT = 4,
    ERRBIT_INVERTED = 8,
};
dw_status status_from_bits(int bits);

inline cudaStream_t as_stream(dw_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while its predecessor in the stream is finishing; it must call pdl_wait()
// before touching anything the predecessor writes (a no-op when the kernel was
// launched normally). pdl_trigger() lets the next kernel get scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                              cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl3(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                               Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// launch_pdl3 with dynamic shared memory.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                   cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

inline unsigned grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace dw

#define DW_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::dw::cuda_fail(e_, #call);       \
    } while (0)

#define DW_LAUNCHED(what)                                               \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return ::dw::cuda_fail(e_, what);        \
    } while (0)

#define DW_REQUIRE(cond, ...)                                           \
    do {                                                                \
        if (!(cond)) {                                                  \
            ::dw::set_error(__VA_ARGS__);                               \
            return DW_ERR_ARG;                                          \
        }                                                               \
    } while (0)

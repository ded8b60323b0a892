// FP32 throughput probe: the denominator of the FP32 roofline of the MPM
// kernels, measured on the GPU that runs them. Each thread runs 16
// independent fused multiply-add chains (scalar FFMA, or eight float2 chains
// of the paired FFMA2 instruction of sm_100 and later) so that the FMA pipes,
// not the chains' latency, bound it.
#include "common.cuh"

namespace dw {

constexpr int PROBE_THREADS = 256;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma(float *out, int iters, float b, float c) {
    float a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = (float)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k];
    if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma2(float *out, int iters, float b, float c) {
    float2 a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
    if (s == 12345.678f) out[blockIdx.x] = s;
}

}  // namespace dw

using namespace dw;

extern "C" dw_status dw_fp32_probe(int32_t paired, int32_t iters, int32_t blocks, float *out,
                                   double *flops, dw_stream stream) {
    DW_REQUIRE(out && flops, "out/flops must not be NULL");
    DW_REQUIRE(iters >= 1 && blocks >= 1, "iters and blocks must be >= 1");
    cudaStream_t s = as_stream(stream);
    // b, c keep the values bounded: a <- a * 0.999 + 1e-3
    if (paired)
        k_probe_ffma2<<<blocks, PROBE_THREADS, 0, s>>>(out, iters, 0.999f, 1e-3f);
    else
        k_probe_ffma<<<blocks, PROBE_THREADS, 0, s>>>(out, iters, 0.999f, 1e-3f);
    DW_LAUNCHED("dw_fp32_probe");
    *flops = 2.0 * 16.0 * 8.0 * (double)iters * PROBE_THREADS * (double)blocks;
    return DW_OK;
}

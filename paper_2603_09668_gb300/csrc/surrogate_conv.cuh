// Weight gradients of the surrogate network's 3x3x3 convolutions on the
// tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation), and the
// helpers the convolution kernels share (GELU and its derivative).
//
// k_wgrad: dW[tap][co][ci] = sum_v g[v][co] in[v + d(tap)][ci] over the
// voxels of a chunk of output tiles of 16 (x) x 8 (y) x 1 (z), written as
// partial sums that k_wgrad_reduce adds up. The training backward pass runs
// the tcgen05 version (surrogate_wgrad_tc.cuh); this warp-level MMA kernel is
// kept as the second implementation surr_weight_grad offers. Activations are
// planar, [C/8][n^3][8] BF16. Shared-memory rows (a voxel's or an output
// channel's values) keep their 16-byte chunks XOR-swizzled by the row index,
// so that the eight rows an ldmatrix matrix reads hit distinct banks.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace dw {

typedef __nv_bfloat16 bf16;

constexpr int CV_TX = 16, CV_TY = 8;   // output tile
constexpr int CV_HX = CV_TX + 2, CV_HY = CV_TY + 2, CV_HZ = 3;
constexpr int CV_HALO = CV_HX * CV_HY * CV_HZ;  // 540 voxels
constexpr int CV_THREADS = 256;

enum { EPI_GELU = 0, EPI_F32 = 1, EPI_DGELU = 2, EPI_GELU_ONLY = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of chunk c (16 B) of row r in a swizzled array with C channels
template <int C>
__device__ __forceinline__ uint32_t swz_off(int r, int c) {
    constexpr int CPV = C / 8;
    int cs = CPV == 4 ? (c ^ ((r >> 1) & 3)) : (c ^ ((r >> 2) & 1));
    return (uint32_t)(r * C * 2 + cs * 16);
}

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                        uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                          uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                          uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// GELU(z) = z Phi(z), evaluated in the tanh form of Hendrycks and Gimpel,
// 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))), with the hardware tanh
// approximation. The tanh form is within 4.8e-4 (absolute, at z = 2.7) of
// z Phi(z) for every z, and its derivative within 8.7e-4 of Phi(z) + z phi(z);
// both stay below the BF16 rounding of the stored activations, and the form
// costs about a quarter of the instructions of the erf form. gelu_grad_f is
// the derivative of the same tanh form.
constexpr float GELU_C = 0.7978845608028654f;  // sqrt(2/pi)
constexpr float GELU_A = 0.044715f;

__device__ __forceinline__ float tanh_approx(float u) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    return t;
}

__device__ __forceinline__ float gelu_f(float z) {
    const float t = tanh_approx(z * fmaf(GELU_A * GELU_C, z * z, GELU_C));
    const float hz = 0.5f * z;
    return fmaf(hz, t, hz);
}

__device__ __forceinline__ float gelu_grad_f(float z) {
    const float z2 = z * z;
    const float t = tanh_approx(z * fmaf(GELU_A * GELU_C, z2, GELU_C));
    // d/dz [0.5 z (1 + t)] = 0.5 (1 + t) + 0.5 z (1 - t^2) sqrt(2/pi) (1 + 3 a z^2)
    const float du = fmaf(3.0f * GELU_A * GELU_C, z2, GELU_C);
    return fmaf(0.5f * z * fmaf(-t, t, 1.0f), du, 0.5f * (1.0f + t));
}

// Loads the 18 x 10 x 3 input halo of the tile at (x0, y0, z0) into smem.
template <int C>
__device__ __forceinline__ void load_halo(const bf16 *__restrict__ in, int n, int x0, int y0,
                                          int z0, unsigned char *halo) {
    constexpr int CPV = C / 8;
    for (int idx = threadIdx.x; idx < CV_HALO * CPV; idx += blockDim.x) {
        const int hr = idx / CPV, c = idx % CPV;
        const int hx = hr % CV_HX, hy = (hr / CV_HX) % CV_HY, hz = hr / (CV_HX * CV_HY);
        const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gx >= 0 && gy >= 0 && gz >= 0 && gx < n && gy < n && gz < n)
            v = *reinterpret_cast<const uint4 *>(
                in + ((size_t)c * n * n * n + ((size_t)gz * n + gy) * n + gx) * 8);
        *reinterpret_cast<uint4 *>(halo + swz_off<C>(hr, c)) = v;
    }
}

// Partial weight gradients of tap plane dz = blockIdx.y - 1 over the tiles of
// chunk blockIdx.x: part[chunk][tap][co][ci] (taps of the plane only) and,
// for blockIdx.y == 0, the bias-gradient partial part_b[chunk][co].
template <int CIN, int COUT>
__global__ void __launch_bounds__(CV_THREADS) k_wgrad(const bf16 *__restrict__ in,
                                                      const bf16 *__restrict__ g, int n,
                                                      int tiles_per_chunk,
                                                      float *__restrict__ part,
                                                      float *__restrict__ part_b) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *gsm = smem;                       // [128][COUT]
    unsigned char *halo = smem + 128 * COUT * 2;     // [540][CIN]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int dz = (int)blockIdx.y - 1;
    const int tiles_x = n / CV_TX, tiles_y = n / CV_TY;
    const int ntiles = tiles_x * tiles_y * n;
    constexpr int MT = COUT / 16, NT = CIN / 8;
    constexpr int ITEMS = 9 * MT;                      // (tap in plane, m tile)
    constexpr int PER_WARP = (ITEMS + 7) / 8;
    float acc[PER_WARP][NT][4];
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.0f;
    float bsum = 0.0f;
    const uint32_t gbase = smem_u32(gsm), hbase = smem_u32(halo);
    const int t0 = blockIdx.x * tiles_per_chunk, t1 = min(ntiles, t0 + tiles_per_chunk);
    for (int tile = t0; tile < t1; ++tile) {
        const int tx = tile % tiles_x, ty = (tile / tiles_x) % tiles_y, z0 = tile / (tiles_x * tiles_y);
        const int x0 = tx * CV_TX, y0 = ty * CV_TY;
        __syncthreads();
        load_halo<CIN>(in, n, x0, y0, z0, halo);
        constexpr int GCPV = COUT / 8;
        for (int idx = threadIdx.x; idx < 128 * GCPV; idx += blockDim.x) {
            const int kv = idx / GCPV, c = idx % GCPV;
            const size_t v = ((size_t)z0 * n + (y0 + kv / 16)) * n + x0 + kv % 16;
            *reinterpret_cast<uint4 *>(gsm + swz_off<COUT>(kv, c)) =
                *reinterpret_cast<const uint4 *>(g + ((size_t)c * n * n * n + v) * 8);
        }
        __syncthreads();
        if (blockIdx.y == 0 && threadIdx.x < COUT) {
            for (int kv = 0; kv < 128; ++kv) {
                const bf16 *row = reinterpret_cast<const bf16 *>(gsm + swz_off<COUT>(kv, threadIdx.x / 8));
                bsum += __bfloat162float(row[threadIdx.x % 8]);
            }
        }
#pragma unroll
        for (int i = 0; i < PER_WARP; ++i) {
            const int item = w + 8 * i;
            if (item >= ITEMS) break;
            const int tl = item / MT, mt = item % MT;  // tap in plane, m tile
            const int dx = tl % 3 - 1, dy = tl / 3 - 1;
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
                uint32_t a0, a1, a2, a3;
                {
                    const int kv = ks * 16 + ((lane >> 4) << 3) + (lane & 7);
                    ldsm_x4_t(a0, a1, a2, a3, gbase + swz_off<COUT>(kv, 2 * mt + ((lane >> 3) & 1)));
                }
                const int kvb = ks * 16 + (((lane >> 3) & 1) << 3) + (lane & 7);
                const int hr = ((dz + 1) * CV_HY + (kvb / 16 + dy + 1)) * CV_HX + (kvb % 16 + dx + 1);
#pragma unroll
                for (int jj = 0; jj < NT / 2; ++jj) {
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4_t(b0, b1, b2, b3, hbase + swz_off<CIN>(hr, 2 * jj + (lane >> 4)));
                    mma_16816(acc[i][2 * jj], a0, a1, a2, a3, b0, b1);
                    mma_16816(acc[i][2 * jj + 1], a0, a1, a2, a3, b2, b3);
                }
            }
        }
    }
    // write partials: row co = 16 mt + gid (+8), col ci = 8 j + 2 tig (+1)
    float *pc = part + (size_t)blockIdx.x * 27 * COUT * CIN;
#pragma unroll
    for (int i = 0; i < PER_WARP; ++i) {
        const int item = w + 8 * i;
        if (item >= ITEMS) break;
        const int tl = item / MT, mt = item % MT;
        const int tap = (dz + 1) * 9 + tl;
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int co = 16 * mt + gid + 8 * h, ci = 8 * j + 2 * tig;
                *reinterpret_cast<float2 *>(pc + ((size_t)tap * COUT + co) * CIN + ci) =
                    make_float2(acc[i][j][2 * h], acc[i][j][2 * h + 1]);
            }
    }
    if (blockIdx.y == 0 && threadIdx.x < COUT) part_b[(size_t)blockIdx.x * COUT + threadIdx.x] = bsum;
}

template <int CIN, int COUT>
constexpr size_t wgrad_smem() {
    return (size_t)128 * COUT * 2 + (size_t)CV_HALO * CIN * 2;
}

}  // namespace dw

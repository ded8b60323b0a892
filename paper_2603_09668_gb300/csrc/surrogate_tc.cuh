// 3x3x3 convolutions of the surrogate network on the fifth-generation tensor
// cores: tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in tensor
// memory), operands in shared memory filled by TMA, one MMA-issuing thread
// per CTA.
//
// Activations are stored planar, [C/8][n^3][8] BF16: plane c holds channels
// 8c..8c+7 of every voxel (16 B per voxel, voxels x fastest), so that a row of
// a tile's halo is one contiguous run of 16-byte voxel records.
//
// The convolution out[v][co] = sum_{tap, ci} W[tap][co][ci] in[v + d(tap)][ci]
// (zero padding) is an implicit GEMM: for an output tile of 8 (x) x 16 (y) x
// 1 (z) voxels, M = 128 voxels, N = COUT, K = 27 taps x CIN. The input halo
// of the tile (10 x 18 x 3 voxels) is loaded by TMA, one box per 8-channel
// plane (box {8 ch, 10, 18, 3, 1} of the 5D view [C/8][z][y][x][8], zero fill
// outside the volume), so that each plane lands as 16-byte voxel rows ordered
// (z, y, x). In that
// "chunk plane" layout the A operand of every tap is a plain shared-memory
// matrix descriptor without swizzling: the 8 x-voxels of one tile row form a
// core matrix (8 rows x 16 B, contiguous), tile rows are 10 voxels (160 B)
// apart (stride-dimension offset), and the next 8 channels are one plane
// further (leading-dimension offset). Shifting the descriptor's start by the
// tap's voxel offset selects the tap: no im2col copy exists anywhere.
// The weights sit in shared memory as [tap][chunk][co][8 ci] (core matrices
// of 8 output channels x 16 B).
//
// Per tile one thread waits for the halo, issues 27 x CIN/16 MMAs
// (128 x COUT x 16 each) into a 32-column tensor-memory accumulator and
// commits them to an mbarrier; when they complete, the halo of the next tile
// is requested (overlapping the epilogue) and the four warps read their 32
// accumulator lanes (one voxel per thread) with tcgen05.ld, add the bias,
// apply the epilogue and store channels-last. Every wait is bounded; a wait
// that runs out sets the error word, drains what is in flight (bounded) and
// frees the tensor memory before the kernel returns.
#pragma once

#include <cuda.h>

#include "surrogate_conv.cuh"

namespace dw {

constexpr int TC_TX = 8, TC_TY = 16;                 // output tile (x, y), z = 1
constexpr int TC_HX = TC_TX + 2, TC_HY = TC_TY + 2;  // halo 10 x 18 x 3
constexpr int TC_PLANE_BYTES = TC_HX * TC_HY * 3 * 16;   // 8640 B of one chunk
constexpr int TC_PLANE = 8704;                        // plane stride, 128-B aligned

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // shared-memory matrix descriptor: start, leading and stride byte offsets
    // (all >> 4), descriptor version 1 (bit 46), no swizzle, base offset 0
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity of an mbarrier; false after about
// a second, or as soon as *abort (if given) is set.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity,
                                        const volatile int *abort) {
    uint64_t t0 = 0;
    for (unsigned it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 0) {
            if (abort && *abort) return false;
            const uint64_t t = globaltimer_ns();
            if (it == 0) t0 = t;
            else if (t - t0 > 1000000000ull) return false;
        }
    }
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMA loads of the halo planes of the tile at (x0, y0, z0), completing on bar.
template <int CIN>
__device__ __forceinline__ void tc_load_halo(const CUtensorMap *tm, uint32_t halo, uint32_t bar,
                                             int x0, int y0, int z0) {
    constexpr int KCH = CIN / 8;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(KCH * TC_PLANE_BYTES) : "memory");
#pragma unroll
    for (int c = 0; c < KCH; ++c)
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
            :: "r"(halo + c * TC_PLANE), "l"((uint64_t)tm), "r"(0), "r"(x0 - 1), "r"(y0 - 1),
               "r"(z0 - 1), "r"(c), "r"(bar)
            : "memory");
}

// tcgen05.ld of N consecutive 32-bit accumulator columns of this warp's 32
// lanes (one row per thread).
template <int N>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&r)[N]);

template <>
__device__ __forceinline__ void tc_ld<16>(uint32_t taddr, float (&r)[16]) {
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
          "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
          "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}

template <>
__device__ __forceinline__ void tc_ld<8>(uint32_t taddr, float (&r)[8]) {
    uint32_t u[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]),
                   "=r"(u[6]), "=r"(u[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

constexpr int TC_NST = 3;        // halo stages
constexpr int TC_EPI_WARPS = 8;  // epilogue warps: lane quarter = warp & 3, column half = warp >> 2
constexpr int TC_THREADS = 32 * (TC_EPI_WARPS + 1);  // + one producer / MMA warp
constexpr int TC_TMEM_COLS = 64;                      // two 32-column accumulators

template <int CIN, int COUT>
constexpr size_t tc_smem() {
    return (size_t)TC_NST * (CIN / 8) * TC_PLANE + (size_t)27 * (CIN / 8) * COUT * 16 + 1024;
}

// Epilogues: EPI_GELU (z and GELU(z) in BF16), EPI_GELU_ONLY (GELU(z)),
// EPI_F32 (z in FP32), EPI_DGELU (acc * GELU'(zprev), BF16). wt holds the
// weights in the operand layout [27][CIN/8][COUT][8].
//
// Roles: warp 8, lane 0 issues the weight copy and the halo loads (a ring of
// TC_NST stages) and the MMAs of every tile into accumulator k % 2; warps 0-7
// read accumulator k % 2, release it, and run the epilogue. mbarriers:
// full[s] (halo landed), empty[s] (the MMAs that read stage s are done),
// accf[a] (accumulator a complete), acce[a] (accumulator a read out).
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(TC_THREADS, 1) k_conv3_tc(
    const __grid_constant__ CUtensorMap tm_in, const bf16 *__restrict__ wt,
    const float *__restrict__ bias, int n, bf16 *__restrict__ out_z, bf16 *__restrict__ out_a,
    float *__restrict__ out_f, const bf16 *__restrict__ zprev, int *err) {
    static_assert(CIN % 16 == 0 && (COUT == 16 || COUT == 32), "unsupported shape");
    constexpr int KCH = CIN / 8;
    constexpr int HBYTES = KCH * TC_PLANE;
    constexpr int WBYTES = 27 * KCH * COUT * 16;
    constexpr int CPW = COUT / 2;  // accumulator columns per epilogue warp
    constexpr uint32_t IDESC = tc_idesc(COUT);
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_NST], empty[TC_NST], accf[2], acce[2], wbar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t hbase = smem_u32(smem), wbase = hbase + TC_NST * HBYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        abort_flag = 0;
        for (int i = 0; i < TC_NST; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&accf[i]), 1);
            mbar_init(smem_u32(&acce[i]), TC_EPI_WARPS);
        }
        mbar_init(smem_u32(&wbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;
    const volatile int *abort_p = &abort_flag;

    const int tiles_x = n / TC_TX, tiles_y = n / TC_TY;
    const int ntiles = tiles_x * tiles_y * n;
    const int K = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    // Programmatic dependent launch: the next layer may be scheduled now (it
    // gets an SM when a CTA of this grid exits); this grid's inputs (the
    // previous layer's output) are read only after griddepcontrol.wait, while
    // the weights, written before the first layer's launch, may be read before.
    pdl_trigger();
    if (warp == TC_EPI_WARPS) {
        if (lane == 0) {
            int issued = 0, consumed = 0, committed = 0;
            auto load = [&](int k) {
                const int t = blockIdx.x + k * gridDim.x;
                tc_load_halo<CIN>(&tm_in, hbase + (k % TC_NST) * HBYTES,
                                  smem_u32(&full[k % TC_NST]), (t % tiles_x) * TC_TX,
                                  ((t / tiles_x) % tiles_y) * TC_TY, t / (tiles_x * tiles_y));
            };
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(smem_u32(&wbar)), "r"(WBYTES) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                :: "r"(wbase), "l"(wt), "r"(WBYTES), "r"(smem_u32(&wbar)) : "memory");
            pdl_wait();
            for (; issued < TC_NST && issued < K; ++issued) load(issued);
            bool ok = tc_wait(smem_u32(&wbar), 0, abort_p);
            for (int k = 0; k < K && ok; ++k) {
                const int s = k % TC_NST, a = k & 1;
                ok = tc_wait(smem_u32(&full[s]), (k / TC_NST) & 1, abort_p);
                if (!ok) break;
                ++consumed;
                ok = tc_wait(smem_u32(&acce[a]), ((k >> 1) & 1) ^ 1, abort_p);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d = taddr + a * 32;
                // descriptors = stage / weight base + compile-time offsets (>> 4) of
                // every (tap, k-step): the unrolled loop issues MMAs back to back
                const uint64_t a0 = tc_desc(hbase + s * HBYTES, TC_PLANE, TC_HX * 16);
                const uint64_t b0 = tc_desc(wbase, COUT * 16, 128);
#pragma unroll
                for (int t = 0; t < 27; ++t) {
                    const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;  // offsets + 1
#pragma unroll
                    for (int kk = 0; kk < KCH / 2; ++kk) {
                        const uint32_t a_off = ((dz * TC_HY + dy) * TC_HX + dx) * 16 + 2 * kk * TC_PLANE;
                        const uint32_t b_off = ((t * KCH + 2 * kk) * COUT) * 16;
                        const uint64_t ad = a0 + (a_off >> 4);
                        const uint64_t bd = b0 + (b_off >> 4);
                        const uint32_t acc = (t | kk) != 0;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                            :: "r"(d), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                            : "memory");
                    }
                }
                tc_commit(smem_u32(&empty[s]));
                tc_commit(smem_u32(&accf[a]));
                ++committed;
                // refill the stage of tile k - 1 (its MMAs were issued one tile earlier)
                if (k >= 1 && issued < K) {
                    const int k1 = k - 1;
                    ok = tc_wait(smem_u32(&empty[k1 % TC_NST]), (k1 / TC_NST) & 1, abort_p);
                    if (!ok) break;
                    load(issued++);
                }
            }
            if (!ok) {
                if (!abort_flag) atomicOr(err, ERRBIT_TIMEOUT);
                abort_flag = 1;
            }
            // drain: halo loads still in flight and the last MMA batch (bounded)
            for (int k = consumed; k < issued; ++k)
                tc_wait(smem_u32(&full[k % TC_NST]), (k / TC_NST) & 1, nullptr);
            if (committed > 0)
                tc_wait(smem_u32(&empty[(committed - 1) % TC_NST]), ((committed - 1) / TC_NST) & 1, nullptr);
        }
        __syncwarp();  // the warp reconverges before the final CTA barrier
    } else {
        const int q = warp & 3, hcol = warp >> 2;
        const int row = q * 32 + lane;  // accumulator lane = tile voxel (x = row & 7, y = row >> 3)
        for (int k = 0; k < K; ++k) {
            const int a = k & 1;
            int ok = 1;  // lane 0 waits for the warp, so the warp stays converged
            if (lane == 0) {
                ok = tc_wait(smem_u32(&accf[a]), (k >> 1) & 1, abort_p);
                if (!ok) {
                    if (!abort_flag) atomicOr(err, ERRBIT_TIMEOUT);
                    abort_flag = 1;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            tc_fence_after();
            float r[CPW];
            tc_ld<CPW>(taddr + ((uint32_t)(q * 32) << 16) + a * 32 + hcol * CPW, r);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acce[a]));
            const int t = blockIdx.x + k * gridDim.x;
            const int x0 = (t % tiles_x) * TC_TX, y0 = ((t / tiles_x) % tiles_y) * TC_TY;
            const int z0 = t / (tiles_x * tiles_y);
            const size_t v = ((size_t)z0 * n + (y0 + (row >> 3))) * n + x0 + (row & 7);
            const size_t nv = (size_t)n * n * n;
            const int c0 = hcol * CPW;
            // planar BF16 outputs: channels c..c+7 of voxel v at ((c / 8) nv + v) * 8
            auto plane = [&](int c) { return ((size_t)((c0 + c) >> 3) * nv + v) * 8; };
            if (EPI == EPI_F32) {
#pragma unroll
                for (int c = 0; c < CPW; c += 4)
                    *reinterpret_cast<float4 *>(out_f + v * COUT + c0 + c) =
                        make_float4(r[c] + bias[c0 + c], r[c + 1] + bias[c0 + c + 1],
                                    r[c + 2] + bias[c0 + c + 2], r[c + 3] + bias[c0 + c + 3]);
            } else if (EPI == EPI_DGELU) {
#pragma unroll
                for (int c = 0; c < CPW; c += 8) {
                    const uint4 zp = *reinterpret_cast<const uint4 *>(zprev + plane(c));
                    const bf16 *zb = reinterpret_cast<const bf16 *>(&zp);
                    __align__(16) bf16 o[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        o[j] = __float2bfloat16_rn(r[c + j] * gelu_grad_f(__bfloat162float(zb[j])));
                    *reinterpret_cast<uint4 *>(out_z + plane(c)) = *reinterpret_cast<const uint4 *>(o);
                }
            } else {
#pragma unroll
                for (int c = 0; c < CPW; c += 8) {
                    __align__(16) bf16 oz[8], oa[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float z = r[c + j] + bias[c0 + c + j];
                        oz[j] = __float2bfloat16_rn(z);
                        oa[j] = __float2bfloat16_rn(gelu_f(z));
                    }
                    if (EPI == EPI_GELU)
                        *reinterpret_cast<uint4 *>(out_z + plane(c)) = *reinterpret_cast<const uint4 *>(oz);
                    *reinterpret_cast<uint4 *>(out_a + plane(c)) = *reinterpret_cast<const uint4 *>(oa);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(taddr), "r"(TC_TMEM_COLS));
    }
}

}  // namespace dw

// Weight gradients of the surrogate network's 3x3x3 convolutions on the
// fifth-generation tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32
// accumulators in tensor memory, operands loaded by TMA).
//
// dW[tap][co][ci] = sum_v g[v][co] in[v + d(tap)][ci] (zero padding) is a
// GEMM over voxels (K). For each (dy, dz) pair of taps one MMA computes
//   D_(dy,dz)[(dx, ci)][co] += sum_{v in a row of 16 x-voxels}
//                              in[v + (dx, dy, dz) - 1][ci] g[v][co]
// with M = 128 rows = 4 dx slots x 32 input channels (the fourth slot, and
// for CIN = 16 the upper half of every slot, are rows whose results are not
// read), N = COUT, K = 16 voxels. Both operands are MN-major: in the planar
// activation layout [C/8][n^3][8] a voxel's 8 channels are one 16-byte row,
// and 8 consecutive voxels of one 8-channel plane form a core matrix (8 K
// rows x 16 B). The input is loaded three times per tile, shifted by dx =
// 0, 1, 2 voxels (three TMA boxes, 16-byte aligned in x because a voxel
// record is 16 bytes), into consecutive slots, so that every 8-row group of
// M, (dx, 8 channels), is one plane further: a uniform stride-dimension
// offset, which is what lets the three dx taps share one MMA. The nine
// (dy, dz) accumulators (9 COUT columns of tensor memory) stay in tensor
// memory over all of a CTA's tiles; the epilogue writes the CTA's partial sums
// once.
//
// Tiles: 16 (x) x 4 (y) voxels of one z slice. A tile's halo for the input is
// 3 slices x 6 rows x 16 voxels per dx slot. Roles: warp 4, lane 0 issues the
// TMA loads (a ring of WG_NST stages) and the MMAs; warps 0-3 wait for the
// last MMA and read the accumulators (warp w: rows 32 w .. 32 w + 31). Every
// wait is bounded (about a second): the kernel then sets ERRBIT_TIMEOUT,
// drains its copies and frees the tensor memory.
#pragma once

#include "surrogate_tc.cuh"

namespace dw {

constexpr int WG_TX = 16, WG_TY = 4;   // tile: 16 x-voxels (one K step) x 4 rows, one z slice
constexpr int WG_HY = WG_TY + 2;       // halo rows
constexpr int WG_ROW = WG_TX * 16;     // bytes of one row of 16 voxel records
constexpr int WG_PLANE = 3 * WG_HY * WG_ROW;  // one 8-channel plane of a slot: 3 slices x 6 rows
constexpr int WG_NST = 3;              // pipeline stages
constexpr int WG_EPI = 4;              // epilogue warps: tensor-memory rows 0-127
constexpr int WG_THREADS = 32 * (WG_EPI + 1);

template <int CIN>
constexpr int wg_slot() { return (CIN / 8) * WG_PLANE; }
template <int COUT>
constexpr int wg_gbytes() { return (COUT / 8) * WG_TY * WG_ROW; }
template <int CIN, int COUT>
constexpr int wg_stage() { return 3 * wg_slot<CIN>() + wg_gbytes<COUT>(); }
// The stages, plus what the M = 128 rows of the last stage's MMAs reach past
// it, plus alignment. An MMA's A operand starts at most 17 rows into a plane
// and spans 16 planes in M and 2 x 128 B in K: 16 planes from the stage start.
template <int CIN, int COUT>
constexpr size_t wg_smem() {
    constexpr int reach = (2 * WG_HY + WG_TY + 1) * WG_ROW + 15 * WG_PLANE + 2 * 128;
    constexpr int extra = reach > wg_stage<CIN, COUT>() ? reach - wg_stage<CIN, COUT>() : 0;
    return (size_t)WG_NST * wg_stage<CIN, COUT>() + extra + 1024;
}
template <int COUT>
constexpr int wg_tmem_cols() { return 9 * COUT <= 256 ? 256 : 512; }

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// MN-major (bits 15 and 16), M = 128, N = n.
__host__ __device__ constexpr uint32_t wg_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

struct WgPipe {
    uint64_t full[WG_NST], empty[WG_NST], done;
    uint32_t tmem_base;
    int abort_flag;
};

// Tiles of this CTA: a contiguous range of the layer's (x, y, z) tiles.
__device__ __forceinline__ void wg_range(int ntiles, int &t0, int &t1) {
    t0 = (int)((int64_t)ntiles * blockIdx.x / gridDim.x);
    t1 = (int)((int64_t)ntiles * (blockIdx.x + 1) / gridDim.x);
}

template <int CIN, int COUT>
__device__ __forceinline__ void wg_load(const CUtensorMap *tm_in, const CUtensorMap *tm_g,
                                        uint32_t stage, uint32_t bar, int n, int tile) {
    const int tx = n / WG_TX, ty = n / WG_TY;
    const int x0 = (tile % tx) * WG_TX, y0 = ((tile / tx) % ty) * WG_TY, z = tile / (tx * ty);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(wg_stage<CIN, COUT>()) : "memory");
#pragma unroll
    for (int d = 0; d < 3; ++d)
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];"
            :: "r"(stage + d * wg_slot<CIN>()), "l"((uint64_t)tm_in), "r"(8 * (x0 - 1 + d)),
               "r"(y0 - 1), "r"(z - 1), "r"(0), "r"(bar)
            : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];"
        :: "r"(stage + 3 * wg_slot<CIN>()), "l"((uint64_t)tm_g), "r"(8 * x0), "r"(y0), "r"(z),
           "r"(0), "r"(bar)
        : "memory");
}

// Partial weight gradients of CTA b: part[b][tap][co][ci] for the CTA's
// tiles. tm_in: the input activations as boxes {128, 6, 3, CIN/8}; tm_g: the
// output gradients as boxes {128, 4, 1, COUT/8} (both views [C/8][z][y][x * 8]).
template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS, 1) k_wgrad_tc(const __grid_constant__ CUtensorMap tm_in,
                                                            const __grid_constant__ CUtensorMap tm_g,
                                                            int n, float *__restrict__ part, int *err) {
    static_assert((CIN == 16 || CIN == 32) && (COUT == 16 || COUT == 32), "unsupported shape");
    constexpr int STAGE = wg_stage<CIN, COUT>(), SLOT = wg_slot<CIN>();
    constexpr int TCOLS = wg_tmem_cols<COUT>();
    constexpr uint32_t IDESC = wg_idesc(COUT);
    extern __shared__ unsigned char smem_raw[];
    __shared__ WgPipe pp;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        pp.abort_flag = 0;
        for (int i = 0; i < WG_NST; ++i) {
            mbar_init(smem_u32(&pp.full[i]), 1);
            mbar_init(smem_u32(&pp.empty[i]), 1);
        }
        mbar_init(smem_u32(&pp.done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&pp.tmem_base)), "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = pp.tmem_base;
    const volatile int *abort_p = &pp.abort_flag;
    const int ntiles = (n / WG_TX) * (n / WG_TY) * n;
    int t0, t1;
    wg_range(ntiles, t0, t1);
    const int cnt = t1 - t0;

    if (warp == WG_EPI) {
        if (lane == 0 && cnt > 0) {
            int issued = 0, consumed = 0;
            bool ok = true;
            while (issued < WG_NST && issued < cnt) {
                wg_load<CIN, COUT>(&tm_in, &tm_g, sbase + (issued % WG_NST) * STAGE,
                                   smem_u32(&pp.full[issued % WG_NST]), n, t0 + issued);
                ++issued;
            }
            for (int j = 0; j < cnt; ++j) {
                const int s = j % WG_NST;
                ok = tc_wait(smem_u32(&pp.full[s]), (j / WG_NST) & 1, abort_p);
                if (!ok) break;
                ++consumed;
                tc_fence_after();
                const uint32_t st = sbase + s * STAGE;
#pragma unroll
                for (int r = 0; r < WG_TY; ++r) {
                    const uint64_t bd = tc_desc(st + 3 * SLOT + r * WG_ROW, 128, WG_TY * WG_ROW);
#pragma unroll
                    for (int b = 0; b < 9; ++b) {  // b = 3 dz + dy
                        const int dz = b / 3, dy = b % 3;
                        const uint64_t ad = tc_desc(st + (dz * WG_HY + r + dy) * WG_ROW, 128, WG_PLANE);
                        const uint32_t d = taddr + (uint32_t)(b * COUT);
                        const uint32_t acc = (j | r) != 0;  // the CTA's first row starts each sum
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                            :: "r"(d), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                            : "memory");
                    }
                }
                tc_commit(smem_u32(&pp.empty[s]));
                // refill the stage of tile j - 1 (its MMAs were issued one tile ago)
                if (j >= 1 && issued < cnt) {
                    const int k1 = j - 1;
                    ok = tc_wait(smem_u32(&pp.empty[k1 % WG_NST]), (k1 / WG_NST) & 1, abort_p);
                    if (!ok) break;
                    wg_load<CIN, COUT>(&tm_in, &tm_g, sbase + (issued % WG_NST) * STAGE,
                                       smem_u32(&pp.full[issued % WG_NST]), n, t0 + issued);
                    ++issued;
                }
            }
            if (ok) {
                tc_commit(smem_u32(&pp.done));
            } else {
                atomicOr(err, ERRBIT_TIMEOUT);
                pp.abort_flag = 1;
            }
            // drain (bounded): copies still in flight, the last MMAs
            for (int k = consumed; k < issued; ++k)
                tc_wait(smem_u32(&pp.full[k % WG_NST]), (k / WG_NST) & 1, nullptr);
            if (consumed > 0)
                tc_wait(smem_u32(&pp.empty[(consumed - 1) % WG_NST]), ((consumed - 1) / WG_NST) & 1,
                        nullptr);
        }
        __syncwarp();
    } else {
        // rows 32 warp .. + 31: m = dx CIN + ci (rows from 3 CIN on are padding)
        const int m = 32 * warp + lane;
        float *pc = part + (size_t)blockIdx.x * 27 * COUT * CIN;
        int okw = 1;
        if (cnt > 0 && lane == 0) okw = tc_wait(smem_u32(&pp.done), 0, abort_p);
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (okw && cnt > 0) {
            tc_fence_after();
            const uint32_t tq = taddr + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
            for (int b = 0; b < 9; ++b) {
#pragma unroll
                for (int c0 = 0; c0 < COUT; c0 += 16) {
                    float r[16];
                    tc_ld<16>(tq + (uint32_t)(b * COUT + c0), r);
                    if (m < 3 * CIN) {
                        const int dx = m / CIN, ci = m % CIN, tap = 3 * b + dx;
#pragma unroll
                        for (int cc = 0; cc < 16; ++cc)
                            pc[((size_t)tap * COUT + c0 + cc) * CIN + ci] = r[cc];
                    }
                }
            }
        } else if (cnt == 0 && m < 3 * CIN) {
            const int dx = m / CIN, ci = m % CIN;
            for (int b = 0; b < 9; ++b)
                for (int co = 0; co < COUT; ++co) pc[((size_t)(3 * b + dx) * COUT + co) * CIN + ci] = 0.0f;
        } else if (!okw && lane == 0) {
            atomicOr(err, ERRBIT_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(TCOLS));
    }
}

// Bias-gradient partials: part_b[b][co] = sum over CTA b's voxels of g[v][co]
// (planar BF16 [COUT/8][nv][8]).
template <int COUT>
__global__ void __launch_bounds__(256) k_bias_grad(const bf16 *__restrict__ g, int64_t nv,
                                                   float *__restrict__ part_b) {
    constexpr int PL = COUT / 8;
    __shared__ float sum[COUT];
    if (threadIdx.x < COUT) sum[threadIdx.x] = 0.0f;
    __syncthreads();
    const int64_t v0 = nv * blockIdx.x / gridDim.x, v1 = nv * (blockIdx.x + 1) / gridDim.x;
    const int pl = threadIdx.x % PL;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t v = v0 + threadIdx.x / PL; v < v1; v += blockDim.x / PL) {
        const uint4 q = *reinterpret_cast<const uint4 *>(g + ((size_t)pl * nv + v) * 8);
        const bf16 *e = reinterpret_cast<const bf16 *>(&q);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += __bfloat162float(e[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) atomicAdd(&sum[8 * pl + j], acc[j]);
    __syncthreads();
    if (threadIdx.x < COUT) part_b[(size_t)blockIdx.x * COUT + threadIdx.x] = sum[threadIdx.x];
}

}  // namespace dw

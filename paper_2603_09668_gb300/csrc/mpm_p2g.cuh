// P2G (Eq. P2G plus the MLS-MPM stress momentum) in three accumulation
// strategies that give the same sums up to float rounding order:
//   DW_P2G_ATOMIC : every particle adds its 27 node contributions to the HBM
//                   grid with float4 atomics.
//   DW_P2G_WARP   : lanes of a warp whose particles share a base cell (runs of
//                   equal cell keys, as produced by mpm_sort) reduce their
//                   contributions with a segmented shuffle reduction; the run
//                   leader issues one float4 atomic per node.
//   DW_P2G_TILE   : a CTA accumulates its particles into a shared-memory tile
//                   spanning their stencils' bounding box (shared atomics, each
//                   lane walking the 27 nodes in a lane-rotated order so lanes
//                   of one cell hit distinct addresses), then flushes the
//                   non-empty tile nodes to HBM with float4 atomics. A CTA whose
//                   particles span more than the tile falls back to ATOMIC.
#pragma once

#include "mpm_math.cuh"

namespace dw {

// Affine momentum matrix A = -dt V0 (4/dx^2) P F^T + m C of one particle.
__device__ __forceinline__ bool p2g_affine(const MpmParams &P, const float F[9], const float C[9],
                                           float A[9]) {
    float Pk[9], PFt[9];
    bool ok = stress_P(P, F, Pk);
    mul3_abt(Pk, F, PFt);
#pragma unroll
    for (int k = 0; k < 9; ++k) A[k] = -P.kappa * PFt[k] + P.p_mass * C[k];
    return ok;
}

struct P2GParticle {
    Stencil s;
    float mv[3];  // m v
    float A[9];
    bool valid;
};

__device__ __forceinline__ void p2g_load(const MpmParams &P, const float *__restrict__ x,
                                         const float *__restrict__ v, const float *__restrict__ C,
                                         const float *__restrict__ F, int64_t n, int64_t p,
                                         P2GParticle &q, int *err) {
    q.valid = false;
    if (p >= n) return;
    float xp[3] = {x[p], x[n + p], x[2 * n + p]};
    if (!make_stencil(P, xp[0], xp[1], xp[2], q.s)) {
        atomicOr(err, ERRBIT_DOMAIN);
        return;
    }
    float Cp[9], Fp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Cp[k] = C[k * n + p];
        Fp[k] = F[k * n + p];
    }
    if (!p2g_affine(P, Fp, Cp, q.A)) atomicOr(err, ERRBIT_INVERTED);
#pragma unroll
    for (int a = 0; a < 3; ++a) q.mv[a] = P.p_mass * v[a * n + p];
    q.valid = true;
}

// Contribution of particle q to stencil node (oi, oj, ok): (m, p).
__device__ __forceinline__ float4 p2g_node_value(const MpmParams &P, const P2GParticle &q, float W,
                                                 float d0, float d1, float d2) {
    float4 r;
    r.x = W * P.p_mass;
    r.y = W * (q.mv[0] + q.A[0] * d0 + q.A[1] * d1 + q.A[2] * d2);
    r.z = W * (q.mv[1] + q.A[3] * d0 + q.A[4] * d1 + q.A[5] * d2);
    r.w = W * (q.mv[2] + q.A[6] * d0 + q.A[7] * d1 + q.A[8] * d2);
    return r;
}

__device__ __forceinline__ void p2g_scatter_global(const MpmParams &P, const P2GParticle &q,
                                                   float4 *__restrict__ grid) {
    const int N = P.N;
#pragma unroll
    for (int oi = 0; oi < 3; ++oi)
#pragma unroll
        for (int oj = 0; oj < 3; ++oj)
#pragma unroll
            for (int ok = 0; ok < 3; ++ok) {
                float W = q.s.w[0][oi] * q.s.w[1][oj] * q.s.w[2][ok];
                float4 val = p2g_node_value(P, q, W, ((float)oi - q.s.fx[0]) * P.dx,
                                            ((float)oj - q.s.fx[1]) * P.dx,
                                            ((float)ok - q.s.fx[2]) * P.dx);
                int64_t id = ((int64_t)(q.s.base[2] + ok) * N + (q.s.base[1] + oj)) * N + (q.s.base[0] + oi);
                atomicAdd(&grid[id], val);
            }
}

__global__ void __launch_bounds__(128) k_p2g_atomic(MpmParams P, const float *__restrict__ x,
                                                    const float *__restrict__ v,
                                                    const float *__restrict__ C,
                                                    const float *__restrict__ F, int64_t n,
                                                    float4 *__restrict__ grid, int *err) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    P2GParticle q;
    p2g_load(P, x, v, C, F, n, p, q, err);
    if (q.valid) p2g_scatter_global(P, q, grid);
}

// ------------------------------------------------------------ warp-aggregated

__global__ void __launch_bounds__(128) k_p2g_warp(MpmParams P, const float *__restrict__ x,
                                                  const float *__restrict__ v,
                                                  const float *__restrict__ C,
                                                  const float *__restrict__ F, int64_t n,
                                                  float4 *__restrict__ grid, int *err) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    P2GParticle q;
    p2g_load(P, x, v, C, F, n, p, q, err);
    const int N = P.N;
    int64_t key = q.valid ? ((int64_t)q.s.base[2] * N + q.s.base[1]) * N + q.s.base[0] : -1 - lane;
    int64_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    bool start = (lane == 0) || (prev != key) || !q.valid;
    unsigned starts = __ballot_sync(0xffffffffu, start);
    unsigned above = lane == 31 ? 0u : (starts & (0xffffffffu << (lane + 1)));
    int run_end = above ? (__ffs(above) - 1) : 32;
    if (starts == 0xffffffffu) {  // no two neighbouring lanes share a cell: plain atomics
        if (q.valid) p2g_scatter_global(P, q, grid);
        return;
    }
    if (!q.valid) {  // zero contributions keep the shuffles uniform
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            q.s.fx[a] = 1.0f;
#pragma unroll
            for (int o = 0; o < 3; ++o) q.s.w[a][o] = 0.0f;
        }
    }
#pragma unroll
    for (int oi = 0; oi < 3; ++oi)
#pragma unroll
        for (int oj = 0; oj < 3; ++oj)
#pragma unroll
            for (int ok = 0; ok < 3; ++ok) {
                float W = q.s.w[0][oi] * q.s.w[1][oj] * q.s.w[2][ok];
                float4 val = p2g_node_value(P, q, W, ((float)oi - q.s.fx[0]) * P.dx,
                                            ((float)oj - q.s.fx[1]) * P.dx,
                                            ((float)ok - q.s.fx[2]) * P.dx);
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    float4 y;
                    y.x = __shfl_down_sync(0xffffffffu, val.x, off);
                    y.y = __shfl_down_sync(0xffffffffu, val.y, off);
                    y.z = __shfl_down_sync(0xffffffffu, val.z, off);
                    y.w = __shfl_down_sync(0xffffffffu, val.w, off);
                    if (lane + off < run_end) {
                        val.x += y.x;
                        val.y += y.y;
                        val.z += y.z;
                        val.w += y.w;
                    }
                }
                if (start && q.valid) {
                    int64_t id = ((int64_t)(q.s.base[2] + ok) * N + (q.s.base[1] + oj)) * N + (q.s.base[0] + oi);
                    atomicAdd(&grid[id], val);
                }
            }
}

// --------------------------------------------------------------- tile ------

constexpr int P2G_TILE_THREADS = 256;
constexpr int P2G_TILE_NODES = 1024;

__device__ __forceinline__ float wsel(const float w[3], int o) {
    return o == 0 ? w[0] : (o == 1 ? w[1] : w[2]);
}

__global__ void __launch_bounds__(P2G_TILE_THREADS) k_p2g_tile(MpmParams P,
                                                               const float *__restrict__ x,
                                                               const float *__restrict__ v,
                                                               const float *__restrict__ C,
                                                               const float *__restrict__ F,
                                                               int64_t n, float4 *__restrict__ grid,
                                                               int *err) {
    __shared__ float tile[4][P2G_TILE_NODES];
    __shared__ int red_lo[3][P2G_TILE_THREADS / 32], red_hi[3][P2G_TILE_THREADS / 32];
    __shared__ int box[6];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int64_t p = (int64_t)blockIdx.x * P2G_TILE_THREADS + tid;
    P2GParticle q;
    p2g_load(P, x, v, C, F, n, p, q, err);
    // bounding box of the stencils' base cells
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = q.valid ? q.s.base[a] : 0x7fffffff;
        hi[a] = q.valid ? q.s.base[a] : -1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        if (lane == 0) {
            red_lo[a][wid] = lo[a];
            red_hi[a][wid] = hi[a];
        }
    }
    __syncthreads();
    if (tid < 3) {
        int l = 0x7fffffff, h = -1;
        for (int w = 0; w < P2G_TILE_THREADS / 32; ++w) {
            l = min(l, red_lo[tid][w]);
            h = max(h, red_hi[tid][w]);
        }
        box[tid] = l;
        box[3 + tid] = h;
    }
    __syncthreads();
    const int bx0 = box[0], by0 = box[1], bz0 = box[2];
    if (box[3] < 0) return;  // no valid particle in this CTA
    const int ex = box[3] - bx0 + 3, ey = box[4] - by0 + 3, ez = box[5] - bz0 + 3;
    const int vol = ex * ey * ez;
    const int N = P.N;
    if (vol > P2G_TILE_NODES) {
        if (q.valid) p2g_scatter_global(P, q, grid);
        return;
    }
    for (int i = tid; i < vol; i += P2G_TILE_THREADS) {
        tile[0][i] = 0.0f;
        tile[1][i] = 0.0f;
        tile[2][i] = 0.0f;
        tile[3][i] = 0.0f;
    }
    __syncthreads();
    if (q.valid) {
        const int lx = q.s.base[0] - bx0, ly = q.s.base[1] - by0, lz = q.s.base[2] - bz0;
        for (int step = 0; step < 27; ++step) {
            int o = step + lane;
            o = o >= 27 ? o - 27 : o;
            o = o >= 27 ? o - 27 : o;
            int oi = o % 3, oj = (o / 3) % 3, ok = o / 9;
            float W = wsel(q.s.w[0], oi) * wsel(q.s.w[1], oj) * wsel(q.s.w[2], ok);
            float4 val = p2g_node_value(P, q, W, ((float)oi - q.s.fx[0]) * P.dx,
                                        ((float)oj - q.s.fx[1]) * P.dx, ((float)ok - q.s.fx[2]) * P.dx);
            int li = ((lz + ok) * ey + (ly + oj)) * ex + (lx + oi);
            atomicAdd(&tile[0][li], val.x);
            atomicAdd(&tile[1][li], val.y);
            atomicAdd(&tile[2][li], val.z);
            atomicAdd(&tile[3][li], val.w);
        }
    }
    __syncthreads();
    for (int i = tid; i < vol; i += P2G_TILE_THREADS) {
        float m = tile[0][i];
        if (m == 0.0f) continue;
        int ix = i % ex, iy = (i / ex) % ey, iz = i / (ex * ey);
        int64_t id = ((int64_t)(bz0 + iz) * N + (by0 + iy)) * N + (bx0 + ix);
        atomicAdd(&grid[id], make_float4(m, tile[1][i], tile[2][i], tile[3][i]));
    }
}

inline dw_status launch_p2g(int mode, const MpmParams &P, const float *x, const float *v,
                            const float *C, const float *F, int64_t n, float4 *grid, int *err,
                            cudaStream_t st) {
    if (n == 0) return DW_OK;
    if (mode == DW_P2G_ATOMIC) {
        k_p2g_atomic<<<grid_for(n, 128), 128, 0, st>>>(P, x, v, C, F, n, grid, err);
    } else if (mode == DW_P2G_WARP) {
        k_p2g_warp<<<grid_for(n, 128), 128, 0, st>>>(P, x, v, C, F, n, grid, err);
    } else {
        k_p2g_tile<<<grid_for(n, P2G_TILE_THREADS), P2G_TILE_THREADS, 0, st>>>(P, x, v, C, F, n, grid, err);
    }
    DW_LAUNCHED("p2g");
    return DW_OK;
}

}  // namespace dw

// P2G kernels of the three accumulation strategies (see mpm_p2g.cuh) and
// their launcher.
#include "mpm_p2g.cuh"

namespace dw {

__global__ void __launch_bounds__(128) k_p2g_atomic(MpmParams P, const float *__restrict__ x,
                                                    const float *__restrict__ v,
                                                    const float *__restrict__ C,
                                                    const float *__restrict__ F, int64_t n,
                                                    float4 *__restrict__ grid, int *err,
                                                    ActiveBlocks ab) {
    pdl_wait();
    pdl_trigger();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    P2GParticle q;
    p2g_load(P, x, v, C, F, n, p, q, err);
    if (q.valid) {
        p2g_scatter_global(P, q, grid);
        if (ab.flags) mark_stencil_blocks(ab, q.s.base);
    }
}

__global__ void __launch_bounds__(P2G_WARP_THREADS) k_p2g_warp(MpmParams P,
                                                             const float *__restrict__ x,
                                                             const float *__restrict__ v,
                                                             const float *__restrict__ C,
                                                             const float *__restrict__ F,
                                                             int64_t n, float4 *__restrict__ grid,
                                                             int *err, ActiveBlocks ab) {
    __shared__ float4 rows[P2G_WARP_THREADS / 32][32][P2G_ROW];
    __shared__ int keys[P2G_WARP_THREADS / 32][32];
    pdl_wait();
    pdl_trigger();
    const int wid = threadIdx.x >> 5;
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    P2GParticle q;
    p2g_load(P, x, v, C, F, n, p, q, err);
    p2g_warp_scatter<true>(P, q, grid, ab, rows[wid], keys[wid]);
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
                                                               int *err, ActiveBlocks ab) {
    __shared__ float tile[4][P2G_TILE_NODES];
    __shared__ int red_lo[3][P2G_TILE_THREADS / 32], red_hi[3][P2G_TILE_THREADS / 32];
    __shared__ int box[6];
    pdl_wait();
    pdl_trigger();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int64_t p = (int64_t)blockIdx.x * P2G_TILE_THREADS + tid;
    P2GParticle q;
    p2g_load(P, x, v, C, F, n, p, q, err);
    if (ab.flags && q.valid) mark_stencil_blocks(ab, q.s.base);
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

dw_status launch_p2g(int mode, const MpmParams &P, const float *x, const float *v,
                            const float *C, const float *F, int64_t n, float4 *grid, int *err,
                            const ActiveBlocks &ab, cudaStream_t st) {
    if (n == 0) return DW_OK;
    if (mode == DW_P2G_ATOMIC) {
        DW_CUDA(launch_pdl(k_p2g_atomic, grid_for(n, 128), 128, st, P, x, v, C, F, n, grid, err, ab));
    } else if (mode == DW_P2G_WARP || mode == DW_P2G_AUTO || mode == DW_P2G_PAIR) {
        DW_CUDA(launch_pdl(k_p2g_warp, grid_for(n, P2G_WARP_THREADS), P2G_WARP_THREADS, st, P, x, v,
                           C, F, n, grid, err, ab));
    } else {
        DW_CUDA(launch_pdl(k_p2g_tile, grid_for(n, P2G_TILE_THREADS), P2G_TILE_THREADS, st, P, x, v,
                           C, F, n, grid, err, ab));
    }
    return DW_OK;
}

}  // namespace dw

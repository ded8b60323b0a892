// MLS-MPM substep S of Eq. simulation_mpm and its reverse mode, as a handle
// with a persistent workspace (grid, adjoint grid, per-particle scratch).
//
// Kernels per forward substep: P2G (particles -> grid), grid update (nodes),
// G2P (grid -> particles). Per adjoint substep: P2G + grid update recomputed
// from the input state, then reverse G2P (scatter dL/dv_i to the grid),
// reverse grid update (dL/dp_i, dL/dm_i, scatter into the wind-field
// gradient) and reverse P2G (gather the grid adjoint to the particles).
// Grid layout: float4 per node, node (i, j, k) at ((k N + j) N + i).
#include <stdio.h>

#include <mutex>
#include <new>
#include <vector>
#include <stdlib.h>

#include "mpm_adjoint.cuh"
#include "mpm_handle.cuh"

namespace dw {

// --------------------------------------------------------------- forward --

// Dense grid update over every node (used without an active-block list).
__global__ void k_grid_update(MpmParams P, WindDev wind, float t, float4 *__restrict__ grid_mp,
                              float4 *__restrict__ grid_v, int clear) {
    int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nn = (int64_t)P.N * P.N * P.N;
    if (node >= nn) return;
    int i = (int)(node % P.N), j = (int)((node / P.N) % P.N), k = (int)(node / ((int64_t)P.N * P.N));
    grid_node_update(P, wind, t, node, i, j, k, grid_mp, grid_v, clear);
}

// Grid update over the active blocks only; with clear, also zeroes (m, p)
// and the block flags so that the grid is empty for the next P2G.
__global__ void __launch_bounds__(GRID_THREADS) k_grid_update_active(
    MpmParams P, WindDev wind, float t, float4 *__restrict__ grid_mp, float4 *__restrict__ grid_v,
    int clear, ActiveBlocks ab) {
    pdl_wait();
    pdl_trigger();
    const int nblk = ab.nb * ab.nb * ab.nb;  // entries of the list
    const int sub = threadIdx.x >> 6, lt = threadIdx.x & 63, stride = gridDim.x * 4;
    int e = blockIdx.x * 4 + sub;
    // the first entry is read together with the count, not after it (an
    // entry past the count is read but not used)
    int b = e < nblk ? ab.list[e] : 0;
    const int count = *ab.count;
    for (; e < count; e += stride) {
        const int bn = e + stride < count ? ab.list[e + stride] : 0;  // the next entry
        int i, j, k;
        if (active_node(P, ab.nb, b, lt, i, j, k)) {
            int64_t node = ((int64_t)k * P.N + j) * P.N + i;
            grid_node_update(P, wind, t, node, i, j, k, grid_mp, grid_v, clear);
        }
        if (clear && lt == 0) ab.flags[b] = 0;
        b = bn;
    }
}

// The grid update (clear on) of a segment adjoint's recompute, which also
// keeps the consumed list and each listed node's (m, p) in a grid tape slot
// (entry e's nodes at gtape[64 e + t]).
__global__ void __launch_bounds__(GRID_THREADS) k_grid_update_tape(
    MpmParams P, WindDev wind, float t, float4 *__restrict__ grid_mp, float4 *__restrict__ grid_v,
    ActiveBlocks ab, float4 *__restrict__ gtape, int *__restrict__ gtape_list,
    int *__restrict__ gtape_count) {
    pdl_wait();
    pdl_trigger();
    const int count = *ab.count;
    if (blockIdx.x == 0 && threadIdx.x == 0) *gtape_count = count;
    const int sub = threadIdx.x >> 6, lt = threadIdx.x & 63;
    for (int e = blockIdx.x * 4 + sub; e < count; e += gridDim.x * 4) {
        const int b = ab.list[e];
        if (lt == 0) gtape_list[e] = b;
        int i, j, k;
        if (active_node(P, ab.nb, b, lt, i, j, k)) {
            const int64_t node = ((int64_t)k * P.N + j) * P.N + i;
            gtape[(size_t)e * 64 + lt] = grid_mp[node];
            grid_node_update(P, wind, t, node, i, j, k, grid_mp, grid_v, 1);
        }
        if (lt == 0) ab.flags[b] = 0;
    }
}

// A reverse substep's forward grid from a grid tape slot: the list and its
// count, the listed nodes' (m, p) written back and their grid update (grid
// kept), in place of a P2G of the substep's input and the grid update.
__global__ void __launch_bounds__(GRID_THREADS) k_grid_restore(
    MpmParams P, WindDev wind, float t, float4 *__restrict__ grid_mp, float4 *__restrict__ grid_v,
    ActiveBlocks ab, const float4 *__restrict__ gtape, const int *__restrict__ gtape_list,
    const int *__restrict__ gtape_count) {
    pdl_wait();
    pdl_trigger();
    const int count = *gtape_count;
    if (blockIdx.x == 0 && threadIdx.x == 0) *ab.count = count;
    const int sub = threadIdx.x >> 6, lt = threadIdx.x & 63;
    for (int e = blockIdx.x * 4 + sub; e < count; e += gridDim.x * 4) {
        const int b = gtape_list[e];
        if (lt == 0) ab.list[e] = b;
        int i, j, k;
        if (active_node(P, ab.nb, b, lt, i, j, k)) {
            const int64_t node = ((int64_t)k * P.N + j) * P.N + i;
            grid_mp[node] = gtape[(size_t)e * 64 + lt];
            grid_node_update(P, wind, t, node, i, j, k, grid_mp, grid_v, 0);
        }
    }
}

// x/xo and F/Fo may be the same arrays (in-place substep): every thread reads
// its particle before writing it, so they carry no __restrict__.
__global__ void k_g2p(MpmParams P, const float *x, const float *F,
                      const uint8_t *__restrict__ pinned, const float4 *__restrict__ grid_v,
                      float *xo, float *vo, float *Co, float *Fo, int64_t n, int *err,
                      int *reset_count) {
    pdl_wait();
    pdl_trigger();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (reset_count && p == 0) *reset_count = 0;  // the grid update has consumed the list
    if (p >= n) return;
    float xp[3] = {x[p], x[n + p], x[2 * n + p]};
    float Fp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Fp[k] = F[k * n + p];
    float vn[3], Cn[9];
    g2p_update(P, grid_v, pinned && pinned[p], xp, Fp, vn, Cn);  // out of range: unchanged
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        fin = fin && isfinite(xp[a]);
        xo[a * n + p] = xp[a];
        vo[a * n + p] = vn[a];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Co[k * n + p] = Cn[k];
        Fo[k * n + p] = Fp[k];
    }
    if (!fin || !finite9(Fp)) atomicOr(err, ERRBIT_NONFINITE);
}

// --------------------------------------------------------------- reverse --

// Reverse G2P: scatter dL/dv_i into grid_bv; write partial dL/dx_p, dL/dF_p.
// The node value W_ip (bv_p + D bC_p (x_i - x_p)) has the form of a P2G value
// (momentum m v + A (x_i - x_p) with m v -> bv, A -> D bC and no mass), so it
// goes through the same warp-aggregated scatter; grid_bv holds (0, dL/dv_i).
__global__ void __launch_bounds__(P2G_WARP_THREADS) k_rev_g2p(
    MpmParams P, const float *__restrict__ x, const float *__restrict__ F,
    const uint8_t *__restrict__ pinned, const float4 *__restrict__ grid_v,
    const float *__restrict__ gxo, const float *__restrict__ gvo, const float *__restrict__ gCo,
    const float *__restrict__ gFo, float4 *__restrict__ grid_bv, float *__restrict__ scratch,
    int64_t n, int64_t cap, const float *__restrict__ Cout) {
    __shared__ float4 rows[P2G_WARP_THREADS / 32][32][P2G_ROW];
    __shared__ int keys[P2G_WARP_THREADS / 32][32];
    pdl_wait();
    pdl_trigger();
    const int wid = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    P2GParticle q;
    q.valid = false;
    if (p < n) {
        float xp[3], Fp[9], bxo[3], bvo[3], bCo[9], bFo[9], bx[3], bFin[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xp[a] = x[a * n + p];
            bxo[a] = gxo[a * n + p];
            bvo[a] = gvo[a * n + p];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            Fp[k] = F[k * n + p];
            bCo[k] = gCo[k * n + p];
            bFo[k] = gFo[k * n + p];
        }
        rev_g2p_particle(P, xp, Fp, pinned && pinned[p], grid_v, bxo, bvo, bCo, bFo, q, bx, bFin,
                         Cout, n, p);
#pragma unroll
        for (int a = 0; a < 3; ++a) scratch[a * cap + p] = bx[a];
#pragma unroll
        for (int k = 0; k < 9; ++k) scratch[(3 + k) * cap + p] = bFin[k];
    }
    MpmParams Pz = P;
    Pz.p_mass = 0.0f;  // no mass channel: grid_bv = (0, dL/dv_i)
    const ActiveBlocks none{nullptr, nullptr, nullptr, 0, 0};
    p2g_warp_scatter<true>(Pz, q, grid_bv, none, rows[wid], keys[wid]);
}

__global__ void __launch_bounds__(GRID_THREADS) k_rev_grid_active(
    MpmParams P, WindDev wind, float t, float4 *__restrict__ grid_mp, float4 *__restrict__ grid_bv,
    float4 *__restrict__ grid_bmp, float *__restrict__ g_wind, ActiveBlocks ab) {
    __shared__ float sbox[GRID_THREADS / 32][WIND_BOX];
    pdl_wait();
    pdl_trigger();
    const int count = *ab.count;
    const int sub = threadIdx.x >> 6, lt = threadIdx.x & 63;
    // every lane of a 64-thread group runs the same iterations (one block each)
    for (int e = blockIdx.x * 4 + sub; e < count; e += gridDim.x * 4) {
        int b = ab.list[e];
        int i = 0, j = 0, k = 0;
        bool live = false;
        float3 gw;
        if (active_node(P, ab.nb, b, lt, i, j, k)) {
            int64_t node = ((int64_t)k * P.N + j) * P.N + i;
            live = rev_grid_node(P, node, i, j, k, grid_mp, grid_bv, grid_bmp, gw);
        }
        if (g_wind)
            wind_sample_adjoint_warp(wind, wind_scatter_coarse(P.N, wind.nf), live, i * P.dx,
                                     j * P.dx, k * P.dx, t, gw, g_wind, sbox[threadIdx.x >> 5]);
        if (lt == 0) ab.flags[b] = 0;
    }
}

__global__ void k_rev_p2g(MpmParams P, const float *__restrict__ x, const float *__restrict__ v,
                          const float *__restrict__ C, const float *__restrict__ F,
                          const float4 *__restrict__ grid_bmp, const float *__restrict__ scratch,
                          float *__restrict__ gx, float *__restrict__ gv, float *__restrict__ gC,
                          float *__restrict__ gF, float *__restrict__ g_E, int64_t n, int64_t cap,
                          int *reset_count) {
    pdl_wait();
    pdl_trigger();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (reset_count && p == 0) *reset_count = 0;  // the reverse grid update has consumed the list
    float gE_local = 0.0f;
    if (p < n) {
        float xp[3], vp[3], Cp[9], Fp[9], bx[3], bF[9], bvp[3], bC[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xp[a] = x[a * n + p];
            vp[a] = v[a * n + p];
            bx[a] = scratch[a * cap + p];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            Cp[k] = C[k * n + p];
            Fp[k] = F[k * n + p];
            bF[k] = scratch[(3 + k) * cap + p];
        }
        rev_p2g_particle(P, xp, vp, Cp, Fp, grid_bmp, bx, bF, bvp, bC, gE_local);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gx[a * n + p] = bx[a];
            gv[a * n + p] = bvp[a];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            gC[k * n + p] = bC[k];
            gF[k * n + p] = bF[k];
        }
    }
    if (g_E) {  // one atomic per block
        const float sum = block_sum(gE_local);
        if (threadIdx.x == 0) atomicAdd(g_E, sum);
    }
}

// ------------------------------------------------------------------ sort --

// Launched with whole warps (blocks of 256 threads): one count atomic per
// distinct key of a warp (between re-sorts most particles keep their cell, so
// a warp holds a few keys).
__global__ void k_sort_keys(MpmParams P, int nb, const float *__restrict__ x, int64_t n,
                            int *__restrict__ keys, int *__restrict__ counts) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = p < n;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!ok) return;
    const int k = cell_key(P, nb, x[p], x[n + p], x[2 * n + p]);
    keys[p] = k;
    const unsigned peers = __match_any_sync(act, k);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&counts[k], __popc(peers));
}

// Exclusive scan, three phases: per-block scan of SCAN_ITEMS consecutive
// elements per thread with block totals, scan of the totals (single block,
// loops over chunks), add-back; the last two are one launch for at most
// SCAN_BLOCK blocks.

__device__ __forceinline__ int block_exclusive_scan(int v, int *smem_warp, int &total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) smem_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? smem_warp[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < nw) smem_warp[lane] = si - s;
        if (lane == nw - 1) smem_warp[32] = si;
    }
    __syncthreads();
    total = smem_warp[32];
    int res = incl - v + smem_warp[wid];
    __syncthreads();
    return res;
}

// SCAN_ITEMS elements of one thread: 16-byte pieces when the whole run lies
// inside the array (data is 16-byte aligned, runs start at multiples of 8).
__device__ __forceinline__ void scan_load(const int *data, int64_t len, int64_t i0, int (&v)[SCAN_ITEMS]) {
    if (i0 + SCAN_ITEMS <= len) {
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j += 4) {
            const int4 q = *reinterpret_cast<const int4 *>(data + i0 + j);
            v[j] = q.x;
            v[j + 1] = q.y;
            v[j + 2] = q.z;
            v[j + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) v[j] = i0 + j < len ? data[i0 + j] : 0;
    }
}

__device__ __forceinline__ void scan_store(int *data, int64_t len, int64_t i0, const int (&v)[SCAN_ITEMS]) {
    if (i0 + SCAN_ITEMS <= len) {
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; j += 4)
            *reinterpret_cast<int4 *>(data + i0 + j) = make_int4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j)
            if (i0 + j < len) data[i0 + j] = v[j];
    }
}

__global__ void k_scan_blocks(int *__restrict__ data, int64_t len, int *__restrict__ block_sums) {
    __shared__ int sw[33];
    const int64_t i0 = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    scan_load(data, len, i0, v);
    int run = 0;  // exclusive scan of the thread's elements
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        const int t = v[j];
        v[j] = run;
        run += t;
    }
    int total;
    const int ex = block_exclusive_scan(run, sw, total);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) v[j] += ex;
    scan_store(data, len, i0, v);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int *__restrict__ sums, int64_t nblocks) {
    __shared__ int sw[33];
    int carry = 0;
    for (int64_t base = 0; base < nblocks; base += SCAN_BLOCK) {
        int64_t i = base + threadIdx.x;
        int v = i < nblocks ? sums[i] : 0;
        int total;
        int ex = block_exclusive_scan(v, sw, total);
        if (i < nblocks) sums[i] = ex + carry;
        carry += total;
    }
}

__global__ void k_scan_add(int *__restrict__ data, int64_t len, const int *__restrict__ sums) {
    const int64_t i0 = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    const int add = sums[blockIdx.x];
    int v[SCAN_ITEMS];
    scan_load(data, len, i0, v);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) v[j] += add;
    scan_store(data, len, i0, v);
}

// The add-back for at most SCAN_BLOCK blocks, with the scan of the totals
// folded in: block b sums the totals of blocks 0 .. b - 1 itself.
__global__ void k_scan_add_prefix(int *__restrict__ data, int64_t len, const int *__restrict__ sums) {
    __shared__ int sw[33];
    const int b = blockIdx.x;
    int add;
    block_exclusive_scan((int)threadIdx.x < b ? sums[threadIdx.x] : 0, sw, add);
    const int64_t i0 = (int64_t)b * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    scan_load(data, len, i0, v);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) v[j] += add;
    scan_store(data, len, i0, v);
}

// The scatter and the permutation in one pass (launched with whole warps,
// blocks of 256 threads): particle p, at position pos of its key's range
// (the lanes of a warp that share a key take consecutive positions in lane
// order from one offset atomic), moves its rows to pos of the output arrays;
// ids_out[pos] = ids_in[p] (p without ids_in). v and C may be left out
// (NULL).
__global__ void k_sort_move(const int *__restrict__ keys, int64_t n, int *__restrict__ offsets,
                            const float *__restrict__ x, const float *__restrict__ v,
                            const float *__restrict__ C, const float *__restrict__ F,
                            const uint8_t *__restrict__ pin_in, const int *__restrict__ ids_in,
                            float *__restrict__ xo, float *__restrict__ vo, float *__restrict__ Co,
                            float *__restrict__ Fo, uint8_t *__restrict__ pin_out,
                            int *__restrict__ ids_out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = p < n;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!ok) return;
    const int key = keys[p];
    const unsigned peers = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&offsets[key], __popc(peers));
    base = __shfl_sync(act, base, leader);
    const int64_t k = base + __popc(peers & ((1u << lane) - 1u));
    ids_out[k] = ids_in ? ids_in[p] : (int)p;
#pragma unroll
    for (int a = 0; a < 3; ++a) xo[a * n + k] = x[a * n + p];
#pragma unroll
    for (int c = 0; c < 9; ++c) Fo[c * n + k] = F[c * n + p];
    if (v) {
#pragma unroll
        for (int a = 0; a < 3; ++a) vo[a * n + k] = v[a * n + p];
#pragma unroll
        for (int c = 0; c < 9; ++c) Co[c * n + k] = C[c * n + p];
    }
    if (pin_in) pin_out[k] = pin_in[p];
}

dw_status exclusive_scan(int *data, int64_t len, int *tmp, int64_t tmp_len, cudaStream_t st) {
    int64_t nblocks = (len + SCAN_TILE - 1) / SCAN_TILE;
    if (((uintptr_t)data & 15) != 0) {
        set_error("scan data must be 16-byte aligned");
        return DW_ERR_ARG;
    }
    if (nblocks > tmp_len) {
        set_error("scan workspace too small");
        return DW_ERR_ARG;
    }
    k_scan_blocks<<<(unsigned)nblocks, SCAN_BLOCK, 0, st>>>(data, len, tmp);
    if (nblocks <= SCAN_BLOCK) {  // one thread per block total: two launches
        k_scan_add_prefix<<<(unsigned)nblocks, SCAN_BLOCK, 0, st>>>(data, len, tmp);
    } else {
        k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(tmp, nblocks);
        k_scan_add<<<(unsigned)nblocks, SCAN_BLOCK, 0, st>>>(data, len, tmp);
    }
    DW_LAUNCHED("exclusive scan");
    return DW_OK;
}

// --------------------------------------------------------------- helpers --

dw_status check_state(const MpmHandle *h, const dw_mpm_state *s, const char *name) {
    DW_REQUIRE(s != nullptr, "%s state is NULL", name);
    DW_REQUIRE(s->n >= 0 && s->n <= h->desc.max_particles,
               "%s state has n=%lld particles; the handle holds at most %lld", name,
               (long long)s->n, (long long)h->desc.max_particles);
    DW_REQUIRE(s->n == 0 || (s->x && s->v && s->C && s->F), "%s state has a NULL array", name);
    return DW_OK;
}

static dw_status launch_grid_update(MpmHandle *h, const WindDev &wd, float t, int clear,
                                    cudaStream_t st) {
    ProfScope ps(h, DW_K_GRID, st);
    DW_CUDA(launch_pdl(k_grid_update_active, GRID_CTAS, GRID_THREADS, st, h->P, wd, t, h->grid_mp,
                       h->grid_v, clear, active_blocks(h)));
    return DW_OK;
}

}  // namespace dw

using namespace dw;


namespace dw {

dw_status validate_desc(const dw_mpm_desc *desc) {
    DW_REQUIRE(desc->n_grid >= 8 && desc->n_grid <= 512, "n_grid=%d out of range [8, 512]", desc->n_grid);
    DW_REQUIRE(desc->dt > 0.0f, "dt must be > 0");
    DW_REQUIRE(desc->bc_band >= 0 && desc->bc_band < desc->n_grid / 2, "bc_band out of range");
    DW_REQUIRE(desc->material == DW_NEOHOOKEAN || desc->material == DW_FIXED_COROTATED,
               "unknown material %d", desc->material);
    DW_REQUIRE(desc->E > 0.0f && desc->nu >= 0.0f && desc->nu < 0.5f, "need E > 0 and 0 <= nu < 0.5");
    DW_REQUIRE(desc->p_mass > 0.0f && desc->p_vol > 0.0f, "p_mass and p_vol must be > 0");
    DW_REQUIRE(desc->max_particles >= 0 && desc->max_particles < (1ll << 31),
               "max_particles out of range");
    DW_REQUIRE(desc->p2g_mode >= DW_P2G_AUTO && desc->p2g_mode <= DW_P2G_PAIR, "unknown p2g_mode");
    return DW_OK;
}

}  // namespace dw

extern "C" dw_status mpm_create(const dw_mpm_desc *desc, dw_mpm *out) {
    DW_REQUIRE(desc && out, "desc/out must not be NULL");
    *out = nullptr;
    dw_status st = validate_desc(desc);
    if (st != DW_OK) return st;
    dw_mpm h = new (std::nothrow) dw_mpm_s();
    if (!h) {
        set_error("out of host memory");
        return DW_ERR_OOM;
    }
    h->desc = *desc;
    fill_params(h);
    int N = desc->n_grid;
    h->n_nodes = (int64_t)N * N * N;
    h->nb = (N + 3) / 4;
    h->n_keys = (int64_t)h->nb * h->nb * h->nb * 64;
    h->scan_tmp_len = (h->n_keys + SCAN_BLOCK) / SCAN_BLOCK + 1;
    int64_t cap = desc->max_particles > 0 ? desc->max_particles : 1;
    cudaError_t e = cudaSuccess;
    size_t gbytes = sizeof(float4) * (size_t)h->n_nodes;
#define DW_ALLOC(ptr, bytes) \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes))
    DW_ALLOC(h->grid_mp, gbytes);
    DW_ALLOC(h->grid_v, gbytes);
    DW_ALLOC(h->grid_bv, gbytes);
    DW_ALLOC(h->grid_bmp, gbytes);
    DW_ALLOC(h->pscratch, sizeof(float) * 12 * (size_t)cap);
    DW_ALLOC(h->err, sizeof(int));
    DW_ALLOC(h->keys, sizeof(int) * (size_t)cap);
    DW_ALLOC(h->counts, sizeof(int) * (size_t)(h->n_keys + 1));
    DW_ALLOC(h->scan_tmp, sizeof(int) * (size_t)h->scan_tmp_len);
    const size_t nblk = (size_t)h->nb * h->nb * h->nb;
    h->nblk = (int64_t)nblk;
    DW_ALLOC(h->block_flag, sizeof(int) * nblk);
    DW_ALLOC(h->block_list, sizeof(int) * 2 * nblk);
    DW_ALLOC(h->block_count, sizeof(int) * 2);
    DW_ALLOC(h->roll_state, sizeof(float) * 24 * (size_t)cap);
    DW_ALLOC(h->roll_pinned, (size_t)cap);
    DW_ALLOC(h->roll_ids, sizeof(int32_t) * (size_t)cap);
#undef DW_ALLOC
    if (e == cudaSuccess) e = cudaMemset(h->grid_mp, 0, gbytes);
    if (e == cudaSuccess) e = cudaMemset(h->grid_bv, 0, gbytes);
    if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->block_flag, 0, sizeof(int) * nblk);
    if (e == cudaSuccess) e = cudaMemset(h->block_count, 0, sizeof(int) * 2);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dw_status st = cuda_fail(e, "mpm_create");
        mpm_destroy(h);
        return st;
    }
    *out = h;
    return DW_OK;
}

extern "C" dw_status mpm_destroy(dw_mpm h) {
    if (!h) return DW_OK;
    cudaFree(h->grid_mp);
    cudaFree(h->grid_v);
    cudaFree(h->grid_bv);
    cudaFree(h->grid_bmp);
    cudaFree(h->pscratch);
    cudaFree(h->err);
    cudaFree(h->keys);
    cudaFree(h->counts);
    cudaFree(h->scan_tmp);
    cudaFree(h->block_flag);
    cudaFree(h->block_list);
    cudaFree(h->block_count);
    cudaFree(h->roll_state);
    cudaFree(h->roll_pinned);
    cudaFree(h->roll_ids);
    cudaFree(h->gtape);
    cudaFree(h->gtape_list);
    cudaFree(h->gtape_count);
    profile_free(h);
    delete h;
    return DW_OK;
}

extern "C" dw_status mpm_profile_enable(dw_mpm h, int32_t max_records) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(max_records >= 0 && max_records <= (1 << 20), "max_records out of range");
    profile_free(h);
    h->ev_start.resize(max_records);
    h->ev_stop.resize(max_records);
    h->ev_kernel.assign(max_records, 0);
    for (int i = 0; i < max_records; ++i) {
        DW_CUDA(cudaEventCreate(&h->ev_start[i]));
        DW_CUDA(cudaEventCreate(&h->ev_stop[i]));
    }
    return DW_OK;
}

extern "C" dw_status mpm_profile_read(dw_mpm h, double *total_ms, int64_t *launches) {
    DW_REQUIRE(h && total_ms && launches, "arguments must not be NULL");
    for (int k = 0; k < DW_K_COUNT; ++k) {
        total_ms[k] = 0.0;
        launches[k] = 0;
    }
    for (int i = 0; i < h->prof_used; ++i) {
        DW_CUDA(cudaEventSynchronize(h->ev_stop[i]));
        float ms = 0.0f;
        DW_CUDA(cudaEventElapsedTime(&ms, h->ev_start[i], h->ev_stop[i]));
        total_ms[h->ev_kernel[i]] += ms;
        launches[h->ev_kernel[i]] += 1;
    }
    h->prof_used = 0;
    return DW_OK;
}

extern "C" dw_status mpm_set_material(dw_mpm h, float E, float nu) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(E > 0.0f && nu >= 0.0f && nu < 0.5f, "need E > 0 and 0 <= nu < 0.5");
    h->desc.E = E;
    h->desc.nu = nu;
    fill_params(h);
    return DW_OK;
}

// The substep; tape_slot >= 0 (a segment adjoint's recompute) also keeps
// the grid in that slot of the handle's grid tape.
static dw_status substep_impl(dw_mpm h, const dw_mpm_state *in, const dw_mpm_state *out,
                              const uint8_t *pinned, const dw_wind_field *wind, float t,
                              dw_stream stream, int tape_slot) {
    DW_REQUIRE(h, "handle is NULL");
    dw_status st = check_state(h, in, "input");
    if (st != DW_OK) return st;
    st = check_state(h, out, "output");
    if (st != DW_OK) return st;
    DW_REQUIRE(in->n == out->n, "input and output particle counts differ");
    WindDev wd;
    st = wind_check(wind, &wd);
    if (st != DW_OK) return st;
    cudaStream_t s = as_stream(stream);
    int64_t n = in->n;
    {
        ProfScope ps(h, DW_K_P2G, s);
        st = launch_p2g(h->desc.p2g_mode, h->P, in->x, in->v, in->C, in->F, n, h->grid_mp, h->err,
                        active_blocks(h), s);
    }
    if (st != DW_OK) return st;
    if (tape_slot >= 0) {
        ProfScope ps(h, DW_K_GRID, s);
        DW_CUDA(launch_pdl(k_grid_update_tape, GRID_CTAS, GRID_THREADS, s, h->P, wd, t, h->grid_mp,
                           h->grid_v, active_blocks(h), h->gtape + (size_t)tape_slot * h->nblk * 64,
                           h->gtape_list + (size_t)tape_slot * h->nblk, h->gtape_count + tape_slot));
    } else {
        st = launch_grid_update(h, wd, t, 1, s);
        if (st != DW_OK) return st;
    }
    if (n > 0) {
        ProfScope ps(h, DW_K_G2P, s);
        DW_CUDA(launch_pdl(k_g2p, grid_for(n, 128), 128, s, h->P, (const float *)in->x,
                           (const float *)in->F, pinned, (const float4 *)h->grid_v, out->x, out->v,
                           out->C, out->F, n, h->err, h->block_count));
    }
    return DW_OK;
}

extern "C" dw_status mpm_substep(dw_mpm h, const dw_mpm_state *in, const dw_mpm_state *out,
                                 const uint8_t *pinned, const dw_wind_field *wind, float t,
                                 dw_stream stream) {
    return substep_impl(h, in, out, pinned, wind, t, stream, -1);
}

// The reverse substep; Cout (or NULL): C of the substep's output state, when
// the caller kept it (a segment's recomputed states); tape_slot >= 0: the
// substep's forward grid is in that slot of the handle's grid tape.
static dw_status substep_adjoint(dw_mpm h, const dw_mpm_state *in, const float *Cout,
                                 const dw_mpm_state *g_out, const dw_mpm_state *g_in,
                                 const uint8_t *pinned, const dw_wind_field *wind, float t,
                                 float *g_wind, float *g_E, dw_stream stream, int tape_slot = -1) {
    DW_REQUIRE(h, "handle is NULL");
    dw_status st = check_state(h, in, "input");
    if (st != DW_OK) return st;
    st = check_state(h, g_out, "g_out");
    if (st != DW_OK) return st;
    st = check_state(h, g_in, "g_in");
    if (st != DW_OK) return st;
    DW_REQUIRE(in->n == g_out->n && in->n == g_in->n, "particle counts differ");
    WindDev wd;
    st = wind_check(wind, &wd);
    if (st != DW_OK) return st;
    cudaStream_t s = as_stream(stream);
    int64_t n = in->n;
    int64_t cap = h->desc.max_particles > 0 ? h->desc.max_particles : 1;
    if (tape_slot >= 0) {
        ProfScope ps(h, DW_K_GRID, s);
        DW_CUDA(launch_pdl(k_grid_restore, GRID_CTAS, GRID_THREADS, s, h->P, wd, t, h->grid_mp,
                           h->grid_v, active_blocks(h), h->gtape + (size_t)tape_slot * h->nblk * 64,
                           h->gtape_list + (size_t)tape_slot * h->nblk, h->gtape_count + tape_slot));
    } else {
        {
            ProfScope ps(h, DW_K_P2G, s);
            st = launch_p2g(h->desc.p2g_mode, h->P, in->x, in->v, in->C, in->F, n, h->grid_mp,
                            h->err, active_blocks(h), s);
        }
        if (st != DW_OK) return st;
        st = launch_grid_update(h, wd, t, 0, s);
        if (st != DW_OK) return st;
    }
    if (n > 0) {
        ProfScope ps(h, DW_K_REV_G2P, s);
        DW_CUDA(launch_pdl(k_rev_g2p, grid_for(n, P2G_WARP_THREADS), P2G_WARP_THREADS, s, h->P,
                           in->x, in->F, pinned, h->grid_v, g_out->x, g_out->v, g_out->C,
                           g_out->F, h->grid_bv, h->pscratch, n, cap, Cout));
    }
    {
        ProfScope ps(h, DW_K_REV_GRID, s);
        DW_CUDA(launch_pdl(k_rev_grid_active, GRID_CTAS, GRID_THREADS, s, h->P, wd, t, h->grid_mp,
                           h->grid_bv, h->grid_bmp, g_wind, active_blocks(h)));
    }
    if (n > 0) {
        ProfScope ps(h, DW_K_REV_P2G, s);
        DW_CUDA(launch_pdl(k_rev_p2g, grid_for(n, 128), 128, s, h->P, in->x, in->v, in->C, in->F,
                           h->grid_bmp, h->pscratch, g_in->x, g_in->v, g_in->C, g_in->F, g_E, n,
                           cap, h->block_count));
    }
    return DW_OK;
}

extern "C" dw_status mpm_substep_adjoint(dw_mpm h, const dw_mpm_state *in,
                                         const dw_mpm_state *g_out, const dw_mpm_state *g_in,
                                         const uint8_t *pinned, const dw_wind_field *wind,
                                         float t, float *g_wind, float *g_E, dw_stream stream) {
    return substep_adjoint(h, in, nullptr, g_out, g_in, pinned, wind, t, g_wind, g_E, stream);
}

// The grid tape for `slots` recomputed substeps, grown on demand (nblk
// entries of 64 nodes' (m, p) per slot: 4 MB at 64^3, 34 MB at 128^3); taken
// only while it leaves 8 GB of device memory free. Returns whether it is
// there; without it the reverse pass rebuilds each grid by a P2G.
static bool ensure_grid_tape(MpmHandle *h, int slots) {
    if (slots <= 0) return false;
    if (slots <= h->gtape_slots) return true;
    if (h->gtape_refused && slots >= h->gtape_refused) return false;
    const size_t bytes = (size_t)slots * ((size_t)h->nblk * (64 * sizeof(float4) + sizeof(int)) + sizeof(int));
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || bytes + (8ull << 30) > free_b) {
        cudaGetLastError();
        h->gtape_refused = slots;
        return false;
    }
    cudaFree(h->gtape);
    cudaFree(h->gtape_list);
    cudaFree(h->gtape_count);
    h->gtape = nullptr;
    h->gtape_list = h->gtape_count = nullptr;
    h->gtape_slots = 0;
    cudaError_t e = cudaMalloc((void **)&h->gtape, (size_t)slots * h->nblk * 64 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->gtape_list, (size_t)slots * h->nblk * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->gtape_count, (size_t)slots * sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->gtape);
        cudaFree(h->gtape_list);
        cudaFree(h->gtape_count);
        h->gtape = nullptr;
        h->gtape_list = h->gtape_count = nullptr;
        h->gtape_refused = slots;
        return false;
    }
    h->gtape_slots = slots;
    return true;
}

extern "C" dw_status mpm_segment_adjoint(dw_mpm h, const dw_mpm_state *start, float *tape,
                                         int64_t tape_floats, const dw_mpm_state *g,
                                         const uint8_t *pinned, const dw_wind_field *wind,
                                         float t0, int32_t n_substeps, float *g_wind, float *g_E,
                                         dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    dw_status st = check_state(h, start, "start");
    if (st != DW_OK) return st;
    st = check_state(h, g, "gradient");
    if (st != DW_OK) return st;
    DW_REQUIRE(start->n == g->n, "start and gradient particle counts differ");
    DW_REQUIRE(n_substeps >= 0, "n_substeps must be >= 0");
    const int64_t n = start->n;
    if (n_substeps == 0) return DW_OK;
    const int64_t need = (int64_t)(n_substeps - 1) * 24 * n;
    DW_REQUIRE(n_substeps == 1 || (tape && tape_floats >= need),
               "tape holds %lld floats; %d substeps of %lld particles need %lld",
               (long long)tape_floats, n_substeps, (long long)n, (long long)need);
    const float dt = h->P.dt;
    auto slot = [&](int k) {  // state k (1 .. n_substeps - 1) in the tape
        dw_mpm_state s;
        float *b = tape + (size_t)(k - 1) * 24 * (size_t)n;
        s.x = b;
        s.v = b + 3 * n;
        s.C = b + 6 * n;
        s.F = b + 15 * n;
        s.n = n;
        return s;
    };
    // the recompute keeps each substep's grid when the grid tape fits; with
    // the paired kernel it runs as one fused chain
    const bool gt = ensure_grid_tape(h, n_substeps - 1);
    if (h->desc.p2g_mode == DW_P2G_AUTO || h->desc.p2g_mode == DW_P2G_PAIR) {
        WindDev wd;
        st = wind_check(wind, &wd);
        if (st != DW_OK) return st;
        st = segment_recompute(h, start, tape, pinned, wd, t0, n_substeps, gt, as_stream(stream));
        if (st != DW_OK) return st;
    } else {
        for (int k = 1; k < n_substeps; ++k) {
            const dw_mpm_state in = k == 1 ? *start : slot(k - 1), out = slot(k);
            st = substep_impl(h, &in, &out, pinned, wind, fmaf((float)(k - 1), dt, t0), stream,
                              gt ? k - 1 : -1);
            if (st != DW_OK) return st;
        }
    }
    for (int j = n_substeps - 1; j >= 0; --j) {
        const dw_mpm_state in = j == 0 ? *start : slot(j);
        // the output state j + 1 and substep j's grid are kept for every substep but the last
        const bool kept = j + 1 < n_substeps;
        st = substep_adjoint(h, &in, kept ? slot(j + 1).C : nullptr, g, g, pinned, wind,
                             fmaf((float)j, dt, t0), g_wind, g_E, stream, kept && gt ? j : -1);
        if (st != DW_OK) return st;
    }
    return DW_OK;
}

namespace dw {

dw_status sort_particles(MpmHandle *h, const dw_mpm_state *in, const dw_mpm_state *out,
                         const uint8_t *pinned_in, uint8_t *pinned_out, const int32_t *ids_in,
                         int32_t *ids_out, cudaStream_t s, bool with_vc, bool keys_ready,
                         bool clear_after) {
    int64_t n = in->n;
    if (n == 0) return DW_OK;
    ProfScope ps(h, DW_K_SORT, s);
    if (!keys_ready) {
        DW_CUDA(cudaMemsetAsync(h->counts, 0, sizeof(int) * (size_t)(h->n_keys + 1), s));
        k_sort_keys<<<grid_for(n, 256), 256, 0, s>>>(h->P, h->nb, in->x, n, h->keys, h->counts);
        DW_LAUNCHED("k_sort_keys");
    }
    dw_status st = exclusive_scan(h->counts, h->n_keys, h->scan_tmp, h->scan_tmp_len, s);
    if (st != DW_OK) return st;
    k_sort_move<<<grid_for(n, 256), 256, 0, s>>>(h->keys, n, h->counts, in->x,
                                                 with_vc ? in->v : nullptr, with_vc ? in->C : nullptr,
                                                 in->F, pinned_in, ids_in, out->x, out->v, out->C,
                                                 out->F, pinned_out, ids_out);
    DW_LAUNCHED("k_sort_move");
    if (clear_after) DW_CUDA(cudaMemsetAsync(h->counts, 0, sizeof(int) * (size_t)(h->n_keys + 1), s));
    return DW_OK;
}

}  // namespace dw

extern "C" dw_status mpm_sort(dw_mpm h, const dw_mpm_state *in, const dw_mpm_state *out,
                              const uint8_t *pinned_in, uint8_t *pinned_out,
                              const int32_t *ids_in, int32_t *ids_out, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    dw_status st = check_state(h, in, "input");
    if (st != DW_OK) return st;
    st = check_state(h, out, "output");
    if (st != DW_OK) return st;
    DW_REQUIRE(in->n == out->n, "input and output particle counts differ");
    DW_REQUIRE(in->n == 0 || in->x != out->x, "mpm_sort cannot run in place");
    DW_REQUIRE(!pinned_in || pinned_out, "pinned_out must be given with pinned_in");
    if (in->n == 0) return DW_OK;
    DW_REQUIRE(ids_out, "ids_out must not be NULL");
    DW_REQUIRE(!ids_in || ids_in != ids_out, "ids_in and ids_out must differ");
    return sort_particles(h, in, out, pinned_in, pinned_out, ids_in, ids_out, as_stream(stream));
}

extern "C" dw_status mpm_device_status(dw_mpm h, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    int bits = 0;
    cudaStream_t s = as_stream(stream);
    DW_CUDA(cudaMemcpyAsync(&bits, h->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DW_CUDA(cudaStreamSynchronize(s));
    DW_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int), s));
    DW_CUDA(cudaStreamSynchronize(s));
    return status_from_bits(bits);
}

// ---------------------------------------------------------------------------
// mpm_substep_noalloc: one substep whose scratch grid lives in fixed device
// memory that is part of the loaded library, so the call allocates nothing.
//
// Who needs it: callers that may not allocate device memory at the moment
// they want a substep - code running under a caching allocator's callback or
// inside its lock, a real-time control loop whose rules forbid allocation
// after start-up, or a host framework that has handed the whole device to its
// own memory pool and only lends out input and output buffers. Such callers
// cannot use mpm_create, whose workspace comes from cudaMalloc.
//
// The array below is sized for grids of up to NOALLOC_MAX_GRID^3 nodes and is
// held by every GPU that loads the library until the process exits.
namespace dw {

constexpr int NOALLOC_MAX_GRID = 64;
constexpr int64_t NOALLOC_MAX_NODES = (int64_t)NOALLOC_MAX_GRID * NOALLOC_MAX_GRID * NOALLOC_MAX_GRID;
constexpr int NOALLOC_MAX_DEVICES = 64;

// [0, N^3): (m, p) after P2G; [NOALLOC_MAX_NODES, + N^3): (v, m) after the grid update
static __device__ __align__(256) float4 g_noalloc_grid[2 * NOALLOC_MAX_NODES];
static __device__ __align__(256) int g_noalloc_status;

struct NoallocAddr {
    float4 *grid = nullptr;
    int *status = nullptr;
};
static NoallocAddr g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

// Device addresses of the static arrays on the current device, looked up once
// per device (host code cannot use the symbols' names as device addresses).
static dw_status noalloc_addresses(NoallocAddr *out) {
    int dev = 0;
    DW_CUDA(cudaGetDevice(&dev));
    DW_REQUIRE(dev >= 0 && dev < NOALLOC_MAX_DEVICES, "device %d beyond the supported %d", dev,
               NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocAddr &a = g_noalloc_addr[dev];
    if (!a.grid) {
        void *g = nullptr, *s = nullptr;
        DW_CUDA(cudaGetSymbolAddress(&g, g_noalloc_grid));
        DW_CUDA(cudaGetSymbolAddress(&s, g_noalloc_status));
        a.grid = (float4 *)g;
        a.status = (int *)s;
    }
    *out = a;
    return DW_OK;
}

}  // namespace dw

extern "C" dw_status mpm_substep_noalloc(const dw_mpm_desc *desc, const dw_mpm_state *in,
                                         const dw_mpm_state *out, const uint8_t *pinned,
                                         const dw_wind_field *wind, float t,
                                         int32_t *device_status, dw_stream stream) {
    DW_REQUIRE(desc, "desc must not be NULL");
    DW_REQUIRE(desc->n_grid >= 8 && desc->n_grid <= NOALLOC_MAX_GRID,
               "mpm_substep_noalloc supports n_grid in [8, %d] (its fixed grid holds %lld "
               "nodes); got n_grid=%d", NOALLOC_MAX_GRID, (long long)NOALLOC_MAX_NODES,
               desc->n_grid);
    DW_REQUIRE(desc->dt > 0.0f, "dt must be > 0");
    DW_REQUIRE(desc->bc_band >= 0 && desc->bc_band < desc->n_grid / 2, "bc_band out of range");
    DW_REQUIRE(desc->material == DW_NEOHOOKEAN || desc->material == DW_FIXED_COROTATED,
               "unknown material %d", desc->material);
    DW_REQUIRE(desc->E > 0.0f && desc->nu >= 0.0f && desc->nu < 0.5f, "need E > 0 and 0 <= nu < 0.5");
    DW_REQUIRE(desc->p_mass > 0.0f && desc->p_vol > 0.0f, "p_mass and p_vol must be > 0");
    DW_REQUIRE(desc->p2g_mode >= DW_P2G_AUTO && desc->p2g_mode <= DW_P2G_PAIR, "unknown p2g_mode");
    DW_REQUIRE(in && out, "in/out must not be NULL");
    DW_REQUIRE(in->n >= 0 && in->n == out->n && in->n < (1ll << 31), "bad particle counts");
    DW_REQUIRE(in->n == 0 || (in->x && in->v && in->C && in->F && out->x && out->v && out->C && out->F),
               "state arrays must not be NULL");
    WindDev wd;
    dw_status st = wind_check(wind, &wd);
    if (st != DW_OK) return st;
    NoallocAddr a;
    st = noalloc_addresses(&a);
    if (st != DW_OK) return st;
    MpmHandle tmp;  // host-side parameter holder only; no device memory
    tmp.desc = *desc;
    fill_params(&tmp);
    const MpmParams P = tmp.P;
    const int64_t nodes = (int64_t)desc->n_grid * desc->n_grid * desc->n_grid;
    float4 *grid_mp = a.grid;
    float4 *grid_v = a.grid + NOALLOC_MAX_NODES;
    int *err = device_status ? (int *)device_status : a.status;
    cudaStream_t s = as_stream(stream);
    // the previous call left the array with its contents: P2G needs zeros
    DW_CUDA(cudaMemsetAsync(grid_mp, 0, sizeof(float4) * (size_t)nodes, s));
    int64_t n = in->n;
    const ActiveBlocks dense{nullptr, nullptr, nullptr, 0};
    st = launch_p2g(desc->p2g_mode, P, in->x, in->v, in->C, in->F, n, grid_mp, err, dense, s);
    if (st != DW_OK) return st;
    k_grid_update<<<grid_for(nodes, 256), 256, 0, s>>>(P, wd, t, grid_mp, grid_v, 1);
    DW_LAUNCHED("k_grid_update");
    if (n > 0) {
        k_g2p<<<grid_for(n, 128), 128, 0, s>>>(P, in->x, in->F, pinned, grid_v, out->x, out->v,
                                               out->C, out->F, n, err, nullptr);
        DW_LAUNCHED("k_g2p");
    }
    return DW_OK;
}

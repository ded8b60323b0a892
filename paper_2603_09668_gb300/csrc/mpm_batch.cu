// mpm_batch: many independent MPM scenes advanced together, each substep one
// launch over all of them.
//
// Every scene runs the substep of mpm_rollout (Eq. simulation_mpm: P2G, grid
// update with gravity, wind (Sec. 3.3) and the sticky band, G2P with the F
// update), with its own grid, parameters and wind field. The particles of all
// scenes live in one concatenated SoA state; a static table splits it into
// 128-particle work items that never straddle two scenes, and the active 4^3
// node blocks of all scenes go into one list whose entries carry the scene
// (scene << 20 | block).
//
// Persistent mode: one cooperative launch per substep k. Phase A: the CTAs
// stride over the active-block list of substep k and update those nodes
// (reading and clearing (m, p), writing (v, m)). A grid-wide barrier with a
// bounded wait. Phase B: the CTAs stride over the work items; each particle
// gathers the new grid velocities (G2P of substep k, loads through L2 because
// other CTAs wrote them in phase A), updates x and F, and scatters itself into
// its scene's cleared grid (P2G of substep k + 1), appending newly touched
// blocks to the other list. The last substep of the rollout stores v and C
// instead of scattering; a re-sort runs between two launches (after the P2G
// of the substep that follows it, v and C not kept). Split mode runs the
// phases as two kernels with programmatic dependent launch. Pair mode is
// split mode whose scattering phase B is the two-particles-per-thread body of
// mpm_rollout (k_batch_pair: 64 particles of one scene per warp); the last
// substep of the rollout, and the recompute of a reverse segment, run the
// split-mode kernels.
//
// The sort is one counting sort over all scenes: scene s's keys are offset by
// the number of keys of the scenes before it, so the sorted order keeps every
// scene inside its own particle range.
//
// Reverse mode (checkpointed segments): the states inside a segment are
// recomputed one substep at a time into a caller-owned tape, and the grid
// phase of each recomputed substep keeps its active list and the listed
// nodes' (m, p) in a handle-owned grid tape (when device memory allows).
// Each reverse substep then runs over all scenes at once: the forward grid
// of the substep restored from the grid tape with its grid update (or, for
// the segment's last substep and without a grid tape, a P2G of the
// substep's input and the grid update), reverse G2P (scatter of dL/dv_i into
// each scene's adjoint grid), reverse grid update (dL/dm_i, dL/dp_i, the
// scene's wind gradient) and reverse P2G (gather to the particles, per-scene
// dL/dE).
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "mpm_adjoint.cuh"
#include "mpm_handle.cuh"
#include "mpm_pair_warp.cuh"

namespace dw {

constexpr int BATCH_ITEM = 128;         // particles per work item
constexpr int BATCH_SCENE_SHIFT = 20;   // list entry = scene << 20 | block
constexpr int BATCH_MAX_SCENES = 2048;  // scene < 2^11 keeps entries positive
constexpr unsigned BATCH_SPIN_LIMIT = 1u << 20;  // about a second of polling

struct BatchScene {
    MpmParams P;
    WindDev wind;
    float4 *grid_mp;
    float4 *grid_v;
    int *flags;      // [nb^3]
    int nb;
    int key_offset;  // first sort key of the scene
};

// Arguments of one launch over the batch.
struct BatchView {
    const BatchScene *scenes;
    const int4 *items;  // (scene, first particle, count, 0)
    int n_items;
    float *x, *v, *C, *F;  // concatenated state, stride n
    // when set, the substep writes its whole output state (x, v, C, F) here
    // instead of updating x and F in place (the recompute of a reverse
    // segment, state k in, state k + 1 out)
    float *ox, *ov, *oC, *oF;
    const uint8_t *pinned;
    int64_t n;
    int *list;   // [2][list_cap]
    int *count;  // [2]
    int list_cap;
    int *err;
    unsigned *bar;      // grid barrier: arrivals, generation
    const float *t0;    // time of substep 0 (device, set before each rollout)
    // when set (the recompute of a reverse segment), the grid phase also
    // keeps the consumed list and each listed node's (m, p) in a grid tape
    // slot: entry e's nodes at gtape[64 e + t], the list at gtape_list
    float4 *gtape;
    int *gtape_list;
    int *gtape_count;
};

__global__ void k_batch_set_time(float *t0, float value) { *t0 = value; }

// Grid-wide barrier of a cooperative launch (all CTAs resident) for
// `expected` arriving CTAs (gridDim.x). Returns false when the wait gave up
// (status bit ERRBIT_TIMEOUT set); then every CTA leaves.
__device__ __forceinline__ bool batch_grid_sync(unsigned *bar, int *err, unsigned expected) {
    __shared__ int gave_up;
    __syncthreads();
    if (threadIdx.x == 0) {
        gave_up = 0;
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned it = 0;
            while (*gen == g0) {
                if (++it > BATCH_SPIN_LIMIT) {
                    atomicOr(err, ERRBIT_TIMEOUT);
                    gave_up = 1;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return gave_up == 0;
}

// Phase A: grid update of the blocks in list L at time t0 + k dt (per scene).
// CLEAR: also empty (m, p) and the block flags for the next P2G; without it
// the grid and the list stay for a reverse pass.
template <int THREADS, bool CLEAR = true>
__device__ __forceinline__ void batch_grid_phase(const BatchView &A, int k, int L) {
    constexpr int SUBS = THREADS / 64;
    const int count = A.count[L];
    const int *list = A.list + (size_t)L * A.list_cap;
    const float t0 = *A.t0;
    const int sub = threadIdx.x >> 6, lt = threadIdx.x & 63;
    if (A.gtape && blockIdx.x == 0 && threadIdx.x == 0) *A.gtape_count = count;
    for (int e = blockIdx.x * SUBS + sub; e < count; e += gridDim.x * SUBS) {
        const int ent = list[e];
        const BatchScene &S = A.scenes[ent >> BATCH_SCENE_SHIFT];
        const int b = ent & ((1 << BATCH_SCENE_SHIFT) - 1);
        const MpmParams P = S.P;
        if (A.gtape && lt == 0) A.gtape_list[e] = ent;
        int i, j, kk;
        if (active_node(P, S.nb, b, lt, i, j, kk)) {
            const int64_t node = ((int64_t)kk * P.N + j) * P.N + i;
            if (A.gtape) A.gtape[(size_t)e * 64 + lt] = S.grid_mp[node];
            grid_node_update(P, S.wind, fmaf((float)k, P.dt, t0), node, i, j, kk, S.grid_mp,
                             S.grid_v, CLEAR ? 1 : 0);
        }
        if (CLEAR && lt == 0) S.flags[b] = 0;
    }
}

// Phase B for one work item: G2P of the item's particles; unless FINAL, their
// P2G into the scene's grid with the blocks appended to list Ln.
template <bool FINAL, bool CG>
__device__ __forceinline__ void batch_item(const BatchView &A, const int4 item,
                                           const BatchScene &S, int slot, int Ln,
                                           float4 (*rows)[P2G_ROW], int *keys) {
    const MpmParams &P = S.P;  // read from shared memory where used
    const int64_t n = A.n;
    const int64_t p = (int64_t)item.y + slot;
    P2GParticle q;
    q.valid = false;
    if (slot < item.z) {
        float xp[3], Fp[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) xp[a] = A.x[a * n + p];
#pragma unroll
        for (int c = 0; c < 9; ++c) Fp[c] = A.F[c * n + p];
        const bool pin = A.pinned && A.pinned[p];
        float vn[3], Cn[9];
        g2p_update<CG>(P, S.grid_v, pin, xp, Fp, vn, Cn);
        const bool out = A.ox != nullptr;
        float *xo = out ? A.ox : A.x, *Fo = out ? A.oF : A.F;
#pragma unroll
        for (int a = 0; a < 3; ++a) xo[a * n + p] = xp[a];
#pragma unroll
        for (int c = 0; c < 9; ++c) Fo[c * n + p] = Fp[c];
        if (FINAL || out) {
            float *vo = out ? A.ov : A.v, *Co = out ? A.oC : A.C;
#pragma unroll
            for (int a = 0; a < 3; ++a) vo[a * n + p] = vn[a];
#pragma unroll
            for (int c = 0; c < 9; ++c) Co[c * n + p] = Cn[c];
        }
        const bool fin = isfinite(xp[0]) && isfinite(xp[1]) && isfinite(xp[2]) && finite9(Fp);
        if (!fin) atomicOr(A.err, ERRBIT_NONFINITE);
        if (!FINAL) {
            if (make_stencil(P, xp[0], xp[1], xp[2], q.s)) {
                if (!p2g_affine(P, Fp, Cn, q.A)) atomicOr(A.err, ERRBIT_INVERTED);
#pragma unroll
                for (int a = 0; a < 3; ++a) q.mv[a] = P.p_mass * vn[a];
                q.valid = true;
            } else {
                atomicOr(A.err, ERRBIT_DOMAIN);
            }
        }
    }
    if (!FINAL) {
        const ActiveBlocks ab{S.flags, A.list + (size_t)Ln * A.list_cap, A.count + Ln, S.nb,
                              item.x << BATCH_SCENE_SHIFT};
        p2g_warp_scatter(P, q, S.grid_mp, ab, rows, keys);
    }
}

// Phase B over the work items: each iteration the CTA stages the scene
// records of its THREADS / 128 items in shared memory (so that the scene
// parameters are shared-memory operands instead of registers), then every
// 128-thread group runs one item.
template <int THREADS, bool FINAL, bool CG>
__device__ __forceinline__ void batch_items(const BatchView &A, int Ln,
                                            float4 (*rows)[32][P2G_ROW], int (*keys)[32]) {
    constexpr int PER = THREADS / BATCH_ITEM;
    constexpr int WORDS = sizeof(BatchScene) / 4;
    static_assert(sizeof(BatchScene) % 4 == 0, "scene record is not word-sized");
    __shared__ BatchScene scene[PER];
    __shared__ int4 item[PER];
    const int wid = threadIdx.x >> 5, slot = threadIdx.x % BATCH_ITEM, sub = threadIdx.x / BATCH_ITEM;
    for (int base = blockIdx.x * PER; base < A.n_items; base += gridDim.x * PER) {
        __syncthreads();  // the previous items are done with the staged records
        for (int w = threadIdx.x; w < PER * WORDS; w += THREADS) {
            const int g = w / WORDS, o = w - g * WORDS;
            if (base + g < A.n_items) {
                const int4 it = A.items[base + g];
                if (o == 0) item[g] = it;
                reinterpret_cast<int *>(&scene[g])[o] =
                    reinterpret_cast<const int *>(A.scenes + it.x)[o];
            }
        }
        __syncthreads();
        if (base + sub < A.n_items)
            batch_item<FINAL, CG>(A, item[sub], scene[sub], slot, Ln, rows[wid], keys[wid]);
    }
}

// One substep of every scene in one cooperative launch.
template <int THREADS, bool FINAL>
__global__ void __launch_bounds__(THREADS) k_batch_substep(BatchView A, int k, int L) {
    __shared__ float4 rows[THREADS / 32][32][P2G_ROW];
    __shared__ int keys[THREADS / 32][32];
    // an earlier barrier gave up: do nothing (one read per CTA, shared by all its threads)
    if (__syncthreads_or(threadIdx.x == 0 && (*(volatile int *)A.err & ERRBIT_TIMEOUT))) return;
    batch_grid_phase<THREADS>(A, k, L);
    if (!batch_grid_sync(A.bar, A.err, gridDim.x)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) A.count[L] = 0;  // list L is consumed
    batch_items<THREADS, FINAL, true>(A, 1 - L, rows, keys);
}

// Barrier self-test: `expected` above gridDim.x stands for CTAs that never
// arrive, so every CTA's wait runs out and the status becomes a timeout.
__global__ void k_batch_barrier_probe(unsigned *bar, int *err, unsigned expected) {
    batch_grid_sync(bar, err, expected);
}

// Split mode: the two phases as separate launches.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_batch_grid(BatchView A, int k, int L) {
    pdl_wait();
    pdl_trigger();
    batch_grid_phase<THREADS>(A, k, L);
}

template <int THREADS, bool FINAL>
__global__ void __launch_bounds__(THREADS) k_batch_particles(BatchView A, int L) {
    __shared__ float4 rows[THREADS / 32][32][P2G_ROW];
    __shared__ int keys[THREADS / 32][32];
    pdl_wait();
    pdl_trigger();
    if (blockIdx.x == 0 && threadIdx.x == 0) A.count[L] = 0;
    batch_items<THREADS, FINAL, false>(A, 1 - L, rows, keys);
}

// Pair mode, phase B of a substep that scatters: the paired body of
// mpm_rollout (pair_warp, two particles per thread on FP32 pairs, box-staged
// G2P, row-summed P2G). Warp w of CTA b takes half (b PAIR_WARPS + w) & 1 of
// work item (b PAIR_WARPS + w) >> 1: up to 64 particles of one scene. Each
// warp stages its scene record in shared memory, so that the scene's
// parameters are shared-memory operands, and the material is chosen per warp.
template <bool VEC>
__global__ void __launch_bounds__(PAIR_THREADS, PAIR_MIN_CTAS) k_batch_pair(BatchView A, int L) {
    constexpr int WORDS = sizeof(BatchScene) / 4;
    __shared__ PairWarpSmem smem[PAIR_WARPS];
    __shared__ BatchScene scene[PAIR_WARPS];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hw = blockIdx.x * PAIR_WARPS + wid;
    if ((hw >> 1) >= A.n_items) return;
    const int4 item = A.items[hw >> 1];
    for (int w = lane; w < WORDS; w += 32)
        reinterpret_cast<int *>(&scene[wid])[w] = reinterpret_cast<const int *>(A.scenes + item.x)[w];
    __syncwarp();
    const BatchScene &S = scene[wid];
    const ActiveBlocks ab{S.flags, A.list + (size_t)(1 - L) * A.list_cap, A.count + (1 - L), S.nb,
                          item.x << BATCH_SCENE_SHIFT};
    const int64_t first = item.y;
    pair_warp<-1, false, VEC>(S.P, A.x, A.v, A.C, A.F, A.pinned, S.grid_v, S.grid_mp, A.n,
                              first + (hw & 1) * 64, first + item.z, A.err, ab,
                              blockIdx.x == 0 && threadIdx.x == 0 ? A.count + L : nullptr,
                              smem[wid]);
}

// P2G of every scene from a complete state (start of a segment), list L.
__global__ void __launch_bounds__(BATCH_ITEM) k_batch_p2g(BatchView A, int L) {
    __shared__ float4 rows[BATCH_ITEM / 32][32][P2G_ROW];
    __shared__ int keys[BATCH_ITEM / 32][32];
    const int wid = threadIdx.x >> 5;
    const int4 item = A.items[blockIdx.x];
    const BatchScene &S = A.scenes[item.x];
    const MpmParams P = S.P;
    P2GParticle q;
    q.valid = false;
    if ((int)threadIdx.x < item.z)
        p2g_load(P, A.x, A.v, A.C, A.F, A.n, (int64_t)item.y + threadIdx.x, q, A.err);
    const ActiveBlocks ab{S.flags, A.list + (size_t)L * A.list_cap, A.count + L, S.nb,
                          item.x << BATCH_SCENE_SHIFT};
    p2g_warp_scatter<true>(P, q, S.grid_mp, ab, rows[wid], keys[wid]);
}

// Sort keys of every scene, offset per scene, counted into counts.
// One count atomic per distinct key of a warp.
__global__ void __launch_bounds__(BATCH_ITEM) k_batch_sort_keys(BatchView A, int *__restrict__ keys,
                                                                int *__restrict__ counts) {
    const int4 item = A.items[blockIdx.x];
    const bool ok = (int)threadIdx.x < item.z;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!ok) return;
    const BatchScene &S = A.scenes[item.x];
    const int64_t p = (int64_t)item.y + threadIdx.x, n = A.n;
    const int key = S.key_offset + cell_key(S.P, S.nb, A.x[p], A.x[n + p], A.x[2 * n + p]);
    keys[p] = key;
    const unsigned peers = __match_any_sync(act, key);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&counts[key], __popc(peers));
}

// ---------------------------------------------------------------- reverse --

// Adjoint buffers of a reverse substep over the batch.
struct BatchAdjView {
    const int64_t *node_off;  // [n_scenes] first node of each scene in the batch grids
    const int64_t *wind_off;  // [n_scenes] first float of each scene's wind gradient
    float4 *grid_bv;          // (0, dL/dv_i), zero between calls
    float4 *grid_bmp;         // (dL/dm_i, dL/dp_i)
    float *scratch;           // [12][n]: partial dL/dx_p, dL/dF_p of the reverse G2P
    float *gx, *gv, *gC, *gF; // dL/d(output state) in, dL/d(input state) out
    float *g_wind;            // concatenated per-scene wind gradients, or NULL
    float *g_E;               // [n_scenes], or NULL
    const float *Cout;        // C of the reverse substep's output state (kept in the tape), or NULL
};

// Grid update of list L at substep k keeping (m, p) and the list (the
// recomputed forward grid of a reverse substep).
__global__ void __launch_bounds__(256) k_batch_grid_keep(BatchView A, int k, int L) {
    batch_grid_phase<256, false>(A, k, L);
}

// The recomputed forward grid of reverse substep k from the grid tape: list
// 0 and its count, each listed node's (m, p) written back into the scene's
// grid and its grid update (grid kept), in place of a P2G of the substep's
// input and k_batch_grid_keep.
__global__ void __launch_bounds__(256) k_batch_grid_restore(BatchView A, int k,
                                                            const float4 *__restrict__ gtape,
                                                            const int *__restrict__ gtape_list,
                                                            const int *__restrict__ gtape_count) {
    constexpr int SUBS = 256 / 64;
    const int count = *gtape_count;
    if (blockIdx.x == 0 && threadIdx.x == 0) A.count[0] = count;
    const float t0 = *A.t0;
    const int sub = threadIdx.x >> 6, lt = threadIdx.x & 63;
    for (int e = blockIdx.x * SUBS + sub; e < count; e += gridDim.x * SUBS) {
        const int ent = gtape_list[e];
        if (lt == 0) A.list[e] = ent;
        const BatchScene &S = A.scenes[ent >> BATCH_SCENE_SHIFT];
        const int b = ent & ((1 << BATCH_SCENE_SHIFT) - 1);
        const MpmParams P = S.P;
        int i, j, kk;
        if (active_node(P, S.nb, b, lt, i, j, kk)) {
            const int64_t node = ((int64_t)kk * P.N + j) * P.N + i;
            S.grid_mp[node] = gtape[(size_t)e * 64 + lt];
            grid_node_update(P, S.wind, fmaf((float)k, P.dt, t0), node, i, j, kk, S.grid_mp,
                             S.grid_v, 0);
        }
    }
}

// Reverse G2P of one work item per CTA: scatter into the scene's grid_bv.
__global__ void __launch_bounds__(BATCH_ITEM) k_batch_rev_g2p(BatchView A, BatchAdjView R) {
    __shared__ float4 rows[BATCH_ITEM / 32][32][P2G_ROW];
    __shared__ int keys[BATCH_ITEM / 32][32];
    const int wid = threadIdx.x >> 5;
    const int4 item = A.items[blockIdx.x];
    const BatchScene &S = A.scenes[item.x];
    const MpmParams P = S.P;
    const int64_t n = A.n, p = (int64_t)item.y + threadIdx.x;
    P2GParticle q;
    q.valid = false;
    if ((int)threadIdx.x < item.z) {
        float xp[3], Fp[9], bxo[3], bvo[3], bCo[9], bFo[9], bx[3], bFin[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xp[a] = A.x[a * n + p];
            bxo[a] = R.gx[a * n + p];
            bvo[a] = R.gv[a * n + p];
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            Fp[c] = A.F[c * n + p];
            bCo[c] = R.gC[c * n + p];
            bFo[c] = R.gF[c * n + p];
        }
        rev_g2p_particle(P, xp, Fp, A.pinned && A.pinned[p], S.grid_v, bxo, bvo, bCo, bFo, q, bx,
                         bFin, R.Cout, n, p);
#pragma unroll
        for (int a = 0; a < 3; ++a) R.scratch[a * n + p] = bx[a];
#pragma unroll
        for (int c = 0; c < 9; ++c) R.scratch[(3 + c) * n + p] = bFin[c];
    }
    MpmParams Pz = P;
    Pz.p_mass = 0.0f;  // no mass channel: grid_bv = (0, dL/dv_i)
    const ActiveBlocks none{nullptr, nullptr, nullptr, 0, 0};
    p2g_warp_scatter<true>(Pz, q, R.grid_bv + R.node_off[item.x], none, rows[wid], keys[wid]);
}

// Reverse grid update of the blocks in list L at substep k; clears the
// scene's (m, p), grid_bv and block flags.
__global__ void __launch_bounds__(256) k_batch_rev_grid(BatchView A, BatchAdjView R, int k, int L) {
    constexpr int SUBS = 256 / 64;
    __shared__ float sbox[256 / 32][WIND_BOX];
    const int count = A.count[L];
    const int *list = A.list + (size_t)L * A.list_cap;
    const float t0 = *A.t0;
    const int sub = threadIdx.x >> 6, lt = threadIdx.x & 63;
    // every lane of a 64-thread group runs the same iterations (one block of
    // one scene each), so the wind scatter below is warp-uniform
    for (int e = blockIdx.x * SUBS + sub; e < count; e += gridDim.x * SUBS) {
        const int ent = list[e];
        const int sc = ent >> BATCH_SCENE_SHIFT;
        const BatchScene &S = A.scenes[sc];
        const int b = ent & ((1 << BATCH_SCENE_SHIFT) - 1);
        const MpmParams P = S.P;
        int i = 0, j = 0, kk = 0;
        bool live = false;
        float3 gw;
        if (active_node(P, S.nb, b, lt, i, j, kk)) {
            const int64_t node = ((int64_t)kk * P.N + j) * P.N + i;
            const int64_t no = R.node_off[sc];
            live = rev_grid_node(P, node, i, j, kk, S.grid_mp, R.grid_bv + no, R.grid_bmp + no, gw);
        }
        if (R.g_wind)
            wind_sample_adjoint_warp(S.wind, wind_scatter_coarse(P.N, S.wind.nf), live, i * P.dx,
                                     j * P.dx, kk * P.dx, fmaf((float)k, P.dt, t0), gw,
                                     R.g_wind + R.wind_off[sc], sbox[threadIdx.x >> 5]);
        if (lt == 0) S.flags[b] = 0;
    }
}

// Reverse P2G of one work item per CTA; one dL/dE atomic per item.
__global__ void __launch_bounds__(BATCH_ITEM) k_batch_rev_p2g(BatchView A, BatchAdjView R, int L) {
    if (blockIdx.x == 0 && threadIdx.x == 0) A.count[L] = 0;  // the reverse grid consumed list L
    const int4 item = A.items[blockIdx.x];
    const BatchScene &S = A.scenes[item.x];
    const MpmParams P = S.P;
    const int64_t n = A.n, p = (int64_t)item.y + threadIdx.x;
    float gE = 0.0f;
    if ((int)threadIdx.x < item.z) {
        float xp[3], vp[3], Cp[9], Fp[9], bx[3], bF[9], bvp[3], bC[9];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xp[a] = A.x[a * n + p];
            vp[a] = A.v[a * n + p];
            bx[a] = R.scratch[a * n + p];
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            Cp[c] = A.C[c * n + p];
            Fp[c] = A.F[c * n + p];
            bF[c] = R.scratch[(3 + c) * n + p];
        }
        rev_p2g_particle(P, xp, vp, Cp, Fp, R.grid_bmp + R.node_off[item.x], bx, bF, bvp, bC, gE);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            R.gx[a * n + p] = bx[a];
            R.gv[a * n + p] = bvp[a];
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            R.gC[c * n + p] = bC[c];
            R.gF[c * n + p] = bF[c];
        }
    }
    if (R.g_E) {
        const float sum = block_sum(gE);
        if (threadIdx.x == 0) atomicAdd(R.g_E + item.x, sum);
    }
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_coop(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                               cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

struct GraphKey {
    const void *ptr[6];
    int n_substeps, sort_every, mode, threads, ctas_per_sm;
    bool operator==(const GraphKey &o) const {
        for (int i = 0; i < 6; ++i)
            if (ptr[i] != o.ptr[i]) return false;
        return n_substeps == o.n_substeps && sort_every == o.sort_every && mode == o.mode &&
               threads == o.threads && ctas_per_sm == o.ctas_per_sm;
    }
};

// Pointers and shape a captured segment adjoint was recorded with.
struct AdjKey {
    const void *ptr[12];
    int n_substeps, mode, threads, ctas_per_sm;
    bool operator==(const AdjKey &o) const {
        for (int i = 0; i < 12; ++i)
            if (ptr[i] != o.ptr[i]) return false;
        return n_substeps == o.n_substeps && mode == o.mode && threads == o.threads &&
               ctas_per_sm == o.ctas_per_sm;
    }
};

}  // namespace dw

struct dw_mpm_batch_s {
    int n_scenes = 0;
    std::vector<int64_t> offsets;  // [n_scenes + 1]
    int64_t n_total = 0;
    int64_t total_keys = 0;
    int list_cap = 0;
    int n_items = 0;
    bool items_aligned4 = false;  // n and every scene offset a multiple of 4
    int num_sms = 0;
    int occupancy[2][2] = {{0, 0}, {0, 0}};  // [threads == 256][final]: CTAs per SM
    dw::BatchScene *scenes = nullptr;  // device table
    int4 *items = nullptr;
    float4 *grid_mp = nullptr, *grid_v = nullptr;
    int *flags = nullptr, *list = nullptr, *count = nullptr, *err = nullptr;
    unsigned *bar = nullptr;
    float *t0 = nullptr;
    int *keys = nullptr, *key_counts = nullptr, *scan_tmp = nullptr;
    int64_t scan_tmp_len = 0;
    float *roll_state = nullptr;
    uint8_t *roll_pinned = nullptr;
    int32_t *roll_ids = nullptr;
    // reverse mode (allocated by the first mpm_batch_segment_adjoint)
    std::vector<int64_t> wind_off;  // [n_scenes + 1] floats of the scenes' wind values
    std::vector<int64_t> node_off;  // [n_scenes + 1]
    int64_t *d_node_off = nullptr, *d_wind_off = nullptr;
    float4 *grid_bv = nullptr, *grid_bmp = nullptr;
    float *adj_scratch = nullptr;
    // grid tape of the segment recompute: gtape_slots substeps of list_cap
    // entries (64 nodes' (m, p) each), their lists and counts
    float4 *gtape = nullptr;
    int *gtape_list = nullptr, *gtape_count = nullptr;
    int gtape_slots = 0;
    int gtape_refused = 0;  // slots a failed or oversized allocation was refused for
    cudaGraphExec_t adj_exec = nullptr;  // captured segment adjoint
    dw::AdjKey adj_key = {};
    bool adj_graph_broken = false;
    dw_batch_config cfg = {};
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    dw::GraphKey key = {};
    bool graph_broken = false;  // capture failed once: launch directly from then on
};

namespace dw {

static dw_mpm_state state_view(float *base, int64_t n) {
    dw_mpm_state s;
    s.x = base;
    s.v = base + 3 * n;
    s.C = base + 6 * n;
    s.F = base + 15 * n;
    s.n = n;
    return s;
}

static BatchView view_of(dw_mpm_batch h, const dw_mpm_state &s, const uint8_t *pinned) {
    BatchView A;
    A.scenes = h->scenes;
    A.items = h->items;
    A.n_items = h->n_items;
    A.x = s.x;
    A.v = s.v;
    A.C = s.C;
    A.F = s.F;
    A.ox = A.ov = A.oC = A.oF = nullptr;
    A.pinned = pinned;
    A.n = h->n_total;
    A.list = h->list;
    A.count = h->count;
    A.list_cap = h->list_cap;
    A.err = h->err;
    A.bar = h->bar;
    A.t0 = h->t0;
    A.gtape = nullptr;
    A.gtape_list = nullptr;
    A.gtape_count = nullptr;
    return A;
}

// with_vc = false leaves v and C of `out` unwritten (a rollout between fused
// launches, where v and C are not kept).
static dw_status batch_sort(dw_mpm_batch h, const dw_mpm_state &in, const dw_mpm_state &out,
                            const uint8_t *pin_in, uint8_t *pin_out, const int32_t *ids_in,
                            int32_t *ids_out, cudaStream_t s, bool with_vc = true) {
    const int64_t n = h->n_total;
    DW_CUDA(cudaMemsetAsync(h->key_counts, 0, sizeof(int) * (size_t)(h->total_keys + 1), s));
    k_batch_sort_keys<<<h->n_items, BATCH_ITEM, 0, s>>>(view_of(h, in, pin_in), h->keys,
                                                        h->key_counts);
    DW_LAUNCHED("k_batch_sort_keys");
    dw_status st = exclusive_scan(h->key_counts, h->total_keys, h->scan_tmp, h->scan_tmp_len, s);
    if (st != DW_OK) return st;
    k_sort_move<<<grid_for(n, 256), 256, 0, s>>>(h->keys, n, h->key_counts, in.x,
                                                 with_vc ? in.v : nullptr, with_vc ? in.C : nullptr,
                                                 in.F, pin_in, ids_in, out.x, out.v, out.C, out.F,
                                                 pin_out, ids_out);
    DW_LAUNCHED("k_sort_move");
    return DW_OK;
}

static int occupancy_of(dw_mpm_batch h, int threads, bool final_) {
    return h->occupancy[threads == 256 ? 1 : 0][final_ ? 1 : 0];
}

// One substep launch (or two in split and pair mode). vec: the pair kernel
// may load x and F as float2 and 16-byte pieces.
static dw_status launch_substep(dw_mpm_batch h, const BatchView &A, const dw_batch_config &c,
                                int k, int L, bool final_, cudaStream_t s, bool vec = false) {
    const int T = c.threads;
    if (c.mode == DW_BATCH_PAIR && !final_ && !A.ox) {
        const unsigned ggrid = (unsigned)(c.ctas_per_sm * h->num_sms);
        // PAIR_WARPS halves of 128-particle work items per CTA
        const unsigned pgrid = (unsigned)((2 * h->n_items + PAIR_WARPS - 1) / PAIR_WARPS);
        if (T == 256)
            DW_CUDA(launch_pdl(k_batch_grid<256>, ggrid, 256, s, A, k, L));
        else
            DW_CUDA(launch_pdl(k_batch_grid<128>, ggrid, 128, s, A, k, L));
        DW_CUDA(vec ? launch_pdl(k_batch_pair<true>, pgrid, PAIR_THREADS, s, A, L)
                    : launch_pdl(k_batch_pair<false>, pgrid, PAIR_THREADS, s, A, L));
        return DW_OK;
    }
    if (c.mode == DW_BATCH_PERSISTENT) {
        const int per_sm = std::min(c.ctas_per_sm, occupancy_of(h, T, final_));
        const unsigned grid = (unsigned)(per_sm * h->num_sms);
        if (T == 256)
            DW_CUDA(final_ ? launch_coop(k_batch_substep<256, true>, grid, 256, s, A, k, L)
                           : launch_coop(k_batch_substep<256, false>, grid, 256, s, A, k, L));
        else
            DW_CUDA(final_ ? launch_coop(k_batch_substep<128, true>, grid, 128, s, A, k, L)
                           : launch_coop(k_batch_substep<128, false>, grid, 128, s, A, k, L));
        return DW_OK;
    }
    const unsigned ggrid = (unsigned)(c.ctas_per_sm * h->num_sms);
    const int per = T / BATCH_ITEM;
    const unsigned pgrid = (unsigned)((h->n_items + per - 1) / per);
    if (T == 256) {
        DW_CUDA(launch_pdl(k_batch_grid<256>, ggrid, 256, s, A, k, L));
        DW_CUDA(final_ ? launch_pdl(k_batch_particles<256, true>, pgrid, 256, s, A, L)
                       : launch_pdl(k_batch_particles<256, false>, pgrid, 256, s, A, L));
    } else {
        DW_CUDA(launch_pdl(k_batch_grid<128>, ggrid, 128, s, A, k, L));
        DW_CUDA(final_ ? launch_pdl(k_batch_particles<128, true>, pgrid, 128, s, A, L)
                       : launch_pdl(k_batch_particles<128, false>, pgrid, 128, s, A, L));
    }
    return DW_OK;
}

// The launch sequence of a rollout (the time t0 is already on the device).
// Substep k of the sequence runs at t0 + (k_base + k) dt.
static dw_status enqueue_rollout(dw_mpm_batch h, const dw_mpm_state *state, uint8_t *pinned,
                                 int32_t *ids, int n_substeps, int sort_every,
                                 const dw_batch_config &c, cudaStream_t s, int k_base = 0) {
    const int64_t n = h->n_total;
    DW_CUDA(cudaMemsetAsync(h->bar, 0, 2 * sizeof(unsigned), s));
    dw_mpm_state cur = *state, oth = state_view(h->roll_state, n);
    uint8_t *cur_pin = pinned, *oth_pin = pinned ? h->roll_pinned : nullptr;
    int32_t *cur_ids = ids, *oth_ids = h->roll_ids;
    auto resort = [&](bool with_vc) {
        dw_status r = batch_sort(h, cur, oth, cur_pin, oth_pin, cur_ids, oth_ids, s, with_vc);
        std::swap(cur, oth);
        std::swap(cur_pin, oth_pin);
        std::swap(cur_ids, oth_ids);
        return r;
    };
    // pair kernel vector loads: every work item starts at a multiple of 4
    // particles and the arrays are 16-byte aligned
    auto vec_of = [&](const dw_mpm_state &q) {
        return h->items_aligned4 &&
               ((reinterpret_cast<uintptr_t>(q.x) | reinterpret_cast<uintptr_t>(q.F)) % 16 == 0);
    };
    if (sort_every > 0) {
        dw_status st = resort(true);  // the input state's v and C feed the first P2G
        if (st != DW_OK) return st;
    }
    BatchView A = view_of(h, cur, cur_pin);
    bool vec = vec_of(cur);
    int L = 0;
    k_batch_p2g<<<h->n_items, BATCH_ITEM, 0, s>>>(A, L);
    DW_LAUNCHED("k_batch_p2g");
    for (int k = 0; k < n_substeps; ++k) {
        const bool final_ = k + 1 == n_substeps;
        dw_status st = launch_substep(h, A, c, k_base + k, L, final_, s, vec);
        if (st != DW_OK) return st;
        if (final_) break;
        L = 1 - L;
        // re-sort between two fused launches (the P2G of substep k + 1 has
        // run in the old order; v and C are not kept between them)
        if (sort_every > 0 && (k + 1) % sort_every == 0) {
            st = resort(false);
            if (st != DW_OK) return st;
            A = view_of(h, cur, cur_pin);
            vec = vec_of(cur);
        }
    }
    if (cur.x != state->x) {  // an odd number of sorts: the result is in the workspace
        const size_t b3 = sizeof(float) * 3 * (size_t)n, b9 = sizeof(float) * 9 * (size_t)n;
        DW_CUDA(cudaMemcpyAsync(state->x, cur.x, b3, cudaMemcpyDeviceToDevice, s));
        DW_CUDA(cudaMemcpyAsync(state->v, cur.v, b3, cudaMemcpyDeviceToDevice, s));
        DW_CUDA(cudaMemcpyAsync(state->C, cur.C, b9, cudaMemcpyDeviceToDevice, s));
        DW_CUDA(cudaMemcpyAsync(state->F, cur.F, b9, cudaMemcpyDeviceToDevice, s));
        if (pinned)
            DW_CUDA(cudaMemcpyAsync(pinned, cur_pin, (size_t)n, cudaMemcpyDeviceToDevice, s));
        DW_CUDA(cudaMemcpyAsync(ids, cur_ids, sizeof(int32_t) * (size_t)n,
                                cudaMemcpyDeviceToDevice, s));
    }
    return DW_OK;
}

static void drop_graph(dw_mpm_batch h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    h->exec = nullptr;
}

// Captures the launch sequence into h->exec; false (and no error left behind)
// when this rollout cannot be captured.
static bool capture_rollout(dw_mpm_batch h, const dw_mpm_state *state, uint8_t *pinned,
                            int32_t *ids, int n_substeps, int sort_every) {
    drop_graph(h);
    if (!h->cap_stream &&
        cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    dw_status st = enqueue_rollout(h, state, pinned, ids, n_substeps, sort_every, h->cfg,
                                   h->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    bool ok = st == DW_OK && e == cudaSuccess && graph;
    if (ok) ok = cudaGraphInstantiate(&h->exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (!ok) h->exec = nullptr;
    return ok;
}

static dw_status check_batch_state(dw_mpm_batch h, const dw_mpm_state *s) {
    DW_REQUIRE(s, "state is NULL");
    DW_REQUIRE(s->n == h->n_total, "state has n=%lld particles; the batch has %lld",
               (long long)s->n, (long long)h->n_total);
    DW_REQUIRE(s->x && s->v && s->C && s->F, "state arrays must not be NULL");
    return DW_OK;
}

static dw_status check_config(dw_mpm_batch h, const dw_batch_config *c) {
    DW_REQUIRE(c, "config is NULL");
    DW_REQUIRE(c->mode == DW_BATCH_PERSISTENT || c->mode == DW_BATCH_SPLIT ||
                   c->mode == DW_BATCH_PAIR,
               "unknown mode %d", c->mode);
    DW_REQUIRE(c->threads == 128 || c->threads == 256, "threads must be 128 or 256");
    DW_REQUIRE(c->ctas_per_sm >= 1 && c->ctas_per_sm <= 64, "ctas_per_sm out of range [1, 64]");
    if (c->mode == DW_BATCH_PERSISTENT)
        DW_REQUIRE(occupancy_of(h, c->threads, false) >= 1 && occupancy_of(h, c->threads, true) >= 1,
                   "the persistent kernel with %d threads cannot be resident", c->threads);
    return DW_OK;
}

}  // namespace dw

using namespace dw;

extern "C" dw_status mpm_batch_create(const dw_mpm_scene *scenes, int32_t n_scenes,
                                      dw_mpm_batch *out) {
    DW_REQUIRE(out, "out must not be NULL");
    *out = nullptr;
    DW_REQUIRE(scenes, "scenes must not be NULL");
    DW_REQUIRE(n_scenes >= 1 && n_scenes <= BATCH_MAX_SCENES, "n_scenes=%d out of range [1, %d]",
               n_scenes, BATCH_MAX_SCENES);
    std::vector<BatchScene> tab(n_scenes);
    std::vector<int64_t> offsets(n_scenes + 1, 0);
    std::vector<int64_t> node_off(n_scenes + 1, 0), blk_off(n_scenes + 1, 0);
    std::vector<int64_t> wind_off(n_scenes + 1, 0);
    int64_t total_keys = 0;
    for (int s = 0; s < n_scenes; ++s) {
        const dw_mpm_scene &sc = scenes[s];
        dw_mpm_desc d = sc.desc;
        d.max_particles = 0;
        d.p2g_mode = DW_P2G_AUTO;
        dw_status st = validate_desc(&d);
        if (st != DW_OK) return st;
        DW_REQUIRE(d.n_grid <= 400, "scene %d: n_grid=%d above the batch limit 400", s, d.n_grid);
        DW_REQUIRE(sc.n_particles >= 1, "scene %d has no particles", s);
        st = wind_check(&sc.wind, &tab[s].wind);
        if (st != DW_OK) return st;
        tab[s].P = params_of(d);
        const int nb = (d.n_grid + 3) / 4;
        tab[s].nb = nb;
        tab[s].key_offset = (int)total_keys;
        total_keys += (int64_t)nb * nb * nb * 64;
        offsets[s + 1] = offsets[s] + sc.n_particles;
        node_off[s + 1] = node_off[s] + (int64_t)d.n_grid * d.n_grid * d.n_grid;
        blk_off[s + 1] = blk_off[s] + (int64_t)nb * nb * nb;
        wind_off[s + 1] = wind_off[s] + (int64_t)sc.wind.n_frames * sc.wind.nf * sc.wind.nf *
                                            sc.wind.nf * 3;
        DW_REQUIRE(total_keys < (1ll << 31), "the scenes' grids are too large for one batch");
        DW_REQUIRE(offsets[s + 1] < (1ll << 31), "more than 2^31 - 1 particles in the batch");
    }
    std::vector<int4> items;
    for (int s = 0; s < n_scenes; ++s)
        for (int64_t b = offsets[s]; b < offsets[s + 1]; b += BATCH_ITEM)
            items.push_back(make_int4(s, (int)b, (int)std::min<int64_t>(BATCH_ITEM, offsets[s + 1] - b), 0));
    DW_REQUIRE(items.size() < (1u << 31), "too many work items");

    dw_mpm_batch h = new (std::nothrow) dw_mpm_batch_s();
    if (!h) {
        set_error("out of host memory");
        return DW_ERR_OOM;
    }
    h->n_scenes = n_scenes;
    h->offsets = offsets;
    h->node_off = node_off;
    h->wind_off = wind_off;
    h->n_total = offsets[n_scenes];
    h->total_keys = total_keys;
    h->list_cap = (int)blk_off[n_scenes];
    h->n_items = (int)items.size();
    h->items_aligned4 = true;
    for (int s = 0; s <= n_scenes; ++s) h->items_aligned4 = h->items_aligned4 && offsets[s] % 4 == 0;
    h->scan_tmp_len = (total_keys + SCAN_BLOCK) / SCAN_BLOCK + 1;
    const int64_t n = h->n_total;
    cudaError_t e = cudaSuccess;
#define DW_ALLOC(ptr, bytes) \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes))
    DW_ALLOC(h->scenes, sizeof(BatchScene) * (size_t)n_scenes);
    DW_ALLOC(h->items, sizeof(int4) * items.size());
    DW_ALLOC(h->grid_mp, sizeof(float4) * (size_t)node_off[n_scenes]);
    DW_ALLOC(h->grid_v, sizeof(float4) * (size_t)node_off[n_scenes]);
    DW_ALLOC(h->flags, sizeof(int) * (size_t)blk_off[n_scenes]);
    DW_ALLOC(h->list, sizeof(int) * 2 * (size_t)blk_off[n_scenes]);
    DW_ALLOC(h->count, sizeof(int) * 2);
    DW_ALLOC(h->err, sizeof(int));
    DW_ALLOC(h->bar, sizeof(unsigned) * 2);
    DW_ALLOC(h->t0, sizeof(float));
    DW_ALLOC(h->keys, sizeof(int) * (size_t)n);
    DW_ALLOC(h->key_counts, sizeof(int) * (size_t)(total_keys + 1));
    DW_ALLOC(h->scan_tmp, sizeof(int) * (size_t)h->scan_tmp_len);
    DW_ALLOC(h->roll_state, sizeof(float) * 24 * (size_t)n);
    DW_ALLOC(h->roll_pinned, (size_t)n);
    DW_ALLOC(h->roll_ids, sizeof(int32_t) * (size_t)n);
#undef DW_ALLOC
    if (e == cudaSuccess) {
        for (int s = 0; s < n_scenes; ++s) {
            tab[s].grid_mp = h->grid_mp + node_off[s];
            tab[s].grid_v = h->grid_v + node_off[s];
            tab[s].flags = h->flags + blk_off[s];
        }
        e = cudaMemcpy(h->scenes, tab.data(), sizeof(BatchScene) * tab.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(h->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->grid_mp, 0, sizeof(float4) * (size_t)node_off[n_scenes]);
    if (e == cudaSuccess) e = cudaMemset(h->flags, 0, sizeof(int) * (size_t)blk_off[n_scenes]);
    if (e == cudaSuccess) e = cudaMemset(h->count, 0, sizeof(int) * 2);
    if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->bar, 0, sizeof(unsigned) * 2);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occupancy[0][0], k_batch_substep<128, false>, 128, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occupancy[0][1], k_batch_substep<128, true>, 128, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occupancy[1][0], k_batch_substep<256, false>, 256, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occupancy[1][1], k_batch_substep<256, true>, 256, 0);
    if (e != cudaSuccess) {
        mpm_batch_destroy(h);
        return e == cudaErrorMemoryAllocation ? (set_error("out of device memory"), DW_ERR_OOM)
                                              : cuda_fail(e, "mpm_batch_create");
    }
    h->cfg.mode = DW_BATCH_PAIR;
    h->cfg.threads = 128;
    h->cfg.ctas_per_sm = 4;
    h->cfg.use_graph = 1;
    h->cfg.graph_active = 0;
    *out = h;
    return DW_OK;
}

extern "C" dw_status mpm_batch_destroy(dw_mpm_batch h) {
    if (!h) return DW_OK;
    drop_graph(h);
    if (h->adj_exec) cudaGraphExecDestroy(h->adj_exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->scenes);
    cudaFree(h->items);
    cudaFree(h->grid_mp);
    cudaFree(h->grid_v);
    cudaFree(h->flags);
    cudaFree(h->list);
    cudaFree(h->count);
    cudaFree(h->err);
    cudaFree(h->bar);
    cudaFree(h->t0);
    cudaFree(h->keys);
    cudaFree(h->key_counts);
    cudaFree(h->scan_tmp);
    cudaFree(h->roll_state);
    cudaFree(h->roll_pinned);
    cudaFree(h->roll_ids);
    cudaFree(h->d_node_off);
    cudaFree(h->d_wind_off);
    cudaFree(h->grid_bv);
    cudaFree(h->grid_bmp);
    cudaFree(h->gtape);
    cudaFree(h->gtape_list);
    cudaFree(h->gtape_count);
    cudaFree(h->adj_scratch);
    delete h;
    return DW_OK;
}

extern "C" dw_status mpm_batch_layout(dw_mpm_batch h, int64_t *n_total, int64_t *offsets) {
    DW_REQUIRE(h, "handle is NULL");
    if (n_total) *n_total = h->n_total;
    if (offsets)
        for (int s = 0; s <= h->n_scenes; ++s) offsets[s] = h->offsets[s];
    return DW_OK;
}

extern "C" dw_status mpm_batch_set_config(dw_mpm_batch h, const dw_batch_config *config) {
    DW_REQUIRE(h, "handle is NULL");
    dw_status st = check_config(h, config);
    if (st != DW_OK) return st;
    h->cfg = *config;
    h->cfg.graph_active = 0;
    return DW_OK;
}

extern "C" dw_status mpm_batch_get_config(dw_mpm_batch h, dw_batch_config *config) {
    DW_REQUIRE(h && config, "handle and config must not be NULL");
    *config = h->cfg;
    return DW_OK;
}

extern "C" dw_status mpm_batch_rollout(dw_mpm_batch h, const dw_mpm_state *state, uint8_t *pinned,
                                       int32_t *ids, float t0, int32_t n_substeps,
                                       int32_t sort_every, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    dw_status st = check_batch_state(h, state);
    if (st != DW_OK) return st;
    DW_REQUIRE(n_substeps >= 0, "n_substeps must be >= 0");
    DW_REQUIRE(sort_every >= 0, "sort_every must be >= 0");
    DW_REQUIRE(sort_every == 0 || ids, "ids must be given when sort_every > 0");
    if (n_substeps == 0) return DW_OK;
    cudaStream_t s = as_stream(stream);
    k_batch_set_time<<<1, 1, 0, s>>>(h->t0, t0);
    DW_LAUNCHED("k_batch_set_time");
    if (h->cfg.use_graph && !h->graph_broken) {
        GraphKey key = {{state->x, state->v, state->C, state->F, pinned, ids}, n_substeps,
                        sort_every, h->cfg.mode, h->cfg.threads, h->cfg.ctas_per_sm};
        if (!h->exec || !(key == h->key)) {
            if (capture_rollout(h, state, pinned, ids, n_substeps, sort_every))
                h->key = key;
            else
                h->graph_broken = true;
        }
        if (h->exec) {
            DW_CUDA(cudaGraphLaunch(h->exec, s));
            h->cfg.graph_active = 1;
            return DW_OK;
        }
    }
    h->cfg.graph_active = 0;
    return enqueue_rollout(h, state, pinned, ids, n_substeps, sort_every, h->cfg, s);
}

extern "C" dw_status mpm_batch_device_status(dw_mpm_batch h, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    int bits = 0;
    cudaStream_t s = as_stream(stream);
    DW_CUDA(cudaMemcpyAsync(&bits, h->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DW_CUDA(cudaStreamSynchronize(s));
    DW_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int), s));
    DW_CUDA(cudaMemsetAsync(h->bar, 0, 2 * sizeof(unsigned), s));
    DW_CUDA(cudaStreamSynchronize(s));
    return status_from_bits(bits);
}

extern "C" dw_status mpm_batch_barrier_selftest(dw_mpm_batch h, int32_t missing_ctas,
                                                dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(missing_ctas >= 0 && missing_ctas <= 1024, "missing_ctas out of range [0, 1024]");
    cudaStream_t s = as_stream(stream);
    DW_CUDA(cudaMemsetAsync(h->bar, 0, 2 * sizeof(unsigned), s));
    const unsigned grid = (unsigned)h->num_sms;
    DW_CUDA(launch_coop(k_batch_barrier_probe, grid, 128, s, h->bar, h->err,
                        grid + (unsigned)missing_ctas));
    return mpm_batch_device_status(h, stream);
}

extern "C" dw_status mpm_batch_tune(dw_mpm_batch h, const dw_mpm_state *state,
                                    const uint8_t *pinned, int32_t n_trial_substeps,
                                    dw_batch_config *best, dw_batch_trial *trials,
                                    int32_t max_trials, int32_t *n_trials, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    dw_status st = check_batch_state(h, state);
    if (st != DW_OK) return st;
    DW_REQUIRE(n_trial_substeps >= 1, "n_trial_substeps must be >= 1");
    DW_REQUIRE(max_trials >= 0, "max_trials must be >= 0");
    cudaStream_t s = as_stream(stream);
    const int64_t n = h->n_total;
    // candidates
    std::vector<dw_batch_config> cand;
    for (int T : {128, 256}) {
        const int occ = std::min(occupancy_of(h, T, false), occupancy_of(h, T, true));
        for (int c = 1; c <= occ; ++c)
            cand.push_back(dw_batch_config{DW_BATCH_PERSISTENT, T, c, 0, 0});
        for (int c : {2, 4}) {
            cand.push_back(dw_batch_config{DW_BATCH_SPLIT, T, c, 0, 0});
            cand.push_back(dw_batch_config{DW_BATCH_PAIR, T, c, 0, 0});
        }
    }
    // the trials run on a copy of the state sorted by cell into the workspace
    const dw_mpm_state work = state_view(h->roll_state, n);
    uint8_t *work_pin = pinned ? h->roll_pinned : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DW_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    dw_status result = DW_OK;
    float best_ms = 0.0f;
    int best_i = -1, recorded = 0;
    k_batch_set_time<<<1, 1, 0, s>>>(h->t0, 0.0f);
    DW_LAUNCHED("k_batch_set_time");
    for (size_t i = 0; i < cand.size() && result == DW_OK; ++i) {
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && result == DW_OK; ++rep) {
            result = batch_sort(h, *state, work, pinned, work_pin, nullptr, h->roll_ids, s);
            if (result != DW_OK) break;
            cudaError_t e = cudaEventRecord(e0, s);
            if (e != cudaSuccess) {
                result = cuda_fail(e, "mpm_batch_tune");
                break;
            }
            result = enqueue_rollout(h, &work, work_pin, nullptr, n_trial_substeps, 0, cand[i], s);
            if (result != DW_OK) break;
            e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) {
                result = cuda_fail(e, "mpm_batch_tune");
                break;
            }
            ms = rep == 0 ? t : std::min(ms, t);
        }
        if (result != DW_OK) break;
        int bits = 0;
        if (cudaMemcpy(&bits, h->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            result = cuda_fail(cudaGetLastError(), "mpm_batch_tune");
            break;
        }
        if (bits) {  // a trial failed on the device: report it, keep the old configuration
            result = mpm_batch_device_status(h, stream);
            break;
        }
        const float per = ms / (float)n_trial_substeps;
        if (trials && recorded < max_trials) trials[recorded++] = dw_batch_trial{cand[i], per};
        if (best_i < 0 || per < best_ms) {
            best_i = (int)i;
            best_ms = per;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_trials) *n_trials = recorded;
    if (result != DW_OK) return result;
    const int use_graph = h->cfg.use_graph;
    h->cfg = cand[best_i];
    h->cfg.use_graph = use_graph;
    h->cfg.graph_active = 0;
    if (best) *best = h->cfg;
    return DW_OK;
}

extern "C" dw_status mpm_batch_wind_layout(dw_mpm_batch h, int64_t *n_floats, int64_t *offsets) {
    DW_REQUIRE(h, "handle is NULL");
    if (n_floats) *n_floats = h->wind_off[h->n_scenes];
    if (offsets)
        for (int s = 0; s <= h->n_scenes; ++s) offsets[s] = h->wind_off[s];
    return DW_OK;
}

namespace dw {

// The reverse-mode workspace, allocated once per handle.
static dw_status ensure_adjoint(dw_mpm_batch h) {
    if (h->adj_scratch) return DW_OK;
    const int64_t nodes = h->node_off[h->n_scenes], n = h->n_total;
    cudaError_t e = cudaMalloc((void **)&h->grid_bv, sizeof(float4) * (size_t)nodes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->grid_bmp, sizeof(float4) * (size_t)nodes);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&h->d_node_off, sizeof(int64_t) * (size_t)h->n_scenes);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&h->d_wind_off, sizeof(int64_t) * (size_t)h->n_scenes);
    if (e == cudaSuccess) e = cudaMemset(h->grid_bv, 0, sizeof(float4) * (size_t)nodes);
    if (e == cudaSuccess) e = cudaMemset(h->grid_bmp, 0, sizeof(float4) * (size_t)nodes);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_node_off, h->node_off.data(), sizeof(int64_t) * (size_t)h->n_scenes,
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(h->d_wind_off, h->wind_off.data(), sizeof(int64_t) * (size_t)h->n_scenes,
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->adj_scratch, sizeof(float) * 12 * (size_t)n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->grid_bv);
        cudaFree(h->grid_bmp);
        cudaFree(h->d_node_off);
        cudaFree(h->d_wind_off);
        cudaFree(h->adj_scratch);
        h->grid_bv = h->grid_bmp = nullptr;
        h->d_node_off = h->d_wind_off = nullptr;
        h->adj_scratch = nullptr;
        if (e == cudaErrorMemoryAllocation) {
            set_error("out of device memory for the batch's reverse-mode workspace");
            return DW_ERR_OOM;
        }
        return cuda_fail(e, "mpm_batch_segment_adjoint");
    }
    return DW_OK;
}

// The grid tape for `slots` recompute substeps, grown on demand. It holds
// every block of every scene per slot (list_cap x 1 KB), so it is taken only
// while it leaves 8 GB of device memory free; without it the reverse pass
// recomputes each substep's grid by a P2G of its input (same results up to
// the float atomics' order). Returns whether the tape is there.
static bool ensure_grid_tape(dw_mpm_batch h, int slots) {
    if (slots <= 0) return false;
    if (slots <= h->gtape_slots) return true;
    if (h->gtape_refused && slots >= h->gtape_refused) return false;
    const size_t per = (size_t)h->list_cap * 64 * sizeof(float4) + (size_t)h->list_cap * sizeof(int);
    const size_t bytes = per * (size_t)slots + sizeof(int) * (size_t)slots;
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
    if (h->adj_exec) {  // a captured graph holds the old tape's addresses
        cudaGraphExecDestroy(h->adj_exec);
        h->adj_exec = nullptr;
    }
    cudaError_t e = cudaMalloc((void **)&h->gtape, (size_t)h->list_cap * 64 * sizeof(float4) * (size_t)slots);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&h->gtape_list, (size_t)h->list_cap * sizeof(int) * (size_t)slots);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->gtape_count, sizeof(int) * (size_t)slots);
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

}  // namespace dw

namespace dw {

// The launch sequence of a segment adjoint (the time t0 is already on the
// device): the recompute of states 1 .. n_substeps - 1 into the tape, then
// the reverse substeps.
static dw_status enqueue_segment_adjoint(dw_mpm_batch h, const dw_mpm_state *start, float *tape,
                                         const dw_mpm_state *g, const uint8_t *pinned,
                                         int n_substeps, float *g_wind, float *g_E,
                                         cudaStream_t s) {
    const int64_t n = h->n_total;
    dw_status st = DW_OK;
    const bool gt = h->gtape_slots >= n_substeps - 1 && n_substeps > 1;
    auto slot = [&](int k) {  // state k (1 .. n_substeps - 1) in the tape
        return state_view(tape + (size_t)(k - 1) * 24 * (size_t)n, n);
    };
    // recompute: one P2G of the start state, then substeps k = 0 .. n - 2,
    // each reading state k and writing state k + 1 whole into the tape while
    // it scatters the P2G of substep k + 1 (the last one does not scatter)
    if (n_substeps > 1) {
        DW_CUDA(cudaMemsetAsync(h->bar, 0, 2 * sizeof(unsigned), s));
        k_batch_p2g<<<h->n_items, BATCH_ITEM, 0, s>>>(view_of(h, *start, pinned), 0);
        DW_LAUNCHED("k_batch_p2g");
        int L = 0;
        for (int k = 0; k + 1 < n_substeps; ++k) {
            BatchView A = view_of(h, k == 0 ? *start : slot(k), pinned);
            const dw_mpm_state o = slot(k + 1);
            A.ox = o.x;
            A.ov = o.v;
            A.oC = o.C;
            A.oF = o.F;
            if (gt) {  // the grid phase of substep k keeps its grid in tape slot k
                A.gtape = h->gtape + (size_t)k * h->list_cap * 64;
                A.gtape_list = h->gtape_list + (size_t)k * h->list_cap;
                A.gtape_count = h->gtape_count + k;
            }
            const bool final_ = k + 2 == n_substeps;
            st = launch_substep(h, A, h->cfg, k, L, final_, s);
            if (st != DW_OK) return st;
            if (!final_) L = 1 - L;
        }
    }
    BatchAdjView R;
    R.node_off = h->d_node_off;
    R.wind_off = h->d_wind_off;
    R.grid_bv = h->grid_bv;
    R.grid_bmp = h->grid_bmp;
    R.scratch = h->adj_scratch;
    R.gx = g->x;
    R.gv = g->v;
    R.gC = g->C;
    R.gF = g->F;
    R.g_wind = g_wind;
    R.g_E = g_E;
    R.Cout = nullptr;
    const unsigned ggrid = (unsigned)(8 * h->num_sms);
    for (int j = n_substeps - 1; j >= 0; --j) {
        const dw_mpm_state in = j == 0 ? *start : slot(j);
        const BatchView A = view_of(h, in, pinned);
        if (gt && j + 1 < n_substeps) {  // the recompute kept substep j's grid
            k_batch_grid_restore<<<ggrid, 256, 0, s>>>(A, j, h->gtape + (size_t)j * h->list_cap * 64,
                                                      h->gtape_list + (size_t)j * h->list_cap,
                                                      h->gtape_count + j);
            DW_LAUNCHED("k_batch_grid_restore");
        } else {
            k_batch_p2g<<<h->n_items, BATCH_ITEM, 0, s>>>(A, 0);
            DW_LAUNCHED("k_batch_p2g");
            k_batch_grid_keep<<<ggrid, 256, 0, s>>>(A, j, 0);
            DW_LAUNCHED("k_batch_grid_keep");
        }
        // C of the output state j + 1, in the tape for every substep but the last
        R.Cout = j + 1 < n_substeps ? slot(j + 1).C : nullptr;
        k_batch_rev_g2p<<<h->n_items, BATCH_ITEM, 0, s>>>(A, R);
        DW_LAUNCHED("k_batch_rev_g2p");
        k_batch_rev_grid<<<ggrid, 256, 0, s>>>(A, R, j, 0);
        DW_LAUNCHED("k_batch_rev_grid");
        k_batch_rev_p2g<<<h->n_items, BATCH_ITEM, 0, s>>>(A, R, 0);
        DW_LAUNCHED("k_batch_rev_p2g");
    }
    return DW_OK;
}

// Captures the segment adjoint into h->adj_exec; false (and no error left
// behind) when it cannot be captured.
static bool capture_adjoint(dw_mpm_batch h, const dw_mpm_state *start, float *tape,
                            const dw_mpm_state *g, const uint8_t *pinned, int n_substeps,
                            float *g_wind, float *g_E) {
    if (h->adj_exec) cudaGraphExecDestroy(h->adj_exec);
    h->adj_exec = nullptr;
    if (!h->cap_stream &&
        cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    dw_status st = enqueue_segment_adjoint(h, start, tape, g, pinned, n_substeps, g_wind, g_E,
                                           h->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    bool ok = st == DW_OK && e == cudaSuccess && graph;
    if (ok) ok = cudaGraphInstantiate(&h->adj_exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (!ok) h->adj_exec = nullptr;
    return ok;
}

}  // namespace dw

extern "C" dw_status mpm_batch_segment_adjoint(dw_mpm_batch h, const dw_mpm_state *start,
                                               float *tape, int64_t tape_floats,
                                               const dw_mpm_state *g, const uint8_t *pinned,
                                               float t0, int32_t n_substeps, float *g_wind,
                                               float *g_E, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    dw_status st = check_batch_state(h, start);
    if (st != DW_OK) return st;
    st = check_batch_state(h, g);
    if (st != DW_OK) return st;
    DW_REQUIRE(n_substeps >= 0, "n_substeps must be >= 0");
    if (n_substeps == 0) return DW_OK;
    const int64_t n = h->n_total;
    const int64_t need = (int64_t)(n_substeps - 1) * 24 * n;
    DW_REQUIRE(n_substeps == 1 || (tape && tape_floats >= need),
               "tape holds %lld floats; %d substeps of %lld particles need %lld",
               (long long)tape_floats, n_substeps, (long long)n, (long long)need);
    st = ensure_adjoint(h);
    if (st != DW_OK) return st;
    ensure_grid_tape(h, n_substeps - 1);
    cudaStream_t s = as_stream(stream);
    k_batch_set_time<<<1, 1, 0, s>>>(h->t0, t0);
    DW_LAUNCHED("k_batch_set_time");
    if (h->cfg.use_graph && !h->adj_graph_broken) {
        // The graph reads the start state from the workspace, so that one
        // capture serves every segment of a rollout (each starts from its own
        // checkpoint).
        const dw_mpm_state ws = state_view(h->roll_state, n);
        const AdjKey key = {{ws.x, nullptr, nullptr, nullptr, tape, g->x, g->v, g->C, g->F, pinned,
                             g_wind, g_E},
                            n_substeps, h->cfg.mode, h->cfg.threads, h->cfg.ctas_per_sm};
        if (!h->adj_exec || !(key == h->adj_key)) {
            if (capture_adjoint(h, &ws, tape, g, pinned, n_substeps, g_wind, g_E))
                h->adj_key = key;
            else
                h->adj_graph_broken = true;
        }
        if (h->adj_exec) {
            const size_t b3 = sizeof(float) * 3 * (size_t)n, b9 = sizeof(float) * 9 * (size_t)n;
            DW_CUDA(cudaMemcpyAsync(ws.x, start->x, b3, cudaMemcpyDeviceToDevice, s));
            DW_CUDA(cudaMemcpyAsync(ws.v, start->v, b3, cudaMemcpyDeviceToDevice, s));
            DW_CUDA(cudaMemcpyAsync(ws.C, start->C, b9, cudaMemcpyDeviceToDevice, s));
            DW_CUDA(cudaMemcpyAsync(ws.F, start->F, b9, cudaMemcpyDeviceToDevice, s));
            DW_CUDA(cudaGraphLaunch(h->adj_exec, s));
            return DW_OK;
        }
    }
    return enqueue_segment_adjoint(h, start, tape, g, pinned, n_substeps, g_wind, g_E, s);
}

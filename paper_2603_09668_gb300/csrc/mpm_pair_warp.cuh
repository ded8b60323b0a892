// The warp body of the fused G2P/P2G substep with two particles per thread
// (k_g2p2g_pair of mpm_rollout.cu, and the batched k_batch_pair of
// mpm_batch.cu, whose warps each take 64 particles of one scene).
#pragma once

#include <limits.h>

#include "mpm_grid.cuh"
#include "mpm_pair.cuh"

namespace dw {

// The same substep body as k_g2p2g with two consecutive particles per thread (a warp holds 64), their arithmetic on float2 pairs
// (FFMA2, FMUL2, FADD2), which halves the FP32 instruction count.
//   G2P: the warp's particles, sorted by cell, lie in a few neighbouring
//   cells; lanes stage the grid velocities of the box spanned by all of the
//   warp's stencils in shared memory (at most BOX_MAX nodes, one load per
//   node), and every particle reads its 27 nodes from there. A warp whose box
//   is larger reads the grid directly.
//   P2G: per pass (one z layer of the stencil, 9 nodes) each lane writes its
//   two particles' summed node values into one row; when a run of equal cells
//   starts between the two particles, the second gets a row of its own right
//   after its lane's row, so rows stay in particle order. A warp whose rows
//   form one run sums them in three groups of lanes and issues one float4
//   atomic per node; otherwise three groups of lanes each walk a third of the
//   rows and flush a float4 atomic at every run end.
//   Active blocks of the next grid are marked for every run's first particle,
//   eight lanes per run; the flags of the first four runs are loaded before
//   the passes and tested after them.
constexpr int PAIR_THREADS = 128;
constexpr int PAIR_WARPS = PAIR_THREADS / 32;
// resident CTAs per SM the launch bounds ask for: 96 registers per thread
constexpr int PAIR_MIN_CTAS = 65536 / (96 * PAIR_THREADS);
constexpr unsigned FULL = 0xffffffffu;

template <bool VEC>
__device__ __forceinline__ float2 ld_pair(const float *a, int64_t q, bool v1) {
    if (VEC) return __ldcg(reinterpret_cast<const float2 *>(a + q));
    return make_float2(__ldcg(a + q), v1 ? __ldcg(a + q + 1) : 0.0f);
}

template <bool VEC>
__device__ __forceinline__ void st_pair(float *a, int64_t q, float2 v, bool v1) {
    if (VEC) {
        *reinterpret_cast<float2 *>(a + q) = v;
    } else {
        a[q] = v.x;
        if (v1) a[q + 1] = v.y;
    }
}

__device__ __forceinline__ void mark_block(const ActiveBlocks &ab, int id) {
    if (*(volatile int *)&ab.flags[id] == 0 && atomicExch(&ab.flags[id], 1) == 0)
        ab.list[atomicAdd(ab.count, 1)] = ab.tag | id;
}

// Block d (bit a of d: one block further along axis a) of the blocks that the
// stencil of base cell `base` touches; -1 when the stencil does not reach it.
__device__ __forceinline__ int stencil_block(const ActiveBlocks &ab, int bx, int by, int bz, int d) {
    const int cx = (bx >> 2) + (d & 1), cy = (by >> 2) + ((d >> 1) & 1), cz = (bz >> 2) + (d >> 2);
    if (cx > ((bx + 2) >> 2) || cy > ((by + 2) >> 2) || cz > ((bz + 2) >> 2)) return -1;
    return (cz * ab.nb + cy) * ab.nb + cx;
}

// Per-warp shared memory of k_g2p2g_pair, reused between the phases.
constexpr int BOX_MAX = 256;  // staged grid nodes per warp
constexpr int PAIR_ROWS = 64;  // at most one row per particle
struct PairWarpSmem {
    union {
        struct {
            float box[3 * BOX_MAX];  // G2P: grid velocity components of the warp's box of nodes
            float F[9][64];          // F of the warp's 64 particles (copied before the wait)
        } g;
        float4 rows[PAIR_ROWS + 1][P2G_ROW];  // P2G: node values per row (+ a zero row)
    };
    int keys[PAIR_ROWS];  // cell of each row (-1: adds nothing)
};

// Rows of one run (32 rows): lanes 9g + L sum rows 11g .. 11g + 10 of node L
// (row 32 is zero), the three partial sums meet in lanes 0-8, one float4
// atomic per node.
__device__ __forceinline__ void rows_one_run(const float4 (*rows)[P2G_ROW], int key, int ok, int N,
                                             float4 *__restrict__ grid) {
    const int lane = threadIdx.x & 31;
    const int g = lane / 9, L = lane - 9 * g;
    float2 a = pr::s2(0.0f), b = pr::s2(0.0f);
    if (g < 3) {
        const float4 (*rr)[P2G_ROW] = rows + 11 * g;
#pragma unroll
        for (int i = 0; i < 11; ++i) {
            const float4 t = rr[i][L];
            a = pr::add(a, make_float2(t.x, t.y));
            b = pr::add(b, make_float2(t.z, t.w));
        }
    }
#pragma unroll
    for (int d = 9; d <= 18; d += 9) {
        const float ax = __shfl_down_sync(FULL, a.x, d), ay = __shfl_down_sync(FULL, a.y, d);
        const float bx = __shfl_down_sync(FULL, b.x, d), by = __shfl_down_sync(FULL, b.y, d);
        if (lane < 9 && lane + d < 27) {
            a = pr::add(a, make_float2(ax, ay));
            b = pr::add(b, make_float2(bx, by));
        }
    }
    if (lane < 9 && key >= 0)
        atomicAdd(&grid[key + (ok * N + L / 3) * N + L % 3], make_float4(a.x, a.y, b.x, b.y));
}

// Any number of runs: the rows (in particle order) are cut into three
// ranges of `per` rows; lane 9g + L walks range g (rows r0 .. r0 + cnt - 1,
// cnt <= NR) for node L and flushes its sum with a float4 atomic at every run
// end and at the end of its range (a run that crosses a range boundary is
// flushed in parts). e: bit i set when row r0 + i ends a run or the range.
template <int NR>
__device__ __forceinline__ void rows_walk(const float4 (*rows)[P2G_ROW], const int *keys, int r0,
                                          int cnt, unsigned e, int ok, int N,
                                          float4 *__restrict__ grid) {
    const int lane = threadIdx.x & 31;
    const int g = lane / 9, L = lane - 9 * g;
    if (g >= 3) return;
    const int off = (ok * N + L / 3) * N + L % 3;
    const float4 (*rr)[P2G_ROW] = rows + r0;
    const int *kk = keys + r0;
    float2 a = pr::s2(0.0f), b = pr::s2(0.0f);
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        if (i >= 11 && i >= cnt) break;  // ranges of up to 11 rows need no test
        const float4 t = rr[i][L];
        a = pr::add(a, make_float2(t.x, t.y));
        b = pr::add(b, make_float2(t.z, t.w));
        if ((e >> i) & 1u) {
            const int k = kk[i];
            if (k >= 0) atomicAdd(&grid[k + off], make_float4(a.x, a.y, b.x, b.y));
            a = pr::s2(0.0f);
            b = a;
        }
    }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// G2P of a warp whose stencils span more than BOX_MAX nodes: both particles
// read the grid directly. Inlined: an out-of-line call keeps the stencil and
// the G2P sums, whose addresses it takes, in local memory on every path.
__device__ __forceinline__ void g2p_direct(const MpmParams &P, const pr::Stencil2 &s,
                                        const float4 *__restrict__ grid_v, float2 *vn, float2 *Cn) {
    const int N = P.N;
    const int gk0 = (s.b0[2] * N + s.b0[1]) * N + s.b0[0];
    const int gk1 = (s.b1[2] * N + s.b1[1]) * N + s.b1[0];
    float2 v[3], c[9];
    pr::g2p_sums2<false>(P, s, grid_v + gk0, grid_v + gk1, v, c);
#pragma unroll
    for (int a = 0; a < 3; ++a) vn[a] = v[a];
#pragma unroll
    for (int k = 0; k < 9; ++k) Cn[k] = c[k];
}

// Output arrays of a substep that writes its whole output state elsewhere
// (the recompute of a reverse segment: state k in, state k + 1 out), and the
// next sort's key and count arrays (the substep before a re-sort).
struct PairOut {
    float *x = nullptr, *v = nullptr, *C = nullptr, *F = nullptr;
    int *keys = nullptr;    // [n] cell key of each updated particle (KEYS)
    int *counts = nullptr;  // [keys] particles per key, added to (KEYS)
};

// The substep body for one warp: particles wq .. min(wq + 64, wend) - 1 of
// arrays with row stride n. MAT < 0 takes the material from P at run time
// (warp-uniform). reset_count, when not NULL, is cleared after the
// dependency wait (the active list the grid update has consumed). With OUT
// the updated x, v, C and F go to `out` (x and F are not updated in place).
// With KEYS the substep also writes the sort key (cell_key) of every updated
// particle to out.keys and counts it in out.counts (one atomic per distinct
// key of a warp and particle slot), the first pass of the re-sort after it.
template <int MAT, bool STORE_VC, bool VEC, bool OUT = false, bool KEYS = false>
__device__ __forceinline__ void pair_warp(
    const MpmParams &P, float *__restrict__ x, float *__restrict__ v, float *__restrict__ C,
    float *__restrict__ F, const uint8_t *__restrict__ pinned, const float4 *__restrict__ grid_v,
    float4 *__restrict__ grid_next, int64_t n, int64_t wq, int64_t wend, int *err,
    const ActiveBlocks &ab_next, int *reset_count, PairWarpSmem &ws, PairOut out = {}) {
    using namespace pr;
    const int lane = threadIdx.x & 31;
    const int64_t q = wq + 2 * lane;
    const bool v0 = q < wend, v1 = q + 1 < wend;
    // Before the dependency wait (x and F were last written two launches
    // back, see k_g2p2g): x into registers; with VEC (n a multiple of 4,
    // 16-byte aligned arrays) F of a full 64-particle group is copied into
    // shared memory in 16-byte pieces through L2, else F is loaded later.
    float2 xp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) xp[a] = s2(0.0f);
    bool pin0 = false, pin1 = false;
    const bool full = wq + 64 <= wend;
    if (v0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) xp[a] = ld_pair<VEC>(x + a * n, q, v1);
        if (pinned) {
            pin0 = pinned[q] != 0;
            pin1 = v1 && pinned[q + 1] != 0;
        }
    }
    if (VEC && full) {
        for (int i = lane; i < 144; i += 32) {  // 9 rows of 64 floats
            const int k = i >> 4, c = (i & 15) * 4;
            cp_async16(&ws.g.F[k][c], F + k * n + wq + c);
        }
        cp_async_commit();
    }
    const int N = P.N;

    // ---------------------------------------------------------------- G2P
    float2 vn[3], Cn[9];
    bool g0ok, g1ok;
    {
        // The stencils and the warp's box depend on x alone, so they are
        // computed before the dependency wait; the grid is read after it.
        Stencil2 s;
        stencil2(P, xp, s, g0ok, g1ok);
        g0ok = g0ok && v0;
        g1ok = g1ok && v1;
        // box of the warp's stencils (particles with a stencil on the grid)
        int lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = __reduce_min_sync(FULL, min(g0ok ? s.b0[a] : INT_MAX, g1ok ? s.b1[a] : INT_MAX));
            hi[a] = __reduce_max_sync(FULL, max(g0ok ? s.b0[a] : INT_MIN, g1ok ? s.b1[a] : INT_MIN));
        }
        const int ex = hi[0] - lo[0] + 3, ey = hi[1] - lo[1] + 3, ez = hi[2] - lo[2] + 3;
        const bool any = lo[0] <= hi[0];
        const int vol = any ? ex * ey * ez : 0;
        pdl_wait();
        pdl_trigger();
        if (reset_count) *reset_count = 0;
        const unsigned vmask = __ballot_sync(FULL, v0);
        if (vmask == 0) return;  // the whole warp lies beyond n
        if (any && vol <= BOX_MAX) {
            // stage the box (lanes stride over its nodes), then read it per particle
            const int exy = ex * ey;
            const float inv_exy = 1.0f / (float)exy, inv_ex = 1.0f / (float)ex;
            for (int i = lane; i < vol; i += 32) {
                const int iz = (int)(((float)i + 0.5f) * inv_exy);  // exact for i < 256
                const int rem = i - iz * exy;
                const int iy = (int)(((float)rem + 0.5f) * inv_ex);
                const int ix = rem - iy * ex;
                const float4 g = grid_v[((lo[2] + iz) * N + (lo[1] + iy)) * N + (lo[0] + ix)];
                ws.g.box[i] = g.x;
                ws.g.box[BOX_MAX + i] = g.y;
                ws.g.box[2 * BOX_MAX + i] = g.z;
            }
            __syncwarp();
            const int o0 = g0ok ? ((s.b0[2] - lo[2]) * ey + (s.b0[1] - lo[1])) * ex + (s.b0[0] - lo[0]) : 0;
            const int o1 = g1ok ? ((s.b1[2] - lo[2]) * ey + (s.b1[1] - lo[1])) * ex + (s.b1[0] - lo[0]) : 0;
            g2p_box2<BOX_MAX>(P, s, ws.g.box, o0, o1, ex, exy, vn, Cn);
        } else {
            g2p_direct(P, s, grid_v, vn, Cn);
        }
    }
    float2 Fp[9];
    if (VEC && full) {
        cp_async_wait_all();
        __syncwarp();  // pieces copied by the other lanes
#pragma unroll
        for (int k = 0; k < 9; ++k) Fp[k] = *reinterpret_cast<const float2 *>(&ws.g.F[k][2 * lane]);
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) Fp[k] = v0 ? ld_pair<VEC>(F + k * n, q, v1) : s2(0.0f);
    }
    __syncwarp();  // the box and F are read: the rows may overwrite them
    if (lane < 9) ws.rows[32][lane] = make_float4(0.f, 0.f, 0.f, 0.f);  // pad of rows_one_run
    // pinned particles: v = C = 0; a stencil off the grid: unchanged, v = C = 0
    const bool z0 = pin0 || !g0ok, z1 = pin1 || !g1ok;
    if (z0 || z1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) vn[c] = make_float2(z0 ? 0.0f : vn[c].x, z1 ? 0.0f : vn[c].y);
#pragma unroll
        for (int k = 0; k < 9; ++k) Cn[k] = make_float2(z0 ? 0.0f : Cn[k].x, z1 ? 0.0f : Cn[k].y);
    }
    float2 Fn[9];
    {
        const float2 dt2 = s2(P.dt);
        float2 M[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) M[k] = mul(dt2, Cn[k]);
        M[0] = add(M[0], s2(1.0f));
        M[4] = add(M[4], s2(1.0f));
        M[8] = add(M[8], s2(1.0f));
        mul3_2(M, Fp, Fn);
#pragma unroll
        for (int a = 0; a < 3; ++a) xp[a] = fma(dt2, vn[a], xp[a]);
    }
    if (v0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) st_pair<VEC>((OUT ? out.x : x) + a * n, q, xp[a], v1);
#pragma unroll
        for (int k = 0; k < 9; ++k) st_pair<VEC>((OUT ? out.F : F) + k * n, q, Fn[k], v1);
        if (STORE_VC || OUT) {
#pragma unroll
            for (int a = 0; a < 3; ++a) st_pair<VEC>((OUT ? out.v : v) + a * n, q, vn[a], v1);
#pragma unroll
            for (int k = 0; k < 9; ++k) st_pair<VEC>((OUT ? out.C : C) + k * n, q, Cn[k], v1);
        }
        // one non-finite entry makes the sum non-finite
        float2 sum = add(add(xp[0], xp[1]), xp[2]);
#pragma unroll
        for (int k = 0; k < 9; ++k) sum = add(sum, Fn[k]);
        if (!isfinite(sum.x) || (v1 && !isfinite(sum.y))) atomicOr(err, ERRBIT_NONFINITE);
    }

    // ------------------------------------------------ P2G of the next substep
    float2 A[9];
    bool a0ok, a1ok;
    affine2<MAT>(P, Fn, Cn, A, a0ok, a1ok);
    float2 mv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) mv[c] = mul(s2(P.p_mass), vn[c]);
    Stencil2 t;
    bool p0ok, p1ok;
    stencil2(P, xp, t, p0ok, p1ok);
    if (KEYS) {
        const int kk0 = cell_key(P, ab_next.nb, xp[0].x, xp[1].x, xp[2].x);
        const int kk1 = cell_key(P, ab_next.nb, xp[0].y, xp[1].y, xp[2].y);
        const unsigned m0 = __ballot_sync(FULL, v0), m1 = __ballot_sync(FULL, v1);
        if (v0) {
            out.keys[q] = kk0;
            const unsigned peers = __match_any_sync(m0, kk0);
            if (lane == __ffs(peers) - 1) atomicAdd(&out.counts[kk0], __popc(peers));
        }
        if (v1) {
            out.keys[q + 1] = kk1;
            const unsigned peers = __match_any_sync(m1, kk1);
            if (lane == __ffs(peers) - 1) atomicAdd(&out.counts[kk1], __popc(peers));
        }
    }
    if ((v0 && !p0ok) || (v1 && !p1ok)) atomicOr(err, ERRBIT_DOMAIN);
    p0ok = p0ok && v0;
    p1ok = p1ok && v1;
    if ((p0ok && !a0ok) || (p1ok && !a1ok)) atomicOr(err, ERRBIT_INVERTED);
    const int nk0 = p0ok ? (t.b0[2] * N + t.b0[1]) * N + t.b0[0] : -1;
    const int nk1 = p1ok ? (t.b1[2] * N + t.b1[1]) * N + t.b1[0] : -1;
    // a particle without a stencil adds nothing
    if (!p0ok || !p1ok) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t.fx[a] = make_float2(p0ok ? t.fx[a].x : 1.0f, p1ok ? t.fx[a].y : 1.0f);
#pragma unroll
            for (int o = 0; o < 3; ++o)
                t.w[a][o] = make_float2(p0ok ? t.w[a][o].x : 0.0f, p1ok ? t.w[a][o].y : 0.0f);
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) A[k] = make_float2(p0ok ? A[k].x : 0.0f, p1ok ? A[k].y : 0.0f);
#pragma unroll
        for (int c = 0; c < 3; ++c) mv[c] = make_float2(p0ok ? mv[c].x : 0.0f, p1ok ? mv[c].y : 0.0f);
    }
    // node value = W (m, r0 + oi sx + oj sy + ok sz), r0 = m v - A fx dx, s = dx A's columns
    float2 r0[3], sx[3], sy[3], sz[3];
    {
        const float2 dxs = s2(P.dx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 in = fma(A[3 * c + 2], t.fx[2], fma(A[3 * c + 1], t.fx[1], mul(A[3 * c], t.fx[0])));
            r0[c] = fnma(in, dxs, mv[c]);
            sx[c] = mul(A[3 * c], dxs);
            sy[c] = mul(A[3 * c + 1], dxs);
            sz[c] = mul(A[3 * c + 2], dxs);
        }
    }
    // Rows, in particle order: a lane adds its two particles into one row;
    // when its second particle lies in another cell (a run starts inside the
    // pair) that particle gets a row of its own right after the lane's row.
    const bool split = nk1 >= 0 && nk1 != nk0;
    const unsigned smask = __ballot_sync(FULL, split);
    const int pos = lane + __popc(smask & ((1u << lane) - 1u));  // this lane's row
    const int R = 32 + __popc(smask);
    float w2y[3];  // the second particle's z weights, kept out of the summed row when split
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        w2y[o] = t.w[2][o].y;
        if (split) t.w[2][o].y = 0.0f;
    }
    uint64_t ends;
    bool st_main;
    {
        const int lastkey = split ? nk1 : nk0;
        const int prevlast = __shfl_up_sync(FULL, lastkey, 1);
        st_main = lane == 0 || nk0 != prevlast;
        unsigned lo = 0u, hi = 0u;
        if (st_main) {
            if (pos < 32) lo |= 1u << pos; else hi |= 1u << (pos - 32);
        }
        if (split) {
            if (pos + 1 < 32) lo |= 1u << (pos + 1); else hi |= 1u << (pos + 1 - 32);
        }
        lo = __reduce_or_sync(FULL, lo);
        hi = __reduce_or_sync(FULL, hi);
        const uint64_t starts = ((uint64_t)hi << 32) | lo;
        ends = (starts >> 1) | (1ull << (R - 1));
        ws.keys[pos] = nk0;
        if (split) ws.keys[pos + 1] = nk1;
    }
    const bool one_run = R == 32 && ends == (1ull << 31);
    const int per = (R + 2) / 3, gw = lane / 9;
    const int wr0 = gw * per, wcnt = max(0, min(R, wr0 + per) - wr0);
    const unsigned e_walk = (gw < 3 && wcnt > 0)
                                ? (unsigned)((ends >> wr0) & ((1ull << per) - 1ull)) | (1u << (wcnt - 1))
                                : 0u;
    // Active blocks of the next grid: the stencil blocks of every run's first
    // particle, four runs at a time (eight lanes per run, one block per lane).
    // The flags of the first four runs are loaded now and tested after the
    // passes, so that the loads' latency overlaps them.
    const unsigned m0 = __ballot_sync(FULL, st_main && nk0 >= 0), m1 = smask;
    const int n0 = __popc(m0), nr = n0 + __popc(m1);
    auto mark_id = [&](int j0) {
        const int j = j0 + (lane >> 3);
        int src = 0, h = 0;
        if (j < nr) {
            if (j < n0) {
                src = __fns(m0, 0, j + 1);
            } else {
                src = __fns(m1, 0, j - n0 + 1);
                h = 1;
            }
        }
        const int c0 = __shfl_sync(FULL, t.b0[0], src), c1 = __shfl_sync(FULL, t.b0[1], src),
                  c2 = __shfl_sync(FULL, t.b0[2], src);
        const int d0 = __shfl_sync(FULL, t.b1[0], src), d1 = __shfl_sync(FULL, t.b1[1], src),
                  d2 = __shfl_sync(FULL, t.b1[2], src);
        if (j >= nr) return -1;
        return h ? stencil_block(ab_next, d0, d1, d2, lane & 7)
                 : stencil_block(ab_next, c0, c1, c2, lane & 7);
    };
    int mid = -1, mflag = 1;
    if (ab_next.flags) {
        mid = mark_id(0);
        if (mid >= 0) mflag = *(volatile int *)&ab_next.flags[mid];
    }
    const float2 pm = s2(P.p_mass);
    // one z layer of the stencil per pass, the pass body kept once (code size)
#pragma unroll 1
    for (int ok = 0; ok < 3; ++ok) {
        const float2 wz = ok == 0 ? t.w[2][0] : (ok == 1 ? t.w[2][1] : t.w[2][2]);
        const float wz1 = ok == 0 ? w2y[0] : (ok == 1 ? w2y[1] : w2y[2]);
        float2 rz[3];  // r0 + ok sz
#pragma unroll
        for (int c = 0; c < 3; ++c) rz[c] = ok == 0 ? r0[c] : fma(s2((float)ok), sz[c], r0[c]);
#pragma unroll
        for (int oj = 0; oj < 3; ++oj) {
            const float2 wyz = mul(t.w[1][oj], wz);
            const float wyz1 = t.w[1][oj].y * wz1;
            float2 b[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 u = rz[c];
                if (oj == 1) u = add(u, sy[c]);
                if (oj == 2) u = fma(s2(2.0f), sy[c], u);
                b[c] = u;
            }
#pragma unroll
            for (int oi = 0; oi < 3; ++oi) {
                const float2 W = mul(t.w[0][oi], wyz);
                float2 bb[3];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    bb[c] = oi == 0 ? b[c] : (oi == 1 ? add(b[c], sx[c]) : fma(s2(2.0f), sx[c], b[c]));
                const float2 Wm = mul(W, pm), v0p = mul(W, bb[0]), v1p = mul(W, bb[1]),
                             v2p = mul(W, bb[2]);
                ws.rows[pos][3 * oj + oi] =
                    make_float4(Wm.x + Wm.y, v0p.x + v0p.y, v1p.x + v1p.y, v2p.x + v2p.y);
                if (smask) {
                    const float W1 = t.w[0][oi].y * wyz1;
                    if (split)
                        ws.rows[pos + 1][3 * oj + oi] = make_float4(W1 * P.p_mass, W1 * bb[0].y,
                                                                    W1 * bb[1].y, W1 * bb[2].y);
                }
            }
        }
        __syncwarp();
        if (one_run)
            rows_one_run(ws.rows, ws.keys[0], ok, N, grid_next);
        else if (R <= 33)
            rows_walk<11>(ws.rows, ws.keys, wr0, wcnt, e_walk, ok, N, grid_next);
        else
            rows_walk<22>(ws.rows, ws.keys, wr0, wcnt, e_walk, ok, N, grid_next);
        __syncwarp();
    }
    if (ab_next.flags) {
        if (mid >= 0 && mflag == 0 && atomicExch(&ab_next.flags[mid], 1) == 0)
            ab_next.list[atomicAdd(ab_next.count, 1)] = ab_next.tag | mid;
        for (int j0 = 4; j0 < nr; j0 += 4) {
            const int id = mark_id(j0);
            if (id >= 0) mark_block(ab_next, id);
        }
    }
}

}  // namespace dw

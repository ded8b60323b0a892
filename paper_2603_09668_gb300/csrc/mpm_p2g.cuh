// P2G (Eq. P2G plus the MLS-MPM stress momentum) in three accumulation
// strategies that give the same sums up to float rounding order:
//   DW_P2G_ATOMIC : every particle adds its 27 node contributions to the HBM
//                   grid with float4 atomics.
//   DW_P2G_WARP   : lanes of a warp whose particles share a base cell (runs of
//                   equal cell keys, as produced by mpm_sort) sum their
//                   contributions through a shared-memory transpose and issue
//                   one float4 atomic per node and run (the default: AUTO).
//   DW_P2G_TILE   : a CTA accumulates its particles into a shared-memory tile
//                   spanning their stencils' bounding box (shared atomics, each
//                   lane walking the 27 nodes in a lane-rotated order so lanes
//                   of one cell hit distinct addresses), then flushes the
//                   non-empty tile nodes to HBM with float4 atomics. A CTA whose
//                   particles span more than the tile falls back to ATOMIC.
#pragma once

#include "mpm_math.cuh"

namespace dw {

// Active 4^3-node blocks: P2G marks every block its stencils touch and appends
// newly marked blocks to a list, so the grid update visits only those blocks.
// flags == nullptr disables the marking (the dense grid update is used then).
struct ActiveBlocks {
    int *flags;  // [nb^3], zero between substeps
    int *list;   // [nb^3]
    int *count;  // [1], zero between substeps
    int nb;      // blocks per axis
    int tag;     // or-ed into every list entry (the scene of a batched list)
};

__device__ __forceinline__ void mark_stencil_blocks(const ActiveBlocks &ab, const int base[3]) {
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = base[a] >> 2;
        hi[a] = (base[a] + 2) >> 2;
    }
    for (int bz = lo[2]; bz <= hi[2]; ++bz)
        for (int by = lo[1]; by <= hi[1]; ++by)
            for (int bx = lo[0]; bx <= hi[0]; ++bx) {
                int id = (bz * ab.nb + by) * ab.nb + bx;
                if (*(volatile int *)&ab.flags[id] == 0 && atomicExch(&ab.flags[id], 1) == 0)
                    ab.list[atomicAdd(ab.count, 1)] = ab.tag | id;
            }
}

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

// ------------------------------------------------------------ warp-aggregated
//
// Each warp reduces the contributions of lanes whose particles share a base
// cell (runs of equal keys among consecutive lanes; after mpm_sort most warps
// of a dense object are a single run) through a shared-memory transpose: every
// lane writes its node values (float4: m, p) into its own row, then the rows
// of each node are summed per run and one float4 atomic per node and run is
// issued (27 lanes sum a single run or two runs; more runs: lane L walks the
// 32 rows of node L). The 27
// stencil nodes go in three passes of 9 to keep the buffer small; a row of 9
// float4 (144 B) keeps the float4 row stores free of bank conflicts.

constexpr int P2G_WARP_THREADS = 128;
constexpr int P2G_PASS = 9;  // nodes per pass
constexpr int P2G_ROW = 9;   // float4 per row

// TWO_RUN enables the 27-lane two-run reduction; it pays off in the
// standalone scatter kernels, while the fused G2P/P2G kernel, already at its
// register and instruction-cache limits, runs faster without it.
template <bool TWO_RUN = false>
__device__ __forceinline__ void p2g_warp_scatter(const MpmParams &P, P2GParticle &q,
                                                 float4 *__restrict__ grid, const ActiveBlocks &ab,
                                                 float4 (*rows)[P2G_ROW], int *keys) {
    const int lane = threadIdx.x & 31;
    const int N = P.N;
    const int key = q.valid ? (q.s.base[2] * N + q.s.base[1]) * N + q.s.base[0] : -1;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned starts = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
    const unsigned ends = (starts >> 1) | 0x80000000u;
    keys[lane] = key;
    if (ab.flags && q.valid && ((starts >> lane) & 1u)) mark_stencil_blocks(ab, q.s.base);
    if (!q.valid) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            q.s.fx[a] = 1.0f;
#pragma unroll
            for (int o = 0; o < 3; ++o) q.s.w[a][o] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) q.A[k] = 0.0f;
        q.mv[0] = q.mv[1] = q.mv[2] = 0.0f;
    }
    // node value = W_o (r0 + oi sx + oj sy + ok sz) with r0 = m v - A fx dx and
    // s = dx times the columns of A; the mass part is W_o m
    float r0[3], sx[3], sy[3], sz[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        r0[c] = q.mv[c] - (q.A[3 * c] * q.s.fx[0] + q.A[3 * c + 1] * q.s.fx[1] + q.A[3 * c + 2] * q.s.fx[2]) * P.dx;
        sx[c] = q.A[3 * c] * P.dx;
        sy[c] = q.A[3 * c + 1] * P.dx;
        sz[c] = q.A[3 * c + 2] * P.dx;
    }
#pragma unroll
    for (int pass = 0; pass < 3; ++pass) {
        // pass = ok: the 9 nodes of one z layer, line by line along x
        const int ok = pass;
#pragma unroll
        for (int oj = 0; oj < 3; ++oj) {
            const float wyz = q.s.w[1][oj] * q.s.w[2][ok];
            float b[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float t = r0[c];
                if (oj == 1) t += sy[c];
                if (oj == 2) t += 2.0f * sy[c];
                if (ok == 1) t += sz[c];
                if (ok == 2) t += 2.0f * sz[c];
                b[c] = t;
            }
#pragma unroll
            for (int oi = 0; oi < 3; ++oi) {
                const float W = q.s.w[0][oi] * wyz;
                float4 val;
                val.x = W * P.p_mass;
                val.y = W * (oi == 0 ? b[0] : (oi == 1 ? b[0] + sx[0] : b[0] + 2.0f * sx[0]));
                val.z = W * (oi == 0 ? b[1] : (oi == 1 ? b[1] + sx[1] : b[1] + 2.0f * sx[1]));
                val.w = W * (oi == 0 ? b[2] : (oi == 1 ? b[2] + sx[2] : b[2] + 2.0f * sx[2]));
                rows[lane][3 * oj + oi] = val;
            }
        }
        __syncwarp();
        if (ends == 0x80000000u) {
            // The whole warp is one run (dense objects, sorted): lanes 9g + L
            // (g = 0, 1, 2) sum rows 11g .. 11g + 10 of node L, then the three
            // partial sums meet in lane L.
            const int g = lane / 9, L = lane - 9 * g;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g < 3) {
                const int r0i = 11 * g, r1i = min(32, r0i + 11);
#pragma unroll 4
                for (int r = r0i; r < r1i; ++r) {
                    const float4 t = rows[r][L];
                    acc.x += t.x;
                    acc.y += t.y;
                    acc.z += t.z;
                    acc.w += t.w;
                }
            }
#pragma unroll
            for (int d = 9; d <= 18; d += 9) {
                const float ax = __shfl_down_sync(0xffffffffu, acc.x, d);
                const float ay = __shfl_down_sync(0xffffffffu, acc.y, d);
                const float az = __shfl_down_sync(0xffffffffu, acc.z, d);
                const float aw = __shfl_down_sync(0xffffffffu, acc.w, d);
                if (lane < 9 && lane + d < 27) {
                    acc.x += ax;
                    acc.y += ay;
                    acc.z += az;
                    acc.w += aw;
                }
            }
            const int k = keys[0];
            if (lane < 9 && k >= 0) {
                const int off = (ok * N + lane / 3) * N + lane % 3;
                atomicAdd(&grid[(int64_t)k + off], acc);
            }
        } else if (TWO_RUN && __popc(starts) == 2) {
            // Two runs (a warp across one cell boundary, the common case
            // after it in a dense object): as above, with one accumulator
            // per run; rows b.. belong to the second run.
            const int b = __ffs(starts & ~1u) - 1;
            const int g = lane / 9, L = lane - 9 * g;
            float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
            if (g < 3) {
                const int r0i = 11 * g, r1i = min(32, r0i + 11);
#pragma unroll 4
                for (int r = r0i; r < r1i; ++r) {
                    const float4 t = rows[r][L];
                    const float f0 = r < b ? 1.0f : 0.0f, f1 = 1.0f - f0;
                    a0.x = fmaf(f0, t.x, a0.x);
                    a0.y = fmaf(f0, t.y, a0.y);
                    a0.z = fmaf(f0, t.z, a0.z);
                    a0.w = fmaf(f0, t.w, a0.w);
                    a1.x = fmaf(f1, t.x, a1.x);
                    a1.y = fmaf(f1, t.y, a1.y);
                    a1.z = fmaf(f1, t.z, a1.z);
                    a1.w = fmaf(f1, t.w, a1.w);
                }
            }
#pragma unroll
            for (int d = 9; d <= 18; d += 9) {
                const float x0 = __shfl_down_sync(0xffffffffu, a0.x, d);
                const float y0 = __shfl_down_sync(0xffffffffu, a0.y, d);
                const float z0 = __shfl_down_sync(0xffffffffu, a0.z, d);
                const float w0 = __shfl_down_sync(0xffffffffu, a0.w, d);
                const float x1 = __shfl_down_sync(0xffffffffu, a1.x, d);
                const float y1 = __shfl_down_sync(0xffffffffu, a1.y, d);
                const float z1 = __shfl_down_sync(0xffffffffu, a1.z, d);
                const float w1 = __shfl_down_sync(0xffffffffu, a1.w, d);
                if (lane < 9 && lane + d < 27) {
                    a0.x += x0;
                    a0.y += y0;
                    a0.z += z0;
                    a0.w += w0;
                    a1.x += x1;
                    a1.y += y1;
                    a1.z += z1;
                    a1.w += w1;
                }
            }
            if (lane < 9) {
                const int off = (ok * N + lane / 3) * N + lane % 3;
                const int k0 = keys[0], k1 = keys[b];
                if (k0 >= 0) atomicAdd(&grid[(int64_t)k0 + off], a0);
                if (k1 >= 0) atomicAdd(&grid[(int64_t)k1 + off], a1);
            }
        } else if (lane < P2G_PASS) {
            const int off = (ok * N + lane / 3) * N + lane % 3;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
            for (int r = 0; r < 32; ++r) {
                const float4 t = rows[r][lane];
                acc.x += t.x;
                acc.y += t.y;
                acc.z += t.z;
                acc.w += t.w;
                if ((ends >> r) & 1u) {
                    const int k = keys[r];
                    if (k >= 0) atomicAdd(&grid[(int64_t)k + off], acc);
                    acc = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
        __syncwarp();
    }
}

// Launches P2G of n particles into grid (DW_P2G_* strategy); defined in mpm_p2g.cu.
dw_status launch_p2g(int mode, const MpmParams &P, const float *x, const float *v, const float *C,
                     const float *F, int64_t n, float4 *grid, int *err, const ActiveBlocks &ab,
                     cudaStream_t st);

}  // namespace dw

// mpm_rollout: many substeps of one scene in one call, with the G2P of
// substep k and the P2G of substep k + 1 fused into one kernel.
//
// A substep is P2G -> grid update -> G2P (Eq. simulation_mpm). Inside a
// rollout the particle state between two substeps is consumed only by the
// next P2G, so k_g2p2g does, per particle: gather the grid velocities of
// substep k (G2P), update x and F, then scatter the updated particle into the
// zeroed grid of substep k + 1 (P2G) while v and C are still in registers.
// Per inner substep the particle arrays see one read and one write of x and F
// (96 B per particle) instead of the four arrays of the unfused kernels.
// Every `sort_every` substeps the particles are re-sorted by cell between two
// fused launches (the P2G of the next substep has run in the old order; the
// grid does not depend on the order), moving x, F, pinned and ids: v and C
// are written only by the G2P of the last substep, where the state is
// complete.
#include <limits.h>
#include <math.h>

#include "mpm_handle.cuh"
#include "mpm_pair_warp.cuh"

namespace dw {

// Loads x and F of particle p through L2 (ld.global.cg).
__device__ __forceinline__ void load_xF(const float *x, const float *F, int64_t n, int64_t p,
                                        float xp[3], float Fp[9]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) xp[a] = __ldcg(x + a * n + p);
#pragma unroll
    for (int k = 0; k < 9; ++k) Fp[k] = __ldcg(F + k * n + p);
}

// One thread per particle. x and F are loaded before the programmatic-launch
// wait: they were last written two launches back by a kernel that has
// completed once this one runs (the grid update in between waits for it before
// it lets this kernel start), and the loads go through L2; only grid_v, which
// the grid update writes, is read after the wait.
// Ten resident CTAs per SM (48 registers, a few spilled) hide more of the
// grid-velocity gather latency than the eight that 64 registers allow.
template <bool STORE_VC>
__global__ void __launch_bounds__(P2G_WARP_THREADS, 10) k_g2p2g(
    MpmParams P, float *__restrict__ x, float *__restrict__ v, float *__restrict__ C,
    float *__restrict__ F, const uint8_t *__restrict__ pinned, const float4 *__restrict__ grid_v,
    float4 *__restrict__ grid_next, int64_t n, int *err, ActiveBlocks ab_next, int *reset_count) {
    __shared__ float4 rows[P2G_WARP_THREADS / 32][32][P2G_ROW];
    __shared__ int keys[P2G_WARP_THREADS / 32][32];
    const int wid = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float xp[3] = {0.f, 0.f, 0.f}, Fp[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool pin = false;
    if (p < n) {
        load_xF(x, F, n, p, xp, Fp);
        pin = pinned && pinned[p];
    }
    pdl_wait();
    pdl_trigger();
    if (p == 0) *reset_count = 0;  // the grid update has consumed the current list
    P2GParticle q;
    q.valid = false;
    if (p < n) {
        float vn[3], Cn[9];
        g2p_update(P, grid_v, pin, xp, Fp, vn, Cn);
#pragma unroll
        for (int a = 0; a < 3; ++a) x[a * n + p] = xp[a];
#pragma unroll
        for (int k = 0; k < 9; ++k) F[k * n + p] = Fp[k];
        if (STORE_VC) {
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a * n + p] = vn[a];
#pragma unroll
            for (int k = 0; k < 9; ++k) C[k * n + p] = Cn[k];
        }
        bool fin = isfinite(xp[0]) && isfinite(xp[1]) && isfinite(xp[2]) && finite9(Fp);
        if (!fin) atomicOr(err, ERRBIT_NONFINITE);
        if (make_stencil(P, xp[0], xp[1], xp[2], q.s)) {
            if (!p2g_affine(P, Fp, Cn, q.A)) atomicOr(err, ERRBIT_INVERTED);
#pragma unroll
            for (int a = 0; a < 3; ++a) q.mv[a] = P.p_mass * vn[a];
            q.valid = true;
        } else {
            atomicOr(err, ERRBIT_DOMAIN);
        }
    }
    p2g_warp_scatter(P, q, grid_next, ab_next, rows[wid], keys[wid]);
}

// ------------------------------------------------ two particles per thread --
//
// k_g2p2g_pair: the body of k_g2p2g with two particles per thread on paired
// FP32 instructions (pair_warp, mpm_pair_warp.cuh).
// With OUT the output state goes to `out` (the recompute of a reverse segment).
template <int MAT, bool STORE_VC, bool VEC, bool OUT = false, bool KEYS = false>
__global__ void __launch_bounds__(PAIR_THREADS, PAIR_MIN_CTAS) k_g2p2g_pair(
    MpmParams P, float *__restrict__ x, float *__restrict__ v, float *__restrict__ C,
    float *__restrict__ F, const uint8_t *__restrict__ pinned, const float4 *__restrict__ grid_v,
    float4 *__restrict__ grid_next, int64_t n, int *err, ActiveBlocks ab_next, int *reset_count,
    PairOut out) {
    __shared__ PairWarpSmem smem[PAIR_WARPS];
    const int wid = threadIdx.x >> 5;
    const int64_t wq = ((int64_t)blockIdx.x * PAIR_THREADS + wid * 32) * 2;  // the warp's first particle
    pair_warp<MAT, STORE_VC, VEC, OUT, KEYS>(P, x, v, C, F, pinned, grid_v, grid_next, n, wq, n, err,
                                       ab_next,
                                       blockIdx.x == 0 && threadIdx.x == 0 ? reset_count : nullptr,
                                       smem[wid], out);
}

dw_status segment_recompute(MpmHandle *h, const dw_mpm_state *start, float *tape,
                            const uint8_t *pinned, const WindDev &wd, float t0, int n_substeps,
                            bool keep_grid, cudaStream_t s) {
    const int64_t n = start->n;
    if (n_substeps < 2 || n == 0) return DW_OK;
    auto slot = [&](int k) {  // state k (1 .. n_substeps - 1) in the tape
        dw_mpm_state st;
        float *b = tape + (size_t)(k - 1) * 24 * (size_t)n;
        st.x = b;
        st.v = b + 3 * n;
        st.C = b + 6 * n;
        st.F = b + 15 * n;
        st.n = n;
        return st;
    };
    dw_status st;
    {
        ProfScope ps(h, DW_K_P2G, s);
        st = launch_p2g(h->desc.p2g_mode, h->P, start->x, start->v, start->C, start->F, n,
                        h->grid_mp, h->err, active_blocks(h, 0), s);
    }
    if (st != DW_OK) return st;
    const unsigned pair_grid = grid_for(n, 2 * PAIR_THREADS);
    int L = 0;  // list consumed by the next grid update
    for (int k = 0; k + 1 < n_substeps; ++k) {
        const float t = fmaf((float)k, h->P.dt, t0);
        {
            ProfScope ps(h, DW_K_GRID, s);
            if (keep_grid)
                DW_CUDA(launch_pdl(k_grid_update_tape, GRID_CTAS, GRID_THREADS, s, h->P, wd, t,
                                   h->grid_mp, h->grid_v, active_blocks(h, L),
                                   h->gtape + (size_t)k * h->nblk * 64,
                                   h->gtape_list + (size_t)k * h->nblk, h->gtape_count + k));
            else
                DW_CUDA(launch_pdl(k_grid_update_active, GRID_CTAS, GRID_THREADS, s, h->P, wd, t,
                                   h->grid_mp, h->grid_v, 1, active_blocks(h, L)));
        }
        const dw_mpm_state in = k == 0 ? *start : slot(k), out = slot(k + 1);
        if (k + 2 < n_substeps) {  // state k + 1 is scattered for substep k + 1's grid
            ProfScope ps(h, DW_K_G2P2G, s);
            const bool vec = n % 4 == 0 &&
                             ((reinterpret_cast<uintptr_t>(in.x) | reinterpret_cast<uintptr_t>(in.F) |
                               reinterpret_cast<uintptr_t>(out.x) | reinterpret_cast<uintptr_t>(out.F)) %
                                  16 == 0);
            auto kern = h->P.material == DW_NEOHOOKEAN
                            ? (vec ? k_g2p2g_pair<DW_NEOHOOKEAN, false, true, true>
                                   : k_g2p2g_pair<DW_NEOHOOKEAN, false, false, true>)
                            : (vec ? k_g2p2g_pair<DW_FIXED_COROTATED, false, true, true>
                                   : k_g2p2g_pair<DW_FIXED_COROTATED, false, false, true>);
            DW_CUDA(launch_pdl(kern, pair_grid, PAIR_THREADS, s, h->P, in.x, in.v, in.C, in.F,
                               pinned, (const float4 *)h->grid_v, h->grid_mp, n, h->err,
                               active_blocks(h, 1 - L), h->block_count + L,
                               PairOut{out.x, out.v, out.C, out.F}));
            L = 1 - L;
        } else {
            ProfScope ps(h, DW_K_G2P, s);
            DW_CUDA(launch_pdl(k_g2p, grid_for(n, 128), 128, s, h->P, (const float *)in.x,
                               (const float *)in.F, pinned, (const float4 *)h->grid_v, out.x,
                               out.v, out.C, out.F, n, h->err, h->block_count + L));
        }
    }
    return DW_OK;
}

static dw_mpm_state view_of(float *base, int64_t n) {
    dw_mpm_state s;
    s.x = base;
    s.v = base + 3 * n;
    s.C = base + 6 * n;
    s.F = base + 15 * n;
    s.n = n;
    return s;
}

}  // namespace dw

using namespace dw;

extern "C" dw_status mpm_rollout(dw_mpm h, const dw_mpm_state *state, uint8_t *pinned,
                                 int32_t *ids, const dw_wind_field *wind, float t0,
                                 int32_t n_substeps, int32_t sort_every, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    dw_status st = check_state(h, state, "state");
    if (st != DW_OK) return st;
    DW_REQUIRE(n_substeps >= 0, "n_substeps must be >= 0");
    DW_REQUIRE(sort_every >= 0, "sort_every must be >= 0");
    DW_REQUIRE(sort_every == 0 || ids, "ids must be given when sort_every > 0");
    WindDev wd;
    st = wind_check(wind, &wd);
    if (st != DW_OK) return st;
    const int64_t n = state->n;
    if (n == 0 || n_substeps == 0) return DW_OK;
    cudaStream_t s = as_stream(stream);
    dw_mpm_state cur = *state, oth = view_of(h->roll_state, n);
    uint8_t *cur_pin = pinned, *oth_pin = pinned ? h->roll_pinned : nullptr;
    int32_t *cur_ids = ids, *oth_ids = h->roll_ids;
    const unsigned pgrid = grid_for(n, P2G_WARP_THREADS);
    // the fused kernel: two particles per thread (AUTO, PAIR) or one (the other strategies)
    const bool pair = h->desc.p2g_mode == DW_P2G_AUTO || h->desc.p2g_mode == DW_P2G_PAIR;
    const unsigned pair_grid = grid_for(n, 2 * PAIR_THREADS);
    int L = 0;  // active list consumed by the next grid update
    // the fused launch before a re-sort computes and counts the sort keys
    // (paired kernel; the counts are cleared by the sort before)
    auto resort = [&](bool with_vc, bool keys_ready) {
        dw_status r = sort_particles(h, &cur, &oth, cur_pin, oth_pin, cur_ids, oth_ids, s, with_vc,
                                     keys_ready, pair);
        std::swap(cur, oth);
        std::swap(cur_pin, oth_pin);
        std::swap(cur_ids, oth_ids);
        return r;
    };
    if (sort_every > 0) {
        st = resort(true, false);  // the input state's v and C feed the first P2G
        if (st != DW_OK) return st;
    }
    {
        ProfScope ps(h, DW_K_P2G, s);
        st = launch_p2g(h->desc.p2g_mode, h->P, cur.x, cur.v, cur.C, cur.F, n, h->grid_mp, h->err,
                        active_blocks(h, L), s);
    }
    if (st != DW_OK) return st;
    for (int k = 0; k < n_substeps; ++k) {
        const float t = fmaf((float)k, h->P.dt, t0);  // as the batched kernels
        {
            ProfScope ps(h, DW_K_GRID, s);
            DW_CUDA(launch_pdl(k_grid_update_active, GRID_CTAS, GRID_THREADS, s, h->P, wd, t,
                               h->grid_mp, h->grid_v, 1, active_blocks(h, L)));
        }
        if (k + 1 == n_substeps) {
            ProfScope ps(h, DW_K_G2P, s);
            DW_CUDA(launch_pdl(k_g2p, grid_for(n, 128), 128, s, h->P, (const float *)cur.x,
                               (const float *)cur.F, (const uint8_t *)cur_pin,
                               (const float4 *)h->grid_v, cur.x, cur.v, cur.C, cur.F, n, h->err,
                               h->block_count + L));
            break;
        }
        {
            ProfScope ps(h, DW_K_G2P2G, s);
            if (pair) {
                // vector paths: float2 pairs of x and F, 16-byte pieces of F (n a
                // multiple of 4, 16-byte aligned arrays)
                const bool pair_vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(cur.x) |
                                                        reinterpret_cast<uintptr_t>(cur.F)) % 16 == 0);
                const bool keys = sort_every > 0 && (k + 1) % sort_every == 0;
                const bool nh = h->P.material == DW_NEOHOOKEAN;
                auto kern = keys ? (nh ? (pair_vec ? k_g2p2g_pair<DW_NEOHOOKEAN, false, true, false, true>
                                                   : k_g2p2g_pair<DW_NEOHOOKEAN, false, false, false, true>)
                                       : (pair_vec ? k_g2p2g_pair<DW_FIXED_COROTATED, false, true, false, true>
                                                   : k_g2p2g_pair<DW_FIXED_COROTATED, false, false, false, true>))
                                 : (nh ? (pair_vec ? k_g2p2g_pair<DW_NEOHOOKEAN, false, true>
                                                   : k_g2p2g_pair<DW_NEOHOOKEAN, false, false>)
                                       : (pair_vec ? k_g2p2g_pair<DW_FIXED_COROTATED, false, true>
                                                   : k_g2p2g_pair<DW_FIXED_COROTATED, false, false>));
                PairOut po{};
                if (keys) {
                    po.keys = h->keys;
                    po.counts = h->counts;
                }
                DW_CUDA(launch_pdl(kern, pair_grid, PAIR_THREADS, s, h->P, cur.x, cur.v, cur.C,
                                   cur.F, (const uint8_t *)cur_pin, (const float4 *)h->grid_v,
                                   h->grid_mp, n, h->err, active_blocks(h, 1 - L),
                                   h->block_count + L, po));
            } else {
                DW_CUDA(launch_pdl(k_g2p2g<false>, pgrid, P2G_WARP_THREADS, s, h->P, cur.x,
                                   cur.v, cur.C, cur.F, (const uint8_t *)cur_pin,
                                   (const float4 *)h->grid_v, h->grid_mp, n, h->err,
                                   active_blocks(h, 1 - L), h->block_count + L));
            }
        }
        L = 1 - L;
        // Re-sort between two fused launches: the P2G of substep k + 1 has
        // already run (in the old order; the grid does not depend on it), so
        // the sorted order serves the G2P of k + 1 and every P2G after it.
        // v and C are not kept between fused launches, so none is lost.
        if (sort_every > 0 && (k + 1) % sort_every == 0) {
            st = resort(false, pair);
            if (st != DW_OK) return st;
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

// Internal view of an MPM handle shared by the MPM translation units: the
// workspace layout, launch instrumentation and the kernels and host helpers
// one unit launches from another.
#pragma once

#include <vector>

#include "mpm_g2p.cuh"
#include "mpm_grid.cuh"
#include "mpm_math.cuh"
#include "mpm_p2g.cuh"
#include "wind.cuh"

namespace dw {

struct MpmHandle {
    dw_mpm_desc desc;
    MpmParams P;
    int64_t n_nodes;
    float4 *grid_mp = nullptr;   // (m, p) after P2G; zero between calls
    float4 *grid_v = nullptr;    // (v, m) after the grid update
    float4 *grid_bv = nullptr;   // (0, dL/dv_i) during the adjoint; zero between calls
    float4 *grid_bmp = nullptr;  // (dL/dm_i, dL/dp_i) during the adjoint
    float *pscratch = nullptr;   // [12][max_particles]: partial dL/dx (3), dL/dF (9)
    int *err = nullptr;          // device status bits
    // active 4^3 blocks of the grid (built by P2G, consumed by the grid update)
    int64_t nblk = 0;            // nb^3
    int *block_flag = nullptr;   // [nblk]
    int *block_list = nullptr;   // [2][nblk]: two lists so a fused kernel can fill one
    int *block_count = nullptr;  // [2]      while the grid update consumes the other
    // grid tape of a segment adjoint's recompute: per recomputed substep the
    // consumed list and each listed node's (m, p) (nblk entries of 64 nodes)
    float4 *gtape = nullptr;
    int *gtape_list = nullptr, *gtape_count = nullptr;
    int gtape_slots = 0;
    int gtape_refused = 0;       // slots a failed or oversized allocation was refused for
    // rollout workspace: the second state buffer of the sort ping-pong
    float *roll_state = nullptr;     // [24][max_particles]
    uint8_t *roll_pinned = nullptr;  // [max_particles]
    int32_t *roll_ids = nullptr;     // [max_particles]
    // sort workspace
    int nb = 0;                  // 4^3 blocks per axis
    int64_t n_keys = 0;
    int *keys = nullptr;         // [max_particles]
    int *counts = nullptr;       // [n_keys + 1]
    int *scan_tmp = nullptr;     // block sums for the exclusive scan
    int64_t scan_tmp_len = 0;
    // instrumentation: event pairs around kernel launches
    std::vector<cudaEvent_t> ev_start, ev_stop;
    std::vector<int> ev_kernel;
    int prof_used = 0;
};

// Brackets one kernel launch with events when profiling is enabled.
struct ProfScope {
    MpmHandle *h;
    cudaStream_t s;
    int slot = -1;
    ProfScope(MpmHandle *h_, int kid, cudaStream_t s_) : h(h_), s(s_) {
        if (h->prof_used < (int)h->ev_start.size()) {
            slot = h->prof_used++;
            h->ev_kernel[slot] = kid;
            cudaEventRecord(h->ev_start[slot], s);
        }
    }
    ~ProfScope() {
        if (slot >= 0) cudaEventRecord(h->ev_stop[slot], s);
    }
};

inline void profile_free(MpmHandle *h) {
    for (auto e : h->ev_start) cudaEventDestroy(e);
    for (auto e : h->ev_stop) cudaEventDestroy(e);
    h->ev_start.clear();
    h->ev_stop.clear();
    h->ev_kernel.clear();
    h->prof_used = 0;
}

inline MpmParams params_of(const dw_mpm_desc &d) {
    MpmParams P;
    P.N = d.n_grid;
    P.dx = 1.0f / (float)d.n_grid;
    P.inv_dx = (float)d.n_grid;
    P.dt = d.dt;
    P.D = 4.0f * (float)d.n_grid * (float)d.n_grid;
    P.gx = d.gravity[0];
    P.gy = d.gravity[1];
    P.gz = d.gravity[2];
    P.band = d.bc_band;
    P.material = d.material;
    double E = d.E, nu = d.nu;
    P.mu = (float)(E / (2.0 * (1.0 + nu)));                       // Eq. young_poisson
    P.lam = (float)(E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
    P.E = d.E;
    P.p_mass = d.p_mass;
    P.p_vol = d.p_vol;
    P.kappa = d.dt * d.p_vol * P.D;
    return P;
}

inline void fill_params(MpmHandle *h) { h->P = params_of(h->desc); }

constexpr int GRID_THREADS = 256;  // four 4^3 blocks per CTA iteration
constexpr int GRID_CTAS = 4 * 152;

inline ActiveBlocks active_blocks(MpmHandle *h, int which = 0) {
    return ActiveBlocks{h->block_flag, h->block_list + (size_t)which * h->nblk,
                        h->block_count + which, h->nb, 0};
}

// kernels of mpm.cu launched from other units
__global__ void k_grid_update_active(MpmParams P, WindDev wind, float t,
                                     float4 *__restrict__ grid_mp, float4 *__restrict__ grid_v,
                                     int clear, ActiveBlocks ab);
__global__ void k_g2p(MpmParams P, const float *x, const float *F,
                      const uint8_t *__restrict__ pinned, const float4 *__restrict__ grid_v,
                      float *xo, float *vo, float *Co, float *Fo, int64_t n, int *err,
                      int *reset_count);
__global__ void k_grid_update_tape(MpmParams P, WindDev wind, float t, float4 *__restrict__ grid_mp,
                                   float4 *__restrict__ grid_v, ActiveBlocks ab,
                                   float4 *__restrict__ gtape, int *__restrict__ gtape_list,
                                   int *__restrict__ gtape_count);

// The recompute of a segment adjoint (mpm_rollout.cu): states 1 .. n_substeps
// - 1 from `start` into the tape slots, as one fused chain (the P2G of the
// start state, then per substep the grid update, kept in grid tape slot k
// when `keep_grid`, and the paired G2P/P2G kernel writing state k + 1 to its
// slot). For p2g modes AUTO and PAIR.
dw_status segment_recompute(MpmHandle *h, const dw_mpm_state *start, float *tape,
                            const uint8_t *pinned, const WindDev &wd, float t0, int n_substeps,
                            bool keep_grid, cudaStream_t s);

// particle sort (mpm.cu): counting sort by cell key, keys already counted
constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 8;                         // consecutive elements per scan thread
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;    // elements per scan block
__global__ void k_sort_move(const int *__restrict__ keys, int64_t n, int *__restrict__ offsets,
                            const float *__restrict__ x, const float *__restrict__ v,
                            const float *__restrict__ C, const float *__restrict__ F,
                            const uint8_t *__restrict__ pin_in, const int *__restrict__ ids_in,
                            float *__restrict__ xo, float *__restrict__ vo, float *__restrict__ Co,
                            float *__restrict__ Fo, uint8_t *__restrict__ pin_out,
                            int *__restrict__ ids_out);
// In-place exclusive prefix sum of data[0, len); tmp holds at least
// len / SCAN_BLOCK + 1 ints.
dw_status exclusive_scan(int *data, int64_t len, int *tmp, int64_t tmp_len, cudaStream_t st);

// host helpers of mpm.cu
dw_status validate_desc(const dw_mpm_desc *desc);
dw_status check_state(const MpmHandle *h, const dw_mpm_state *s, const char *name);
// with_vc = false leaves v and C of `out` unwritten (a rollout between fused
// launches, where v and C are not kept). keys_ready: h->keys and h->counts
// already hold the keys of `in` and their counts (the fused launch before
// the sort wrote them). clear_after: the counts are cleared at the end, for
// a fused launch that counts the next sort's keys.
dw_status sort_particles(MpmHandle *h, const dw_mpm_state *in, const dw_mpm_state *out,
                         const uint8_t *pinned_in, uint8_t *pinned_out, const int32_t *ids_in,
                         int32_t *ids_out, cudaStream_t s, bool with_vc = true,
                         bool keys_ready = false, bool clear_after = false);

}  // namespace dw

struct dw_mpm_s : dw::MpmHandle {};

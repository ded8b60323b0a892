// Device helpers of the grid update and the particle sort that several MPM
// translation units share: the sticky wall band, the per-node grid update,
// the node of a thread within an active 4^3 block, and the cell sort key.
#pragma once

#include "mpm_math.cuh"
#include "wind.cuh"

namespace dw {

__device__ __forceinline__ bool sticky_node(const MpmParams &P, int i, int j, int k) {
    return i < P.band || j < P.band || k < P.band || i > P.N - 1 - P.band ||
           j > P.N - 1 - P.band || k > P.N - 1 - P.band;
}

// Grid update of one node: v_i = p_i / m_i + dt (g + a_w(x_i, t)), zero in the
// sticky band and at empty nodes; (v, m) goes to grid_v.
__device__ __forceinline__ void grid_node_update(const MpmParams &P, const WindDev &wind, float t,
                                                 int64_t node, int i, int j, int k,
                                                 float4 *__restrict__ grid_mp,
                                                 float4 *__restrict__ grid_v, int clear) {
    float4 mp = grid_mp[node];
    // the wind taps are loaded together with (m, p), not after the test on m
    const float3 a = wind_sample_dev(wind, i * P.dx, j * P.dx, k * P.dx, t);
    float4 out = make_float4(0.f, 0.f, 0.f, mp.x);
    if (mp.x > 0.0f && !sticky_node(P, i, j, k)) {
        float inv_m = 1.0f / mp.x;
        out.x = mp.y * inv_m + P.dt * (P.gx + a.x);
        out.y = mp.z * inv_m + P.dt * (P.gy + a.y);
        out.z = mp.w * inv_m + P.dt * (P.gz + a.z);
    }
    grid_v[node] = out;
    if (clear) grid_mp[node] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Node (i, j, k) of thread t within active block b; false outside the grid.
__device__ __forceinline__ bool active_node(const MpmParams &P, int nb, int b, int t, int &i,
                                            int &j, int &k) {
    int bx = b % nb, by = (b / nb) % nb, bz = b / (nb * nb);
    i = bx * 4 + (t & 3);
    j = by * 4 + ((t >> 2) & 3);
    k = bz * 4 + (t >> 4);
    return i < P.N && j < P.N && k < P.N;
}

// Sort key of a particle: its base cell (floor(x/dx - 0.5), clamped to the
// grid) as 64 * (4^3 block index) + (cell within the block), so that particles
// of one block are contiguous and, within it, grouped by cell.
__device__ __forceinline__ int cell_key(const MpmParams &P, int nb, float px, float py, float pz) {
    float xs[3] = {px * P.inv_dx, py * P.inv_dx, pz * P.inv_dx};
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float b = floorf(xs[a] - 0.5f);
        b = fminf(fmaxf(b, 0.0f), (float)(P.N - 1));  // NaN -> 0
        c[a] = (int)b;
    }
    int blk = ((c[2] >> 2) * nb + (c[1] >> 2)) * nb + (c[0] >> 2);
    int loc = ((c[2] & 3) * 4 + (c[1] & 3)) * 4 + (c[0] & 3);
    return blk * 64 + loc;
}

}  // namespace dw

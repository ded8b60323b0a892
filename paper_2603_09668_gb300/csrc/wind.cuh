// Device-side sampling of the wind force field a_w(x, t): trilinear in space
// over a node-centred nf^3 grid on the unit cube (node j at j / (nf - 1)),
// linear in time between keyframes at k * t_total / (n_frames - 1), clamped
// (the force property of the wind grid field, Sec. 3 and Sec. 3.3).
#pragma once

#include "common.cuh"

namespace dw {

struct WindDev {
    const float *values;  // [n_frames][nf][nf][nf][3], x fastest
    int nf;
    int n_frames;
    float t_total;
};

// The up-to-16 (frame, corner) taps of one sample: element offsets of the
// first component of each tap and its weight.
struct WindTaps {
    int base;       // node index of corner (i0, j0, k0) in frame k0
    int sx, sy, sz; // node strides to the +1 corner per axis (0 if nf == 1)
    int st;         // node stride to the next frame (0 if n_frames == 1)
    int i0[3];      // corner (i0, j0, k0) of the spatial cell
    int kf;         // first keyframe
    float fr[3];
    float ft;
};

__device__ __forceinline__ WindTaps wind_taps(const WindDev &w, float px, float py, float pz,
                                              float t) {
    WindTaps tp;
    const int nf = w.nf;
    float p[3] = {px, py, pz};
    int i0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float q = fminf(fmaxf(p[a], 0.0f), 1.0f);
        if (nf < 2) {
            i0[a] = 0;
            tp.fr[a] = 0.0f;
        } else {
            float s = q * (float)(nf - 1);
            int i = (int)floorf(s);
            i = min(max(i, 0), nf - 2);
            i0[a] = i;
            tp.fr[a] = s - (float)i;
        }
    }
    int k0 = 0;
    tp.ft = 0.0f;
    if (w.n_frames > 1) {
        float tc = fminf(fmaxf(t, 0.0f), w.t_total);
        float s = tc / w.t_total * (float)(w.n_frames - 1);
        k0 = min(max((int)floorf(s), 0), w.n_frames - 2);
        tp.ft = s - (float)k0;
    }
    tp.base = ((k0 * nf + i0[2]) * nf + i0[1]) * nf + i0[0];
#pragma unroll
    for (int a = 0; a < 3; ++a) tp.i0[a] = i0[a];
    tp.kf = k0;
    tp.sx = nf > 1 ? 1 : 0;
    tp.sy = nf > 1 ? nf : 0;
    tp.sz = nf > 1 ? nf * nf : 0;
    tp.st = w.n_frames > 1 ? nf * nf * nf : 0;
    return tp;
}

__device__ __forceinline__ float3 wind_sample_dev(const WindDev &w, float px, float py, float pz,
                                                  float t) {
    WindTaps tp = wind_taps(w, px, py, pz, t);
    float3 acc = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int dk = 0; dk < 2; ++dk) {
        float wt_t = dk ? tp.ft : 1.0f - tp.ft;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
            float wt = wt_t * (cx ? tp.fr[0] : 1.0f - tp.fr[0]) *
                       (cy ? tp.fr[1] : 1.0f - tp.fr[1]) * (cz ? tp.fr[2] : 1.0f - tp.fr[2]);
            // every tap lies inside the field (wind_taps clamps the corner),
            // so all 48 loads are issued without a branch; a zero weight adds
            // a signed zero, which leaves the (never negative-zero) sum as it is
            int node = tp.base + dk * tp.st + cx * tp.sx + cy * tp.sy + cz * tp.sz;
            const float *v = w.values + 3 * (size_t)node;
            acc.x += wt * __ldg(v + 0);
            acc.y += wt * __ldg(v + 1);
            acc.z += wt * __ldg(v + 2);
        }
    }
    return acc;
}

// g_values += taps^T g (atomic scatter into the field gradient).
__device__ __forceinline__ void wind_sample_adjoint_dev(const WindDev &w, float px, float py,
                                                        float pz, float t, float3 g,
                                                        float *g_values) {
    WindTaps tp = wind_taps(w, px, py, pz, t);
#pragma unroll
    for (int dk = 0; dk < 2; ++dk) {
        float wt_t = dk ? tp.ft : 1.0f - tp.ft;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
            float wt = wt_t * (cx ? tp.fr[0] : 1.0f - tp.fr[0]) *
                       (cy ? tp.fr[1] : 1.0f - tp.fr[1]) * (cz ? tp.fr[2] : 1.0f - tp.fr[2]);
            if (wt == 0.0f) continue;
            int node = tp.base + dk * tp.st + cx * tp.sx + cy * tp.sy + cz * tp.sz;
            float *gv = g_values + 3 * (size_t)node;
            atomicAdd(gv + 0, wt * g.x);
            atomicAdd(gv + 1, wt * g.y);
            atomicAdd(gv + 2, wt * g.z);
        }
    }
}

// Per-warp scratch of wind_sample_adjoint_warp: (dL/d values) of a
// 3 x 3 x 3 box of wind nodes in two keyframes.
constexpr int WIND_BOX = 2 * 27 * 3;

// Whether wind gradients scattered from the nodes of an n_grid^3 grid are
// worth aggregating per warp: a wind cell spans at least 4 grid cells, so
// thousands of nodes add into the same few wind nodes.
__host__ __device__ __forceinline__ bool wind_scatter_coarse(int n_grid, int nf) {
    return n_grid >= 4 * (nf - 1);
}

// wind_sample_adjoint_dev for the samples of a whole warp, called by all 32
// lanes together with the same field, time and `box` (lanes with active =
// false add nothing). With box set and the warp's samples in spatial cells
// at most one apart per axis (the nodes of one 4^3 grid block against a
// coarser wind grid), their taps touch one 3 x 3 x 3 box of wind nodes: the
// lanes add into the warp's shared-memory copy of that box (sbox, WIND_BOX
// floats), then each touched entry goes to g_values with one atomic, instead
// of every lane issuing its 48 atomics onto the same few addresses.
// Otherwise each lane scatters as wind_sample_adjoint_dev does.
__device__ __forceinline__ void wind_sample_adjoint_warp(const WindDev &w, bool box, bool active,
                                                         float px, float py, float pz, float t,
                                                         float3 g, float *g_values, float *sbox) {
    if (!box) {
        if (active) wind_sample_adjoint_dev(w, px, py, pz, t, g, g_values);
        return;
    }
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const WindTaps tp = wind_taps(w, px, py, pz, t);
    if (!__any_sync(full, active)) return;
    int mn[3], mx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        mn[a] = __reduce_min_sync(full, active ? tp.i0[a] : 0x7fffffff);
        mx[a] = __reduce_max_sync(full, active ? tp.i0[a] : -1);
    }
    const bool boxed = mx[0] - mn[0] <= 1 && mx[1] - mn[1] <= 1 && mx[2] - mn[2] <= 1;
    if (!boxed) {
        if (active) wind_sample_adjoint_dev(w, px, py, pz, t, g, g_values);
        return;
    }
    for (int e = lane; e < WIND_BOX; e += 32) sbox[e] = 0.0f;
    __syncwarp();
    if (active) {
        const int lx = tp.i0[0] - mn[0], ly = tp.i0[1] - mn[1], lz = tp.i0[2] - mn[2];
        // lane L starts at tap L mod 16, so that lanes of one cell add into
        // different entries at each step (shared atomics on one address
        // serialize)
        for (int s = 0; s < 16; ++s) {
            const int tap = (s + lane) & 15, dk = tap >> 3;
            const int cx = tap & 1, cy = (tap >> 1) & 1, cz = (tap >> 2) & 1;
            const float wt = (dk ? tp.ft : 1.0f - tp.ft) * (cx ? tp.fr[0] : 1.0f - tp.fr[0]) *
                             (cy ? tp.fr[1] : 1.0f - tp.fr[1]) * (cz ? tp.fr[2] : 1.0f - tp.fr[2]);
            if (wt == 0.0f) continue;
            float *b = sbox + 3 * (dk * 27 + ((lz + cz) * 3 + (ly + cy)) * 3 + (lx + cx));
            atomicAdd(b + 0, wt * g.x);
            atomicAdd(b + 1, wt * g.y);
            atomicAdd(b + 2, wt * g.z);
        }
    }
    __syncwarp();
    const int nf = w.nf;
    for (int e = lane; e < WIND_BOX; e += 32) {
        const float v = sbox[e];
        if (v == 0.0f) continue;  // untouched (entries outside the grid are never touched)
        const int comp = e % 3, r = e / 3, dk = r / 27, q = r % 27;
        const int gx = mn[0] + q % 3, gy = mn[1] + (q / 3) % 3, gz = mn[2] + q / 9;
        const int node = (((tp.kf + dk) * nf + gz) * nf + gy) * nf + gx;
        atomicAdd(g_values + 3 * (size_t)node + comp, v);
    }
    __syncwarp();
}

// Host-side validation of a dw_wind_field; fills the device view.
dw_status wind_check(const dw_wind_field *w, WindDev *out);

}  // namespace dw

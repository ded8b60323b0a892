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
            if (wt == 0.0f) continue;
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

// Host-side validation of a dw_wind_field; fills the device view.
dw_status wind_check(const dw_wind_field *w, WindDev *out);

}  // namespace dw

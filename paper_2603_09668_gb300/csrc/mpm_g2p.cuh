// G2P of one particle (Eq. G2P, Eq. deformation_update):
// v_p = sum_i w_ip v_i, C_p = (4/dx^2) sum_i w_ip v_i (x_i - x_p)^T,
// x_p += dt v_p, F_p <- (I + dt C_p) F_p; pinned particles keep v = C = 0.
#pragma once

#include "mpm_math.cuh"

namespace dw {

// Updates x and F in place and returns v and C. Returns false, leaving x and
// F unchanged and v = C = 0, when the stencil leaves the grid.
__device__ __forceinline__ bool g2p_update(const MpmParams &P, const float4 *__restrict__ grid_v,
                                           bool pinned, float x[3], float F[9], float vn[3],
                                           float Cn[9]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) vn[a] = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) Cn[k] = 0.0f;
    Stencil s;
    if (!make_stencil(P, x[0], x[1], x[2], s)) return false;
    const int N = P.N;
    const int64_t base = ((int64_t)s.base[2] * N + s.base[1]) * N + s.base[0];
#pragma unroll
    for (int ok = 0; ok < 3; ++ok)
#pragma unroll
        for (int oj = 0; oj < 3; ++oj)
#pragma unroll
            for (int oi = 0; oi < 3; ++oi) {
                float W = s.w[0][oi] * s.w[1][oj] * s.w[2][ok];
                float d0 = ((float)oi - s.fx[0]) * P.dx, d1 = ((float)oj - s.fx[1]) * P.dx,
                      d2 = ((float)ok - s.fx[2]) * P.dx;
                float4 gv = grid_v[base + ((int64_t)ok * N + oj) * N + oi];
                float wv[3] = {W * gv.x, W * gv.y, W * gv.z};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    vn[a] += wv[a];
                    Cn[3 * a + 0] += wv[a] * d0;
                    Cn[3 * a + 1] += wv[a] * d1;
                    Cn[3 * a + 2] += wv[a] * d2;
                }
            }
#pragma unroll
    for (int k = 0; k < 9; ++k) Cn[k] *= P.D;
    if (pinned) {
#pragma unroll
        for (int a = 0; a < 3; ++a) vn[a] = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) Cn[k] = 0.0f;
    }
    float M[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) M[k] = P.dt * Cn[k];
    M[0] += 1.0f;
    M[4] += 1.0f;
    M[8] += 1.0f;
    float Fn[9];
    mul3(M, F, Fn);
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = Fn[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] += P.dt * vn[a];
    return true;
}

}  // namespace dw

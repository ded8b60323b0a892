// G2P of one particle (Eq. G2P, Eq. deformation_update):
// v_p = sum_i w_ip v_i, C_p = (4/dx^2) sum_i w_ip v_i (x_i - x_p)^T,
// x_p += dt v_p, F_p <- (I + dt C_p) F_p; pinned particles keep v = C = 0.
#pragma once

#include "mpm_math.cuh"

namespace dw {

// Grid velocity load: through L2 only (CG) where the grid was written by
// another CTA earlier in the same kernel, a plain load otherwise.
template <bool CG>
__device__ __forceinline__ float4 load_grid(const float4 *p) {
    if (CG) return __ldcg(p);
    return *p;
}

// Updates x and F in place and returns v and C. Returns false, leaving x and
// F unchanged and v = C = 0, when the stencil leaves the grid.
template <bool CG = false>
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
    // Tensor-product evaluation: for each (oj, ok) line of three nodes along x,
    // a = sum_oi wx v_i and bx = sum_oi oi wx v_i; then v = sum wyz a and
    // S_b = sum_o W o_b v_i per axis b, so that C = (4/dx^2) dx (S - v fx^T).
    float S[3][3];  // S[b][c] = sum_o W o_b v_c
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) S[b][c] = 0.0f;
    const float wx0 = s.w[0][0], wx1 = s.w[0][1], wx2 = s.w[0][2], wx2d = 2.0f * s.w[0][2];
#pragma unroll
    for (int ok = 0; ok < 3; ++ok)
#pragma unroll
        for (int oj = 0; oj < 3; ++oj) {
            const float wyz = s.w[1][oj] * s.w[2][ok];
            const int64_t row = base + ((int64_t)ok * N + oj) * N;
            const float4 g0 = load_grid<CG>(grid_v + row), g1 = load_grid<CG>(grid_v + row + 1),
                         g2 = load_grid<CG>(grid_v + row + 2);
            const float a[3] = {wx0 * g0.x + wx1 * g1.x + wx2 * g2.x,
                                wx0 * g0.y + wx1 * g1.y + wx2 * g2.y,
                                wx0 * g0.z + wx1 * g1.z + wx2 * g2.z};
            const float bx[3] = {wx1 * g1.x + wx2d * g2.x, wx1 * g1.y + wx2d * g2.y,
                                 wx1 * g1.z + wx2d * g2.z};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                vn[c] += wyz * a[c];
                S[0][c] += wyz * bx[c];
                if (oj == 1) S[1][c] += wyz * a[c];
                if (oj == 2) S[1][c] += (2.0f * wyz) * a[c];
                if (ok == 1) S[2][c] += wyz * a[c];
                if (ok == 2) S[2][c] += (2.0f * wyz) * a[c];
            }
        }
    const float Ddx = P.D * P.dx;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) Cn[3 * c + b] = Ddx * (S[b][c] - vn[c] * s.fx[b]);
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

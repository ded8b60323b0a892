// Reverse mode of one MLS-MPM substep (Eq. simulation_mpm), per particle and
// per node, shared by the single-scene adjoint (mpm.cu) and the batched one
// (mpm_batch.cu).
//
// Reverse G2P: the forward G2P maps the grid velocities v_i to v_p, C_p and
// then x_p, F_p (Eq. G2P, Eq. deformation_update); its adjoint gives
// dL/dv_i (scattered, in the form of a P2G value), the partial dL/dx_p of the
// weights and dL/dF_p. Reverse grid update: dL/dm_i, dL/dp_i and the wind
// gradient. Reverse P2G: gathers (dL/dm_i, dL/dp_i) back to the particle
// (dL/dx_p, dL/dv_p, dL/dC_p, dL/dF_p through the stress, dL/dE).
#pragma once

#include "mpm_grid.cuh"
#include "mpm_p2g.cuh"
#include "wind.cuh"

namespace dw {

__device__ __forceinline__ void weight_grad(const MpmParams &P, const Stencil &s, int oi, int oj,
                                            int ok, float g[3]) {
    float wx = s.w[0][oi], wy = s.w[1][oj], wz = s.w[2][ok];
    g[0] = s.dw[0][oi] * wy * wz * P.inv_dx;
    g[1] = wx * s.dw[1][oj] * wz * P.inv_dx;
    g[2] = wx * wy * s.dw[2][ok] * P.inv_dx;
}

// Reverse G2P of one particle at input position xp, input F Fp. bxo, bvo,
// bCo, bFo: dL/d(output x, v, C, F). Writes q (the node value
// W_ip (bv_p + D bC_p (x_i - x_p)), i.e. a P2G value with m v -> bv and
// A -> D bC, to be scattered with the mass channel off), bx = partial dL/dx_p
// and bFin = dL/dF_p through the F update. A particle outside the domain
// gets bx = bFin = 0 and q.valid = false. Cout (or NULL): the C array of the
// substep's output state (row stride `stride`, particle p), when a recompute
// kept it; then C' is read instead of gathered again from the grid.
__device__ __forceinline__ void rev_g2p_particle(const MpmParams &P, const float xp[3],
                                                 const float Fp[9], bool pin,
                                                 const float4 *__restrict__ grid_v,
                                                 const float bxo[3], const float bvo[3],
                                                 const float bCo[9], const float bFo[9],
                                                 P2GParticle &q, float bx[3], float bFin[9],
                                                 const float *__restrict__ Cout = nullptr,
                                                 int64_t stride = 0, int64_t p = 0) {
    q.valid = false;
    Stencil s;
    if (!make_stencil(P, xp[0], xp[1], xp[2], s)) {
#pragma unroll
        for (int a = 0; a < 3; ++a) bx[a] = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) bFin[k] = 0.0f;
        return;
    }
    const int N = P.N;
    // C' of the output state (v' is not needed: its adjoint only uses the
    // weights): kept by the recompute, else gathered from the grid again
    float Cn[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (Cout && !pin) {
#pragma unroll
        for (int k = 0; k < 9; ++k) Cn[k] = Cout[k * stride + p];
    } else if (!pin) {
#pragma unroll
        for (int oi = 0; oi < 3; ++oi)
#pragma unroll
            for (int oj = 0; oj < 3; ++oj)
#pragma unroll
                for (int ok = 0; ok < 3; ++ok) {
                    float W = s.w[0][oi] * s.w[1][oj] * s.w[2][ok];
                    float d[3] = {((float)oi - s.fx[0]) * P.dx, ((float)oj - s.fx[1]) * P.dx,
                                  ((float)ok - s.fx[2]) * P.dx};
                    int64_t id = ((int64_t)(s.base[2] + ok) * N + (s.base[1] + oj)) * N + (s.base[0] + oi);
                    float4 gv = grid_v[id];
                    float wv[3] = {W * gv.x, W * gv.y, W * gv.z};
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) Cn[3 * a + b] += wv[a] * d[b];
                }
#pragma unroll
        for (int k = 0; k < 9; ++k) Cn[k] *= P.D;
    }
    // F' = (I + dt C') F  ->  bF_in = (I + dt C')^T bF', bC' += dt bF' F^T
    float M[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) M[k] = P.dt * Cn[k];
    M[0] += 1.0f;
    M[4] += 1.0f;
    M[8] += 1.0f;
    float bFoFt[9];
    mul3_atb(M, bFo, bFin);
    mul3_abt(bFo, Fp, bFoFt);
    float bC[9], bv[3];
#pragma unroll
    for (int k = 0; k < 9; ++k) bC[k] = bCo[k] + P.dt * bFoFt[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) bv[a] = bvo[a] + P.dt * bxo[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) bx[a] = bxo[a];
    if (pin) return;
#pragma unroll
    for (int oi = 0; oi < 3; ++oi)
#pragma unroll
        for (int oj = 0; oj < 3; ++oj)
#pragma unroll
            for (int ok = 0; ok < 3; ++ok) {
                float W = s.w[0][oi] * s.w[1][oj] * s.w[2][ok];
                float d[3] = {((float)oi - s.fx[0]) * P.dx, ((float)oj - s.fx[1]) * P.dx,
                              ((float)ok - s.fx[2]) * P.dx};
                int64_t id = ((int64_t)(s.base[2] + ok) * N + (s.base[1] + oj)) * N + (s.base[0] + oi);
                float4 gv = grid_v[id];
                float vi[3] = {gv.x, gv.y, gv.z};
                float Cd[3], CtV[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Cd[a] = bC[3 * a] * d[0] + bC[3 * a + 1] * d[1] + bC[3 * a + 2] * d[2];
                    CtV[a] = bC[a] * vi[0] + bC[3 + a] * vi[1] + bC[6 + a] * vi[2];
                }
                float bW = 0.0f;
#pragma unroll
                for (int a = 0; a < 3; ++a) bW += vi[a] * (bv[a] + P.D * Cd[a]);
                float gW[3];
                weight_grad(P, s, oi, oj, ok, gW);
#pragma unroll
                for (int a = 0; a < 3; ++a) bx[a] += -P.D * W * CtV[a] + bW * gW[a];
            }
    q.s = s;
#pragma unroll
    for (int a = 0; a < 3; ++a) q.mv[a] = bv[a];
#pragma unroll
    for (int k = 0; k < 9; ++k) q.A[k] = P.D * bC[k];
    q.valid = true;
}

// Reverse grid update of one node: (dL/dm_i, dL/dp_i) into grid_bmp, and
// clearing of grid_mp and grid_bv for the next call. Returns whether the node
// took part in the grid update (m_i > 0, outside the sticky band); then gw is
// dt dL/dv_i, the cotangent of the wind force sampled at the node, for
// wind_sample_adjoint_warp.
__device__ __forceinline__ bool rev_grid_node(const MpmParams &P, int64_t node, int i, int j,
                                              int k, float4 *__restrict__ grid_mp,
                                              float4 *__restrict__ grid_bv,
                                              float4 *__restrict__ grid_bmp, float3 &gw) {
    float4 mp = grid_mp[node];
    float4 bmp = make_float4(0.f, 0.f, 0.f, 0.f);
    bool live = false;
    gw = make_float3(0.f, 0.f, 0.f);
    if (mp.x > 0.0f && !sticky_node(P, i, j, k)) {
        const float4 b4 = grid_bv[node];  // (0, dL/dv_i)
        const float b[3] = {b4.y, b4.z, b4.w};
        float inv_m = 1.0f / mp.x;
        bmp.y = b[0] * inv_m;
        bmp.z = b[1] * inv_m;
        bmp.w = b[2] * inv_m;
        bmp.x = -(mp.y * b[0] + mp.z * b[1] + mp.w * b[2]) * inv_m * inv_m;
        gw = make_float3(P.dt * b[0], P.dt * b[1], P.dt * b[2]);
        live = true;
    }
    grid_mp[node] = make_float4(0.f, 0.f, 0.f, 0.f);
    grid_bv[node] = make_float4(0.f, 0.f, 0.f, 0.f);
    grid_bmp[node] = bmp;
    return live;
}

// Reverse P2G of one particle at input state (xp, vp, Cp, Fp), gathering
// grid_bmp = (dL/dm_i, dL/dp_i). bx and bF enter with the reverse-G2P
// partials and leave as the complete dL/dx_p, dL/dF_p; writes bvp = dL/dv_p,
// bC = dL/dC_p and gE = this particle's dL/dE.
__device__ __forceinline__ void rev_p2g_particle(const MpmParams &P, const float xp[3],
                                                 const float vp[3], const float Cp[9],
                                                 const float Fp[9],
                                                 const float4 *__restrict__ grid_bmp, float bx[3],
                                                 float bF[9], float bvp[3], float bC[9],
                                                 float &gE) {
    Stencil s;
    float bA[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) bvp[a] = 0.0f;
    gE = 0.0f;
    if (make_stencil(P, xp[0], xp[1], xp[2], s)) {
        float Pk[9], PFt[9], A[9];
        stress_P(P, Fp, Pk);
        mul3_abt(Pk, Fp, PFt);
#pragma unroll
        for (int k = 0; k < 9; ++k) A[k] = -P.kappa * PFt[k] + P.p_mass * Cp[k];
        const int N = P.N;
#pragma unroll
        for (int oi = 0; oi < 3; ++oi)
#pragma unroll
            for (int oj = 0; oj < 3; ++oj)
#pragma unroll
                for (int ok = 0; ok < 3; ++ok) {
                    float W = s.w[0][oi] * s.w[1][oj] * s.w[2][ok];
                    float d[3] = {((float)oi - s.fx[0]) * P.dx, ((float)oj - s.fx[1]) * P.dx,
                                  ((float)ok - s.fx[2]) * P.dx};
                    int64_t id = ((int64_t)(s.base[2] + ok) * N + (s.base[1] + oj)) * N + (s.base[0] + oi);
                    float4 g = grid_bmp[id];
                    float bp[3] = {g.y, g.z, g.w};
                    float bW = P.p_mass * g.x;
                    float AtB[3] = {0.f, 0.f, 0.f};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float mom = P.p_mass * vp[c] + A[3 * c] * d[0] + A[3 * c + 1] * d[1] + A[3 * c + 2] * d[2];
                        bW += bp[c] * mom;
                        bvp[c] += W * P.p_mass * bp[c];
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            bA[3 * c + b] += W * bp[c] * d[b];
                            AtB[b] += A[3 * c + b] * bp[c];
                        }
                    }
                    float gW[3];
                    weight_grad(P, s, oi, oj, ok, gW);
#pragma unroll
                    for (int a = 0; a < 3; ++a) bx[a] += -W * AtB[a] + bW * gW[a];
                }
        // A = -kappa P F^T + m C
        float bAF[9], bAtP[9], bP[9];
        mul3(bA, Fp, bAF);
        mul3_atb(bA, Pk, bAtP);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            bP[k] = -P.kappa * bAF[k];
            bF[k] += -P.kappa * bAtP[k];
        }
        stress_P_adjoint(P, Fp, bP, bF);
        float pp = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) pp += bP[k] * Pk[k];
        gE = pp / P.E;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) bC[k] = P.p_mass * bA[k];
}

// Sum of v over the CTA (blockDim.x a multiple of 32, at most 1024), valid in
// thread 0.
__device__ __forceinline__ float block_sum(float v) {
    __shared__ float red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    float s = 0.0f;
    if (wid == 0) {
        s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

}  // namespace dw

// Two particles per thread: the per-particle MLS-MPM arithmetic of the fused
// G2P/P2G kernel evaluated on float2 pairs with the paired FP32 instructions
// of sm_100 and later (FFMA2, FMUL2, FADD2), so that one instruction advances
// both particles of a thread. Each operation rounds exactly as its scalar
// counterpart in mpm_math.cuh / mpm_g2p.cuh (one rounding per multiply, add
// or fused multiply-add); only the order of a few sums differs.
//   Stencil: quadratic B-spline weights (App. A.3, as in MLS-MPM).
//   G2P: v_p = sum_i w_ip v_i, C_p = (4/dx^2) sum_i w_ip v_i (x_i - x_p)^T,
//        x_p += dt v_p, F_p <- (I + dt C_p) F_p (Eqs. G2P, deformation_update).
//   Stress: Neo-Hookean P = mu (F - F^-T) + lam ln(J) F^-T (Eq. constitutive_model).
#pragma once

#include "mpm_p2g.cuh"

namespace dw {
namespace pr {

__device__ __forceinline__ float2 s2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b with one rounding
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
// c - a b with one rounding
__device__ __forceinline__ float2 fnma(float2 a, float2 b, float2 c) {
    return __ffma2_rn(make_float2(-a.x, -a.y), b, c);
}

// Stencils of the two particles of a thread: bases per particle, offsets and
// weights as pairs (.x = first particle, .y = second).
struct Stencil2 {
    int b0[3], b1[3];
    float2 fx[3];
    float2 w[3][3];
};

// ok0 / ok1: floor(x/dx - 0.5) stays in [0, N - 3] on every axis (false for
// NaN too); a failed particle gets base 0 on the failing and later axes.
__device__ __forceinline__ void stencil2(const MpmParams &P, const float2 x[3], Stencil2 &s,
                                         bool &ok0, bool &ok1) {
    ok0 = ok1 = true;
    const float hi = (float)(P.N - 3);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float2 xs = mul(x[a], s2(P.inv_dx));
        const float bb0 = floorf(xs.x - 0.5f), bb1 = floorf(xs.y - 0.5f);
        ok0 = ok0 && (bb0 >= 0.0f) && (bb0 <= hi);
        ok1 = ok1 && (bb1 >= 0.0f) && (bb1 <= hi);
        const int i0 = ok0 ? (int)bb0 : 0, i1 = ok1 ? (int)bb1 : 0;
        s.b0[a] = i0;
        s.b1[a] = i1;
        const float2 f = sub(xs, make_float2((float)i0, (float)i1));
        s.fx[a] = f;
        const float2 t = sub(s2(1.5f), f);
        s.w[a][0] = mul(mul(t, t), s2(0.5f));
        const float2 u = sub(f, s2(1.0f));
        s.w[a][1] = fnma(u, u, s2(0.75f));
        const float2 r = sub(f, s2(0.5f));
        s.w[a][2] = mul(mul(r, r), s2(0.5f));
    }
}

__device__ __forceinline__ float comp(const float4 &g, int c) {
    return c == 0 ? g.x : (c == 1 ? g.y : g.z);
}

// G2P sums of both particles. Node (oi, oj, ok) of particle j is read from
// src_j[off], off = (ok * 3 + oj) * 3 + oi when STAGED (27 nodes staged in
// shared memory), else off = ok * N^2 + oj * N + oi from the grid itself.
// Tensor-product evaluation as in g2p_update: per line of three nodes along
// x, a = sum wx v_i and bx = sum oi wx v_i; then v = sum wyz a and
// S_b = sum W o_b v_i, C = (4/dx^2) dx (S - v fx^T).
template <bool STAGED>
__device__ __forceinline__ void g2p_sums2(const MpmParams &P, const Stencil2 &s,
                                          const float4 *__restrict__ src0,
                                          const float4 *__restrict__ src1, float2 vn[3],
                                          float2 Cn[9]) {
    float2 S[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        vn[c] = s2(0.0f);
#pragma unroll
        for (int b = 0; b < 3; ++b) S[b][c] = s2(0.0f);
    }
    const int N = P.N, N2 = P.N * P.N;
    const float2 wx0 = s.w[0][0], wx1 = s.w[0][1], wx2 = s.w[0][2], wx2d = add(wx2, wx2);
#pragma unroll
    for (int ok = 0; ok < 3; ++ok)
#pragma unroll
        for (int oj = 0; oj < 3; ++oj) {
            const float2 wyz = mul(s.w[1][oj], s.w[2][ok]);
            const float2 wyz2 = add(wyz, wyz);
            float4 g0[3], g1[3];
#pragma unroll
            for (int oi = 0; oi < 3; ++oi) {
                const int off = STAGED ? (ok * 3 + oj) * 3 + oi : ok * N2 + oj * N + oi;
                g0[oi] = src0[off];
                g1[oi] = src1[off];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 G0 = make_float2(comp(g0[0], c), comp(g1[0], c));
                const float2 G1 = make_float2(comp(g0[1], c), comp(g1[1], c));
                const float2 G2 = make_float2(comp(g0[2], c), comp(g1[2], c));
                const float2 a = fma(wx2, G2, fma(wx1, G1, mul(wx0, G0)));
                const float2 bx = fma(wx2d, G2, mul(wx1, G1));
                vn[c] = fma(wyz, a, vn[c]);
                S[0][c] = fma(wyz, bx, S[0][c]);
                if (oj == 1) S[1][c] = fma(wyz, a, S[1][c]);
                if (oj == 2) S[1][c] = fma(wyz2, a, S[1][c]);
                if (ok == 1) S[2][c] = fma(wyz, a, S[2][c]);
                if (ok == 2) S[2][c] = fma(wyz2, a, S[2][c]);
            }
        }
    const float2 Ddx = s2(P.D * P.dx);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) Cn[3 * c + b] = mul(Ddx, fnma(vn[c], s.fx[b], S[b][c]));
}

// C = A B for 3x3 pairs (row-major).
__device__ __forceinline__ void mul3_2(const float2 A[9], const float2 B[9], float2 C[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = fma(A[3 * i + 2], B[6 + j], fma(A[3 * i + 1], B[3 + j], mul(A[3 * i], B[j])));
}

// C = A B^T
__device__ __forceinline__ void mul3_abt2(const float2 A[9], const float2 B[9], float2 C[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = fma(A[3 * i + 2], B[3 * j + 2],
                               fma(A[3 * i + 1], B[3 * j + 1], mul(A[3 * i], B[3 * j])));
}

// Cofactor matrix, A^-T = cof(A) / det(A).
__device__ __forceinline__ void cof3_2(const float2 A[9], float2 K[9]) {
    K[0] = fnma(A[5], A[7], mul(A[4], A[8]));
    K[1] = fnma(A[3], A[8], mul(A[5], A[6]));
    K[2] = fnma(A[4], A[6], mul(A[3], A[7]));
    K[3] = fnma(A[1], A[8], mul(A[2], A[7]));
    K[4] = fnma(A[2], A[6], mul(A[0], A[8]));
    K[5] = fnma(A[0], A[7], mul(A[1], A[6]));
    K[6] = fnma(A[2], A[4], mul(A[1], A[5]));
    K[7] = fnma(A[0], A[5], mul(A[2], A[3]));
    K[8] = fnma(A[1], A[3], mul(A[0], A[4]));
}

// Affine momentum matrices A = -dt V0 (4/dx^2) P F^T + m C of both particles.
// ok0 / ok1: det F > 0 (the stress is defined; P = 0 otherwise). The
// fixed-corotated model (MAT = DW_FIXED_COROTATED) runs the scalar affine
// update of the one-particle kernels (p2g_affine) per particle: the polar
// iteration's Newton loop ends at a different step for each.
// MAT < 0: the material of P, chosen at run time.
template <int MAT>
__device__ __forceinline__ void affine2(const MpmParams &P, const float2 F[9], const float2 C[9],
                                       float2 A[9], bool &ok0, bool &ok1) {
    if (MAT == DW_NEOHOOKEAN || (MAT < 0 && P.material == DW_NEOHOOKEAN)) {
        float2 Pk[9], K[9];
        cof3_2(F, K);
        // det F = F0 K0 + F1 K1 + F2 K2 (expansion along the first row)
        const float2 J = fma(F[2], K[2], fma(F[1], K[1], mul(F[0], K[0])));
        ok0 = J.x > 0.0f;
        ok1 = J.y > 0.0f;
        const float2 inv = make_float2(ok0 ? 1.0f / J.x : 0.0f, ok1 ? 1.0f / J.y : 0.0f);
        const float2 lnJ = make_float2(ok0 ? logf(J.x) : 0.0f, ok1 ? logf(J.y) : 0.0f);
        // P = mu F + (lam ln J - mu) F^-T
        const float2 mu = make_float2(ok0 ? P.mu : 0.0f, ok1 ? P.mu : 0.0f);
        const float2 c = sub(mul(s2(P.lam), lnJ), mu);
#pragma unroll
        for (int k = 0; k < 9; ++k) Pk[k] = fma(c, mul(K[k], inv), mul(mu, F[k]));
        float2 PFt[9];
        mul3_abt2(Pk, F, PFt);
        const float2 mk = s2(-P.kappa), pm = s2(P.p_mass);
#pragma unroll
        for (int k = 0; k < 9; ++k) A[k] = fma(mk, PFt[k], mul(pm, C[k]));
    } else {
        // one particle after the other, each one's A finished before the
        // other's polar iteration starts (fewer values live across the loop)
        float Fq[9], Cq[9], Aq[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            Fq[k] = F[k].x;
            Cq[k] = C[k].x;
        }
        ok0 = p2g_affine(P, Fq, Cq, Aq);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            A[k].x = Aq[k];
            Fq[k] = F[k].y;
            Cq[k] = C[k].y;
        }
        ok1 = p2g_affine(P, Fq, Cq, Aq);
#pragma unroll
        for (int k = 0; k < 9; ++k) A[k].y = Aq[k];
    }
}

// G2P sums of both particles from a box of staged grid velocities: planes
// box[c * BOXP + ((z * ey) + y) * ex + x] hold component c of the warp's
// nodes; o0 and o1 are the particles' base cells in box coordinates and
// exy = ex * ey. Tensor-product evaluation as in g2p_sums2; every load is
// [line base + constant].
template <int BOXP>
__device__ __forceinline__ void g2p_box2(const MpmParams &P, const Stencil2 &s,
                                         const float *__restrict__ box, int o0, int o1, int ex,
                                         int exy, float2 vn[3], float2 Cn[9]) {
    float2 S[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        vn[c] = s2(0.0f);
#pragma unroll
        for (int b = 0; b < 3; ++b) S[b][c] = s2(0.0f);
    }
    const float2 wx0 = s.w[0][0], wx1 = s.w[0][1], wx2 = s.w[0][2], wx2d = add(wx2, wx2);
#pragma unroll
    for (int ok = 0; ok < 3; ++ok)
#pragma unroll
        for (int oj = 0; oj < 3; ++oj) {
            const float2 wyz = mul(s.w[1][oj], s.w[2][ok]);
            const float2 wyz2 = add(wyz, wyz);
            const int line = ok * exy + oj * ex;
            const float *p0 = box + o0 + line, *p1 = box + o1 + line;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 G0 = make_float2(p0[c * BOXP], p1[c * BOXP]);
                const float2 G1 = make_float2(p0[c * BOXP + 1], p1[c * BOXP + 1]);
                const float2 G2 = make_float2(p0[c * BOXP + 2], p1[c * BOXP + 2]);
                const float2 a = fma(wx2, G2, fma(wx1, G1, mul(wx0, G0)));
                const float2 bx = fma(wx2d, G2, mul(wx1, G1));
                vn[c] = fma(wyz, a, vn[c]);
                S[0][c] = fma(wyz, bx, S[0][c]);
                if (oj == 1) S[1][c] = fma(wyz, a, S[1][c]);
                if (oj == 2) S[1][c] = fma(wyz2, a, S[1][c]);
                if (ok == 1) S[2][c] = fma(wyz, a, S[2][c]);
                if (ok == 2) S[2][c] = fma(wyz2, a, S[2][c]);
            }
        }
    const float2 Ddx = s2(P.D * P.dx);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) Cn[3 * c + b] = mul(Ddx, fnma(vn[c], s.fx[b], S[b][c]));
}

}  // namespace pr
}  // namespace dw

// Per-particle MLS-MPM arithmetic in float32: quadratic B-spline stencil,
// 3x3 algebra, the two constitutive models and their reverse modes.
//   Weights: App. A.3 ("B-spline kernel weight", quadratic as in MLS-MPM).
//   Neo-Hookean P = mu (F - F^-T) + lam ln(J) F^-T, the gradient of the energy
//   of Eq. constitutive_model; Lame parameters from Eq. young_poisson.
//   Fixed-corotated P = 2 mu (F - R) + lam (J - 1) J F^-T with F = R S the polar
//   decomposition, computed by Newton's iteration X <- (X + X^-T) / 2
//   (Higham 1986, "Computing the polar decomposition - with applications").
#pragma once

#include "common.cuh"

namespace dw {

struct MpmParams {
    int N;           // nodes per axis
    float dx, inv_dx;
    float dt;
    float D;         // 4 / dx^2, the inverse inertia-like tensor of the quadratic kernel
    float gx, gy, gz;
    int band;
    int material;
    float mu, lam, E;
    float p_mass, p_vol;
    float kappa;     // dt * p_vol * D
};

struct Stencil {
    int base[3];
    float fx[3];
    float w[3][3];
    float dw[3][3];
};

// Quadratic B-spline stencil of a particle at (px, py, pz). Returns false when
// floor(x/dx - 0.5) leaves [0, N - 3] on some axis (or x is not finite).
__device__ __forceinline__ bool make_stencil(const MpmParams &P, float px, float py, float pz,
                                             Stencil &s) {
    float xs[3] = {px * P.inv_dx, py * P.inv_dx, pz * P.inv_dx};
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float b = floorf(xs[a] - 0.5f);
        ok = ok && (b >= 0.0f) && (b <= (float)(P.N - 3));  // false for NaN too
        int bi = ok ? (int)b : 0;
        s.base[a] = bi;
        float f = xs[a] - (float)bi;
        s.fx[a] = f;
        s.w[a][0] = 0.5f * (1.5f - f) * (1.5f - f);
        s.w[a][1] = 0.75f - (f - 1.0f) * (f - 1.0f);
        s.w[a][2] = 0.5f * (f - 0.5f) * (f - 0.5f);
        s.dw[a][0] = f - 1.5f;
        s.dw[a][1] = -2.0f * (f - 1.0f);
        s.dw[a][2] = f - 0.5f;
    }
    return ok;
}

__device__ __forceinline__ float det3(const float A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// cofactor matrix, A^-T = cof(A) / det(A)
__device__ __forceinline__ void cof3(const float A[9], float K[9]) {
    K[0] = A[4] * A[8] - A[5] * A[7];
    K[1] = A[5] * A[6] - A[3] * A[8];
    K[2] = A[3] * A[7] - A[4] * A[6];
    K[3] = A[2] * A[7] - A[1] * A[8];
    K[4] = A[0] * A[8] - A[2] * A[6];
    K[5] = A[1] * A[6] - A[0] * A[7];
    K[6] = A[1] * A[5] - A[2] * A[4];
    K[7] = A[2] * A[3] - A[0] * A[5];
    K[8] = A[0] * A[4] - A[1] * A[3];
}

__device__ __forceinline__ void mul3(const float A[9], const float B[9], float C[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// C = A B^T
__device__ __forceinline__ void mul3_abt(const float A[9], const float B[9], float C[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[3 * j] + A[3 * i + 1] * B[3 * j + 1] + A[3 * i + 2] * B[3 * j + 2];
}

// C = A^T B
__device__ __forceinline__ void mul3_atb(const float A[9], const float B[9], float C[9]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[i] * B[j] + A[3 + i] * B[3 + j] + A[6 + i] * B[6 + j];
}

// Polar factor R of F (det F > 0) by Newton's iteration; false if det <= 0.
__device__ __forceinline__ bool polar_R(const float F[9], float R[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = F[k];
    bool converged = false;
    for (int it = 0; it < 40; ++it) {
        float K[9];
        cof3(R, K);
        float J = det3(R);
        if (!(J > 0.0f)) return false;
        float inv = 1.0f / J;
        float change = 0.0f, norm = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float xn = 0.5f * (R[k] + K[k] * inv);
            change += (xn - R[k]) * (xn - R[k]);
            norm += xn * xn;
            R[k] = xn;
        }
        if (converged) break;                    // one more step after the test passes
        converged = change <= 1e-10f * norm;     // quadratic: the next step is at rounding level
    }
    return true;
}

// First Piola-Kirchhoff stress. Returns false for det F <= 0.
__device__ __forceinline__ bool stress_P(const MpmParams &P, const float F[9], float Pk[9]) {
    float K[9];
    cof3(F, K);
    float J = det3(F);
    if (!(J > 0.0f)) {
#pragma unroll
        for (int k = 0; k < 9; ++k) Pk[k] = 0.0f;
        return false;
    }
    if (P.material == DW_NEOHOOKEAN) {
        float inv = 1.0f / J;
        float lnJ = logf(J);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float FinvT = K[k] * inv;
            Pk[k] = P.mu * (F[k] - FinvT) + P.lam * lnJ * FinvT;
        }
    } else {
        float R[9];
        polar_R(F, R);
#pragma unroll
        for (int k = 0; k < 9; ++k) Pk[k] = 2.0f * P.mu * (F[k] - R[k]) + P.lam * (J - 1.0f) * K[k];
    }
    return true;
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// Reverse mode of stress_P: Fbar += (dP/dF)^T Pbar.
__device__ __forceinline__ void stress_P_adjoint(const MpmParams &P, const float F[9],
                                                 const float Pbar[9], float Fbar[9]) {
    float K[9];
    cof3(F, K);
    float J = det3(F);
    if (!(J > 0.0f)) return;
    if (P.material == DW_NEOHOOKEAN) {
        // P = mu F + (lam lnJ - mu) F^-T:
        // Fbar += mu Pbar + lam <Pbar, F^-T> F^-T - (lam lnJ - mu) F^-T Pbar^T F^-T
        float inv = 1.0f / J;
        float FinvT[9];
        float pf = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            FinvT[k] = K[k] * inv;
            pf += Pbar[k] * FinvT[k];
        }
        float T1[9], T2[9];
        mul3_abt(FinvT, Pbar, T1);  // F^-T Pbar^T
        mul3(T1, FinvT, T2);
        float c = P.lam * logf(J) - P.mu;
#pragma unroll
        for (int k = 0; k < 9; ++k) Fbar[k] += P.mu * Pbar[k] + P.lam * pf * FinvT[k] - c * T2[k];
    } else {
        // P = 2mu F - 2mu R + lam (J - 1) cof(F)
        float R[9];
        polar_R(F, R);
        float S[9];
        mul3_atb(R, F, S);
        // rotation: R^T dR = skew(omega), (tr(S) I - S) omega = axial(M - M^T), M = R^T dF.
        // Reverse: Fbar += R skew(b), b = (tr(S) I - S)^-1 axial(A - A^T), A = R^T (-2 mu Pbar).
        float A[9];
        mul3_atb(R, Pbar, A);
        float s = -2.0f * P.mu;
        float a[3] = {s * (A[7] - A[5]), s * (A[2] - A[6]), s * (A[3] - A[1])};
        float trS = S[0] + S[4] + S[8];
        float Km[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                Km[3 * i + j] = -0.5f * (S[3 * i + j] + S[3 * j + i]) + (i == j ? trS : 0.0f);
        float Kc[9];
        cof3(Km, Kc);
        float dinv = 1.0f / det3(Km);
        float b[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) b[i] = (Kc[i] * a[0] + Kc[3 + i] * a[1] + Kc[6 + i] * a[2]) * dinv;
        float Sk[9] = {0.0f, -b[2], b[1], b[2], 0.0f, -b[0], -b[1], b[0], 0.0f};
        float RS[9];
        mul3(R, Sk, RS);
        // cofactor: columns of cof(F) are f2 x f3, f3 x f1, f1 x f2
        float f0[3] = {F[0], F[3], F[6]}, f1[3] = {F[1], F[4], F[7]}, f2[3] = {F[2], F[5], F[8]};
        float g0[3] = {Pbar[0], Pbar[3], Pbar[6]}, g1[3] = {Pbar[1], Pbar[4], Pbar[7]},
              g2[3] = {Pbar[2], Pbar[5], Pbar[8]};
        float d0[3], d1[3], d2[3], t1[3], t2[3];
        cross3(g1, f2, t1);
        cross3(f1, g2, t2);
#pragma unroll
        for (int r = 0; r < 3; ++r) d0[r] = t1[r] + t2[r];
        cross3(f2, g0, t1);
        cross3(g2, f0, t2);
#pragma unroll
        for (int r = 0; r < 3; ++r) d1[r] = t1[r] + t2[r];
        cross3(g0, f1, t1);
        cross3(f0, g1, t2);
#pragma unroll
        for (int r = 0; r < 3; ++r) d2[r] = t1[r] + t2[r];
        float pk = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) pk += Pbar[k] * K[k];
        float lj = P.lam * (J - 1.0f);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            Fbar[3 * r + 0] += 2.0f * P.mu * Pbar[3 * r + 0] + RS[3 * r + 0] + P.lam * pk * K[3 * r + 0] + lj * d0[r];
            Fbar[3 * r + 1] += 2.0f * P.mu * Pbar[3 * r + 1] + RS[3 * r + 1] + P.lam * pk * K[3 * r + 1] + lj * d1[r];
            Fbar[3 * r + 2] += 2.0f * P.mu * Pbar[3 * r + 2] + RS[3 * r + 2] + P.lam * pk * K[3 * r + 2] + lj * d2[r];
        }
    }
}

__device__ __forceinline__ bool finite9(const float A[9]) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 9; ++k) ok = ok && isfinite(A[k]);
    return ok;
}

}  // namespace dw

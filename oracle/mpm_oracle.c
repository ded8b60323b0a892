/*
 * FP64 CPU oracle for the differentiable MLS-MPM substep of DiffWind.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow restatement of the
 * method that the CUDA path is checked against. Only tests/, the smoke check
 * in __graft_entry__.py and the cpu_baseline leg of bench.py may load it. It
 * shares no code, header or table with the CUDA library.
 *
 * What it computes (one substep S of Eq. simulation_mpm, Sec. 3.3):
 *   (x, v, F, C)^t  ->  (x, v, F, C)^{t+1}  given E, nu, the wind force field
 *   F_w and dt.
 *   1. Quadratic B-spline weights w_ip on the 3x3x3 stencil (App. A.3, the
 *      "B-spline kernel weight" of Eq. G2P; quadratic as in MLS-MPM).
 *   2. First Piola-Kirchhoff stress P(F): Neo-Hookean (Eq. constitutive_model,
 *      read as dpsi/dF of the printed energy: mu(F - F^-T) + lam ln(J) F^-T)
 *      or fixed-corotated 2mu(F - R) + lam(J - 1) J F^-T; Lame parameters
 *      from E and nu by Eq. young_poisson.
 *   3. P2G (Eq. P2G) plus the MLS-MPM stress momentum
 *      -dt V0 (4/dx^2) P F^T (x_i - x_p) that MLS-MPM adds (App. A.3 cites
 *      MLS-MPM; Cauchy stress sigma = J^-1 P F^T, Sec. 3.1).
 *   4. Grid update: v_i = p_i / m_i + dt (g + a_w(x_i, t)), the wind force
 *      applied per unit mass on the background grid (Sec. 3, Sec. 3.2);
 *      sticky walls zero v_i in a band of bc_band nodes at every face.
 *   5. G2P (Eq. G2P) with the APIC/MLS affine matrix
 *      C_p = (4/dx^2) sum_i w_ip v_i (x_i - x_p)^T, x += dt v, and
 *      F <- (I + dt C) F with the C of this G2P (Eq. deformation_update).
 *      Pinned particles keep v = 0 and C = 0 (so x and F do not change).
 *   6. Wind force field a_w(x, t): node-centred nf^3 grid spanning the unit
 *      cube (node j at j/(nf-1)), trilinear in space, linear in time between
 *      n_frames keyframes at k * t_total / (n_frames - 1), clamped.
 * Plus the hand-derived reverse-mode adjoint of the whole substep, which the
 * tests pin against central finite differences of the forward in FP64.
 *
 * Layouts (the same conventions the C-ABI documents): particle arrays are
 * structure-of-arrays, x[a*n + p], C[(3a+b)*n + p] (row-major 3x3 per
 * particle); the wind field is values[(((f*nf + k)*nf + j)*nf + i)*3 + c]
 * with i the x index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 3
#define ORC_ERR_NONFINITE 4
#define ORC_ERR_DOMAIN 5
#define ORC_ERR_INVERTED 7

typedef struct {
    int n_grid;        /* nodes per axis; dx = 1 / n_grid */
    double dt;         /* substep length */
    double gravity[3]; /* body acceleration */
    int bc_band;       /* sticky wall band width, in nodes */
    int material;      /* 0 = Neo-Hookean, 1 = fixed-corotated */
    double E, nu;      /* Young's modulus and Poisson ratio */
    double p_mass;     /* particle mass m_p */
    double p_vol;      /* particle rest volume V_p^0 */
} orc_mpm_params;

typedef struct {
    const double *values; /* [n_frames][nf][nf][nf][3] */
    int nf;
    int n_frames;
    double t_total;
} orc_wind;

/* ---------------------------------------------------------------- 3x3 -- */

static double det3(const double A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* cofactor matrix; A^-T = cof(A) / det(A) */
static void cof3(const double A[9], double K[9]) {
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

static void matmul3(const double A[9], const double B[9], double Cm[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            Cm[3 * i + j] = s;
        }
}

static void transpose3(const double A[9], double T[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * i + j] = A[3 * j + i];
}

static double dot9(const double A[9], const double B[9]) {
    double s = 0.0;
    for (int k = 0; k < 9; ++k) s += A[k] * B[k];
    return s;
}

static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* --------------------------------------------------------- constitutive -- */

/* Eq. young_poisson */
void orc_lame(double E, double nu, double *mu, double *lam) {
    *mu = E / (2.0 * (1.0 + nu));
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

/* Polar decomposition F = R S by Newton's iteration X <- (X + X^-T) / 2
 * (Higham 1986, "Computing the polar decomposition - with applications"),
 * iterated in FP64 until it stops moving. Requires det F > 0. */
int orc_polar(const double F[9], double R[9], double S[9]) {
    if (!(det3(F) > 0.0)) return ORC_ERR_INVERTED;
    double X[9];
    memcpy(X, F, sizeof X);
    for (int it = 0; it < 200; ++it) {
        double K[9], Xn[9];
        cof3(X, K);
        double J = det3(X);
        double change = 0.0, norm = 0.0;
        for (int k = 0; k < 9; ++k) {
            Xn[k] = 0.5 * (X[k] + K[k] / J);
            change += (Xn[k] - X[k]) * (Xn[k] - X[k]);
            norm += Xn[k] * Xn[k];
        }
        memcpy(X, Xn, sizeof X);
        if (change <= 1e-30 * norm) break;
    }
    memcpy(R, X, sizeof X);
    double Rt[9];
    transpose3(R, Rt);
    matmul3(Rt, F, S);
    return ORC_OK;
}

/* Neo-Hookean energy of Eq. constitutive_model */
double orc_neohookean_psi(const double F[9], double mu, double lam) {
    double tr = 0.0;
    for (int k = 0; k < 9; ++k) tr += F[k] * F[k]; /* trace(F^T F) */
    double lnJ = log(det3(F));
    return 0.5 * mu * (tr - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ;
}

/* P = dpsi/dF of the Neo-Hookean energy: mu (F - F^-T) + lam ln(J) F^-T */
int orc_neohookean_P(const double F[9], double mu, double lam, double P[9]) {
    double J = det3(F);
    if (!(J > 0.0)) return ORC_ERR_INVERTED;
    double K[9];
    cof3(F, K);
    double lnJ = log(J);
    for (int k = 0; k < 9; ++k) {
        double FinvT = K[k] / J;
        P[k] = mu * (F[k] - FinvT) + lam * lnJ * FinvT;
    }
    return ORC_OK;
}

/* fixed-corotated energy mu |F - R|^2 + lam/2 (J - 1)^2 (Stomakhin et al. 2012) */
double orc_fixedcorot_psi(const double F[9], double mu, double lam) {
    double R[9], S[9];
    if (orc_polar(F, R, S) != ORC_OK) return NAN;
    double s = 0.0;
    for (int k = 0; k < 9; ++k) s += (F[k] - R[k]) * (F[k] - R[k]);
    double J = det3(F);
    return mu * s + 0.5 * lam * (J - 1.0) * (J - 1.0);
}

/* P = 2 mu (F - R) + lam (J - 1) J F^-T, with J F^-T = cof(F) */
int orc_fixedcorot_P(const double F[9], double mu, double lam, double P[9]) {
    double R[9], S[9], K[9];
    int st = orc_polar(F, R, S);
    if (st != ORC_OK) return st;
    cof3(F, K);
    double J = det3(F);
    for (int k = 0; k < 9; ++k) P[k] = 2.0 * mu * (F[k] - R[k]) + lam * (J - 1.0) * K[k];
    return ORC_OK;
}

int orc_stress(int material, const double F[9], double mu, double lam, double P[9]) {
    if (material == 0) return orc_neohookean_P(F, mu, lam, P);
    if (material == 1) return orc_fixedcorot_P(F, mu, lam, P);
    return ORC_ERR_ARG;
}

/* Reverse mode of P(F): given Pbar = dL/dP, add dL/dF to Fbar. */
int orc_stress_adjoint(int material, const double F[9], double mu, double lam,
                       const double Pbar[9], double Fbar[9]) {
    double J = det3(F);
    if (!(J > 0.0)) return ORC_ERR_INVERTED;
    double K[9];
    cof3(F, K);
    if (material == 0) {
        /* P = mu F + (lam lnJ - mu) F^-T
         * Fbar += mu Pbar + lam <Pbar, F^-T> F^-T - (lam lnJ - mu) F^-T Pbar^T F^-T */
        double FinvT[9], PbT[9], T1[9], T2[9];
        for (int k = 0; k < 9; ++k) FinvT[k] = K[k] / J;
        double lnJ = log(J);
        double pf = dot9(Pbar, FinvT);
        transpose3(Pbar, PbT);
        matmul3(FinvT, PbT, T1);
        matmul3(T1, FinvT, T2);
        for (int k = 0; k < 9; ++k)
            Fbar[k] += mu * Pbar[k] + lam * pf * FinvT[k] - (lam * lnJ - mu) * T2[k];
        return ORC_OK;
    }
    if (material == 1) {
        /* P = 2mu F - 2mu R + lam (J - 1) cof(F) */
        double R[9], S[9];
        int st = orc_polar(F, R, S);
        if (st != ORC_OK) return st;
        /* rotation part: R^T dR = Omega skew, (tr(S) I - S) omega = axial(M - M^T),
         * M = R^T dF; the reverse of dR is R skew(b), b = (tr(S) I - S)^-1 a,
         * a = axial(A - A^T), A = R^T Gr with Gr = dL/dR = -2 mu Pbar. */
        double Rt[9], A[9], Gr[9];
        for (int k = 0; k < 9; ++k) Gr[k] = -2.0 * mu * Pbar[k];
        transpose3(R, Rt);
        matmul3(Rt, Gr, A);
        double a[3] = {A[7] - A[5], A[2] - A[6], A[3] - A[1]};
        double trS = S[0] + S[4] + S[8];
        double Km[9];
        for (int k = 0; k < 9; ++k) Km[k] = -0.5 * (S[k] + S[(k % 3) * 3 + k / 3]);
        Km[0] += trS;
        Km[4] += trS;
        Km[8] += trS;
        double Kc[9];
        cof3(Km, Kc);
        double dK = det3(Km);
        double b[3];
        for (int i = 0; i < 3; ++i) /* Km^-1 = cof(Km)^T / det(Km) */
            b[i] = (Kc[0 * 3 + i] * a[0] + Kc[1 * 3 + i] * a[1] + Kc[2 * 3 + i] * a[2]) / dK;
        double Sk[9] = {0.0, -b[2], b[1], b[2], 0.0, -b[0], -b[1], b[0], 0.0};
        double RS[9];
        matmul3(R, Sk, RS);
        /* cofactor part: d cof(F) with columns f2 x f3, f3 x f1, f1 x f2 */
        double f[3][3], g[3][3];
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 3; ++r) {
                f[c][r] = F[3 * r + c];
                g[c][r] = Pbar[3 * r + c];
            }
        double d[3][3], t1[3], t2[3];
        cross3(g[1], f[2], t1);
        cross3(f[1], g[2], t2);
        for (int r = 0; r < 3; ++r) d[0][r] = t1[r] + t2[r];
        cross3(f[2], g[0], t1);
        cross3(g[2], f[0], t2);
        for (int r = 0; r < 3; ++r) d[1][r] = t1[r] + t2[r];
        cross3(g[0], f[1], t1);
        cross3(f[0], g[1], t2);
        for (int r = 0; r < 3; ++r) d[2][r] = t1[r] + t2[r];
        double pk = dot9(Pbar, K);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                int k = 3 * r + c;
                Fbar[k] += 2.0 * mu * Pbar[k] + RS[k] + lam * pk * K[k] +
                           lam * (J - 1.0) * d[c][r];
            }
        return ORC_OK;
    }
    return ORC_ERR_ARG;
}

/* ------------------------------------------------------------- weights -- */

void orc_bspline_weights(double fx, double w[3]) {
    w[0] = 0.5 * (1.5 - fx) * (1.5 - fx);
    w[1] = 0.75 - (fx - 1.0) * (fx - 1.0);
    w[2] = 0.5 * (fx - 0.5) * (fx - 0.5);
}

static void bspline_dweights(double fx, double dw[3]) {
    dw[0] = fx - 1.5;
    dw[1] = -2.0 * (fx - 1.0);
    dw[2] = fx - 0.5;
}

typedef struct {
    int base[3];
    double fx[3];
    double w[3][3];
    double dw[3][3];
} stencil;

static int make_stencil(int N, const double xp[3], stencil *s) {
    for (int a = 0; a < 3; ++a) {
        double xs = xp[a] * (double)N; /* x / dx */
        if (!isfinite(xs)) return ORC_ERR_NONFINITE;
        int b = (int)floor(xs - 0.5);
        if (b < 0 || b > N - 3) return ORC_ERR_DOMAIN;
        s->base[a] = b;
        s->fx[a] = xs - (double)b;
        orc_bspline_weights(s->fx[a], s->w[a]);
        bspline_dweights(s->fx[a], s->dw[a]);
    }
    return ORC_OK;
}

static int64_t node_index(int N, int i, int j, int k) {
    return ((int64_t)k * N + j) * N + i;
}

/* ---------------------------------------------------------------- wind -- */

typedef struct {
    int64_t idx[16]; /* element offsets (times 3) of the 16 contributing nodes */
    double wt[16];
} wind_taps;

static void wind_make_taps(const orc_wind *w, const double pos[3], double t, wind_taps *tp) {
    int nf = w->nf;
    int i0[3];
    double fr[3];
    for (int a = 0; a < 3; ++a) {
        double p = pos[a];
        if (p < 0.0) p = 0.0;
        if (p > 1.0) p = 1.0;
        if (nf < 2) {
            i0[a] = 0;
            fr[a] = 0.0;
            continue;
        }
        double s = p * (double)(nf - 1);
        int i = (int)floor(s);
        if (i > nf - 2) i = nf - 2;
        if (i < 0) i = 0;
        i0[a] = i;
        fr[a] = s - (double)i;
    }
    int k0 = 0;
    double ft = 0.0;
    if (w->n_frames > 1) {
        double tc = t;
        if (tc < 0.0) tc = 0.0;
        if (tc > w->t_total) tc = w->t_total;
        double s = tc / w->t_total * (double)(w->n_frames - 1);
        k0 = (int)floor(s);
        if (k0 > w->n_frames - 2) k0 = w->n_frames - 2;
        ft = s - (double)k0;
    }
    int n = 0;
    int nt = (w->n_frames > 1) ? 2 : 1;
    int nc = (nf > 1) ? 2 : 1;
    for (int dk = 0; dk < nt; ++dk)
        for (int cz = 0; cz < nc; ++cz)
            for (int cy = 0; cy < nc; ++cy)
                for (int cx = 0; cx < nc; ++cx) {
                    double wt = (nt > 1 ? (dk ? ft : 1.0 - ft) : 1.0);
                    if (nc > 1) {
                        wt *= (cx ? fr[0] : 1.0 - fr[0]);
                        wt *= (cy ? fr[1] : 1.0 - fr[1]);
                        wt *= (cz ? fr[2] : 1.0 - fr[2]);
                    }
                    int64_t f = k0 + dk;
                    int64_t node = ((f * nf + (i0[2] + cz)) * nf + (i0[1] + cy)) * nf + (i0[0] + cx);
                    tp->idx[n] = node * 3;
                    tp->wt[n] = wt;
                    ++n;
                }
    for (; n < 16; ++n) {
        tp->idx[n] = 0;
        tp->wt[n] = 0.0;
    }
}

static void wind_sample_one(const orc_wind *w, const double pos[3], double t, double out[3]) {
    wind_taps tp;
    wind_make_taps(w, pos, t, &tp);
    out[0] = out[1] = out[2] = 0.0;
    for (int n = 0; n < 16; ++n)
        for (int c = 0; c < 3; ++c) out[c] += tp.wt[n] * w->values[tp.idx[n] + c];
}

static void wind_sample_adjoint_one(const orc_wind *w, const double pos[3], double t,
                                    const double g[3], double *g_values) {
    wind_taps tp;
    wind_make_taps(w, pos, t, &tp);
    for (int n = 0; n < 16; ++n)
        for (int c = 0; c < 3; ++c) g_values[tp.idx[n] + c] += tp.wt[n] * g[c];
}

/* a_w at n positions pos[3][n] (structure of arrays) and time t */
void orc_wind_sample(const double *values, int nf, int n_frames, double t_total,
                     const double *pos, int64_t n, double t, double *out) {
    orc_wind w = {values, nf, n_frames, t_total};
    for (int64_t p = 0; p < n; ++p) {
        double q[3] = {pos[p], pos[n + p], pos[2 * n + p]}, o[3];
        wind_sample_one(&w, q, t, o);
        for (int c = 0; c < 3; ++c) out[c * n + p] = o[c];
    }
}

/* g_values += S^T g_out, the transpose of orc_wind_sample in the field values */
void orc_wind_sample_adjoint(const double *values, int nf, int n_frames, double t_total,
                             const double *pos, int64_t n, double t, const double *g_out,
                             double *g_values) {
    orc_wind w = {values, nf, n_frames, t_total};
    for (int64_t p = 0; p < n; ++p) {
        double q[3] = {pos[p], pos[n + p], pos[2 * n + p]};
        double g[3] = {g_out[p], g_out[n + p], g_out[2 * n + p]};
        wind_sample_adjoint_one(&w, q, t, g, g_values);
    }
}

/* ---------------------------------------------------------- substep ---- */

static void load_particle(int64_t n, int64_t p, const double *x, const double *v,
                          const double *C, const double *F, double xp[3], double vp[3],
                          double Cp[9], double Fp[9]) {
    for (int a = 0; a < 3; ++a) {
        if (x) xp[a] = x[a * n + p];
        if (v) vp[a] = v[a * n + p];
    }
    for (int k = 0; k < 9; ++k) {
        if (C) Cp[k] = C[k * n + p];
        if (F) Fp[k] = F[k * n + p];
    }
}

/* P2G (Eq. P2G + MLS stress). gm[N^3], gp[3][N^3] are overwritten. */
int orc_mpm_p2g(const orc_mpm_params *pr, int64_t n, const double *x, const double *v,
                const double *C, const double *F, double *gm, double *gp) {
    int N = pr->n_grid;
    int64_t nn = (int64_t)N * N * N;
    double dx = 1.0 / N, D = 4.0 * N * N; /* 4 / dx^2 */
    double mu, lam;
    orc_lame(pr->E, pr->nu, &mu, &lam);
    memset(gm, 0, sizeof(double) * nn);
    memset(gp, 0, sizeof(double) * nn * 3);
    for (int64_t p = 0; p < n; ++p) {
        double xp[3], vp[3], Cp[9], Fp[9];
        load_particle(n, p, x, v, C, F, xp, vp, Cp, Fp);
        stencil s;
        int st = make_stencil(N, xp, &s);
        if (st != ORC_OK) return st;
        double P[9], Ft[9], PFt[9], A[9];
        st = orc_stress(pr->material, Fp, mu, lam, P);
        if (st != ORC_OK) return st;
        transpose3(Fp, Ft);
        matmul3(P, Ft, PFt);
        double kappa = pr->dt * pr->p_vol * D;
        for (int k = 0; k < 9; ++k) A[k] = -kappa * PFt[k] + pr->p_mass * Cp[k];
        for (int oi = 0; oi < 3; ++oi)
            for (int oj = 0; oj < 3; ++oj)
                for (int ok = 0; ok < 3; ++ok) {
                    double W = s.w[0][oi] * s.w[1][oj] * s.w[2][ok];
                    double dpos[3] = {(oi - s.fx[0]) * dx, (oj - s.fx[1]) * dx, (ok - s.fx[2]) * dx};
                    int64_t id = node_index(N, s.base[0] + oi, s.base[1] + oj, s.base[2] + ok);
                    gm[id] += W * pr->p_mass;
                    for (int c = 0; c < 3; ++c) {
                        double mom = pr->p_mass * vp[c];
                        for (int b = 0; b < 3; ++b) mom += A[3 * c + b] * dpos[b];
                        gp[c * nn + id] += W * mom;
                    }
                }
    }
    return ORC_OK;
}

static int in_sticky_band(int N, int band, int i, int j, int k) {
    return i < band || j < band || k < band || i > N - 1 - band || j > N - 1 - band ||
           k > N - 1 - band;
}

/* Grid update: gv[3][N^3] overwritten. */
int orc_mpm_grid_update(const orc_mpm_params *pr, const double *gm, const double *gp,
                        const orc_wind *wind, double t, double *gv) {
    int N = pr->n_grid;
    int64_t nn = (int64_t)N * N * N;
    double dx = 1.0 / N;
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                int64_t id = node_index(N, i, j, k);
                double vi[3] = {0.0, 0.0, 0.0};
                if (gm[id] > 0.0 && !in_sticky_band(N, pr->bc_band, i, j, k)) {
                    double xi[3] = {i * dx, j * dx, k * dx}, aw[3];
                    wind_sample_one(wind, xi, t, aw);
                    for (int c = 0; c < 3; ++c)
                        vi[c] = gp[c * nn + id] / gm[id] + pr->dt * (pr->gravity[c] + aw[c]);
                }
                for (int c = 0; c < 3; ++c) gv[c * nn + id] = vi[c];
            }
    return ORC_OK;
}

/* G2P (Eq. G2P, Eq. deformation_update) */
int orc_mpm_g2p(const orc_mpm_params *pr, int64_t n, const double *x, const double *F,
                const uint8_t *pinned, const double *gv, double *x_out, double *v_out,
                double *C_out, double *F_out) {
    int N = pr->n_grid;
    int64_t nn = (int64_t)N * N * N;
    double dx = 1.0 / N, D = 4.0 * N * N;
    for (int64_t p = 0; p < n; ++p) {
        double xp[3], Fp[9];
        load_particle(n, p, x, NULL, NULL, F, xp, NULL, NULL, Fp);
        stencil s;
        int st = make_stencil(N, xp, &s);
        if (st != ORC_OK) return st;
        double vn[3] = {0, 0, 0}, Cn[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int oi = 0; oi < 3; ++oi)
            for (int oj = 0; oj < 3; ++oj)
                for (int ok = 0; ok < 3; ++ok) {
                    double W = s.w[0][oi] * s.w[1][oj] * s.w[2][ok];
                    double dpos[3] = {(oi - s.fx[0]) * dx, (oj - s.fx[1]) * dx, (ok - s.fx[2]) * dx};
                    int64_t id = node_index(N, s.base[0] + oi, s.base[1] + oj, s.base[2] + ok);
                    for (int a = 0; a < 3; ++a) {
                        double va = gv[a * nn + id];
                        vn[a] += W * va;
                        for (int b = 0; b < 3; ++b) Cn[3 * a + b] += D * W * va * dpos[b];
                    }
                }
        if (pinned && pinned[p]) {
            memset(vn, 0, sizeof vn);
            memset(Cn, 0, sizeof Cn);
        }
        double Fn[9], Mdt[9];
        for (int k = 0; k < 9; ++k) Mdt[k] = pr->dt * Cn[k];
        Mdt[0] += 1.0;
        Mdt[4] += 1.0;
        Mdt[8] += 1.0;
        matmul3(Mdt, Fp, Fn);
        for (int a = 0; a < 3; ++a) {
            x_out[a * n + p] = xp[a] + pr->dt * vn[a];
            v_out[a * n + p] = vn[a];
        }
        for (int k = 0; k < 9; ++k) {
            C_out[k * n + p] = Cn[k];
            F_out[k * n + p] = Fn[k];
        }
    }
    return ORC_OK;
}

/* One substep S of Eq. simulation_mpm. Outputs may not alias inputs. */
int orc_mpm_substep(const orc_mpm_params *pr, int64_t n, const double *x, const double *v,
                    const double *C, const double *F, const uint8_t *pinned,
                    const double *wind_values, int nf, int n_frames, double t_total, double t,
                    double *x_out, double *v_out, double *C_out, double *F_out) {
    if (!pr || pr->n_grid < 4 || n < 0) return ORC_ERR_ARG;
    int N = pr->n_grid;
    int64_t nn = (int64_t)N * N * N;
    orc_wind wind = {wind_values, nf, n_frames, t_total};
    double *gm = (double *)malloc(sizeof(double) * nn);
    double *gp = (double *)malloc(sizeof(double) * nn * 3);
    double *gv = (double *)malloc(sizeof(double) * nn * 3);
    int st = ORC_ERR_OOM;
    if (gm && gp && gv) {
        st = orc_mpm_p2g(pr, n, x, v, C, F, gm, gp);
        if (st == ORC_OK) st = orc_mpm_grid_update(pr, gm, gp, &wind, t, gv);
        if (st == ORC_OK) st = orc_mpm_g2p(pr, n, x, F, pinned, gv, x_out, v_out, C_out, F_out);
    }
    free(gm);
    free(gp);
    free(gv);
    return st;
}

/* Gradient of the stencil weight product W_o = w_x w_y w_z with respect to x_p. */
static void weight_grad(int N, const stencil *s, int oi, int oj, int ok, double gW[3]) {
    double wx = s->w[0][oi], wy = s->w[1][oj], wz = s->w[2][ok];
    gW[0] = s->dw[0][oi] * wy * wz * N;
    gW[1] = wx * s->dw[1][oj] * wz * N;
    gW[2] = wx * wy * s->dw[2][ok] * N;
}

/* Reverse mode of orc_mpm_substep. Given the gradients of a scalar loss with
 * respect to the substep outputs (gx_out .. gF_out), writes the gradients with
 * respect to the substep inputs (gx .. gF, overwritten), and accumulates the
 * gradients with respect to the wind field values (g_wind, same layout as the
 * field) and Young's modulus (*g_E). */
int orc_mpm_substep_adjoint(const orc_mpm_params *pr, int64_t n, const double *x,
                            const double *v, const double *C, const double *F,
                            const uint8_t *pinned, const double *wind_values, int nf,
                            int n_frames, double t_total, double t, const double *gx_out,
                            const double *gv_out, const double *gC_out, const double *gF_out,
                            double *gx, double *gvp, double *gC, double *gF, double *g_wind,
                            double *g_E) {
    if (!pr || pr->n_grid < 4 || n < 0) return ORC_ERR_ARG;
    int N = pr->n_grid;
    int64_t nn = (int64_t)N * N * N;
    double dx = 1.0 / N, D = 4.0 * N * N;
    double mu, lam;
    orc_lame(pr->E, pr->nu, &mu, &lam);
    double kappa = pr->dt * pr->p_vol * D;
    orc_wind wind = {wind_values, nf, n_frames, t_total};
    double *gm = (double *)malloc(sizeof(double) * nn);
    double *gp = (double *)malloc(sizeof(double) * nn * 3);
    double *gvg = (double *)malloc(sizeof(double) * nn * 3);
    double *bv = (double *)calloc((size_t)nn * 3, sizeof(double)); /* dL/d v_i */
    double *bm = (double *)calloc((size_t)nn, sizeof(double));     /* dL/d m_i */
    double *bp = (double *)calloc((size_t)nn * 3, sizeof(double)); /* dL/d p_i */
    int st = ORC_ERR_OOM;
    if (!(gm && gp && gvg && bv && bm && bp)) goto done;

    /* forward recompute of the grid */
    st = orc_mpm_p2g(pr, n, x, v, C, F, gm, gp);
    if (st != ORC_OK) goto done;
    st = orc_mpm_grid_update(pr, gm, gp, &wind, t, gvg);
    if (st != ORC_OK) goto done;

    /* reverse G2P: scatter dL/dv_i; per-particle partials of x and F */
    for (int64_t p = 0; p < n; ++p) {
        double xp[3], Fp[9];
        load_particle(n, p, x, NULL, NULL, F, xp, NULL, NULL, Fp);
        stencil s;
        st = make_stencil(N, xp, &s);
        if (st != ORC_OK) goto done;
        /* recompute the G2P outputs v', C' */
        double vn[3] = {0, 0, 0}, Cn[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int oi = 0; oi < 3; ++oi)
            for (int oj = 0; oj < 3; ++oj)
                for (int ok = 0; ok < 3; ++ok) {
                    double W = s.w[0][oi] * s.w[1][oj] * s.w[2][ok];
                    double dpos[3] = {(oi - s.fx[0]) * dx, (oj - s.fx[1]) * dx, (ok - s.fx[2]) * dx};
                    int64_t id = node_index(N, s.base[0] + oi, s.base[1] + oj, s.base[2] + ok);
                    for (int a = 0; a < 3; ++a) {
                        double va = gvg[a * nn + id];
                        vn[a] += W * va;
                        for (int b = 0; b < 3; ++b) Cn[3 * a + b] += D * W * va * dpos[b];
                    }
                }
        int pin = pinned && pinned[p];
        if (pin) {
            memset(vn, 0, sizeof vn);
            memset(Cn, 0, sizeof Cn);
        }
        double bxo[3], bvo[3], bCo[9], bFo[9];
        load_particle(n, p, gx_out, gv_out, gC_out, gF_out, bxo, bvo, bCo, bFo);
        /* F' = (I + dt C') F */
        double Mdt[9], MdtT[9], bFin[9], Ft[9], bFoFt[9];
        for (int k = 0; k < 9; ++k) Mdt[k] = pr->dt * Cn[k];
        Mdt[0] += 1.0;
        Mdt[4] += 1.0;
        Mdt[8] += 1.0;
        transpose3(Mdt, MdtT);
        matmul3(MdtT, bFo, bFin);
        transpose3(Fp, Ft);
        matmul3(bFo, Ft, bFoFt);
        double bCn[9], bvn[3];
        for (int k = 0; k < 9; ++k) bCn[k] = bCo[k] + pr->dt * bFoFt[k];
        for (int a = 0; a < 3; ++a) bvn[a] = bvo[a] + pr->dt * bxo[a]; /* x' = x + dt v' */
        if (pin) {
            memset(bvn, 0, sizeof bvn);
            memset(bCn, 0, sizeof bCn);
        }
        double bxp[3] = {bxo[0], bxo[1], bxo[2]};
        for (int oi = 0; oi < 3; ++oi)
            for (int oj = 0; oj < 3; ++oj)
                for (int ok = 0; ok < 3; ++ok) {
                    double W = s.w[0][oi] * s.w[1][oj] * s.w[2][ok];
                    double dpos[3] = {(oi - s.fx[0]) * dx, (oj - s.fx[1]) * dx, (ok - s.fx[2]) * dx};
                    int64_t id = node_index(N, s.base[0] + oi, s.base[1] + oj, s.base[2] + ok);
                    double vi[3] = {gvg[id], gvg[nn + id], gvg[2 * nn + id]};
                    double Cd[3], CtV[3];
                    for (int a = 0; a < 3; ++a) {
                        Cd[a] = 0.0;
                        CtV[a] = 0.0;
                        for (int b = 0; b < 3; ++b) {
                            Cd[a] += bCn[3 * a + b] * dpos[b];
                            CtV[a] += bCn[3 * b + a] * vi[b];
                        }
                    }
                    double bW = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        bv[a * nn + id] += W * bvn[a] + D * W * Cd[a];
                        bW += vi[a] * bvn[a] + D * vi[a] * Cd[a];
                    }
                    double gW[3];
                    weight_grad(N, &s, oi, oj, ok, gW);
                    for (int a = 0; a < 3; ++a) bxp[a] += -D * W * CtV[a] + bW * gW[a];
                }
        for (int a = 0; a < 3; ++a) gx[a * n + p] = bxp[a];
        for (int k = 0; k < 9; ++k) gF[k * n + p] = bFin[k];
    }

    /* reverse grid update: dL/dp_i, dL/dm_i, and the wind field */
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                int64_t id = node_index(N, i, j, k);
                if (!(gm[id] > 0.0) || in_sticky_band(N, pr->bc_band, i, j, k)) continue;
                double b[3] = {bv[id], bv[nn + id], bv[2 * nn + id]};
                double m = gm[id], pdotb = 0.0;
                for (int c = 0; c < 3; ++c) {
                    bp[c * nn + id] = b[c] / m;
                    pdotb += gp[c * nn + id] * b[c];
                }
                bm[id] = -pdotb / (m * m);
                if (g_wind) {
                    double xi[3] = {i * dx, j * dx, k * dx};
                    double ga[3] = {pr->dt * b[0], pr->dt * b[1], pr->dt * b[2]};
                    wind_sample_adjoint_one(&wind, xi, t, ga, g_wind);
                }
            }

    /* reverse P2G: gather the grid adjoint back to the particles */
    double gE_acc = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        double xp[3], vp[3], Cp[9], Fp[9];
        load_particle(n, p, x, v, C, F, xp, vp, Cp, Fp);
        stencil s;
        st = make_stencil(N, xp, &s);
        if (st != ORC_OK) goto done;
        double P[9], Ft[9], PFt[9], A[9];
        st = orc_stress(pr->material, Fp, mu, lam, P);
        if (st != ORC_OK) goto done;
        transpose3(Fp, Ft);
        matmul3(P, Ft, PFt);
        for (int k = 0; k < 9; ++k) A[k] = -kappa * PFt[k] + pr->p_mass * Cp[k];
        double bA[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, bvp[3] = {0, 0, 0};
        double bxp[3] = {gx[p], gx[n + p], gx[2 * n + p]};
        for (int oi = 0; oi < 3; ++oi)
            for (int oj = 0; oj < 3; ++oj)
                for (int ok = 0; ok < 3; ++ok) {
                    double W = s.w[0][oi] * s.w[1][oj] * s.w[2][ok];
                    double dpos[3] = {(oi - s.fx[0]) * dx, (oj - s.fx[1]) * dx, (ok - s.fx[2]) * dx};
                    int64_t id = node_index(N, s.base[0] + oi, s.base[1] + oj, s.base[2] + ok);
                    double bpi[3] = {bp[id], bp[nn + id], bp[2 * nn + id]};
                    double bW = pr->p_mass * bm[id];
                    double AtB[3] = {0, 0, 0};
                    for (int c = 0; c < 3; ++c) {
                        double mom = pr->p_mass * vp[c];
                        for (int b = 0; b < 3; ++b) mom += A[3 * c + b] * dpos[b];
                        bW += bpi[c] * mom;
                        bvp[c] += W * pr->p_mass * bpi[c];
                        for (int b = 0; b < 3; ++b) {
                            bA[3 * c + b] += W * bpi[c] * dpos[b];
                            AtB[b] += A[3 * c + b] * bpi[c];
                        }
                    }
                    double gW[3];
                    weight_grad(N, &s, oi, oj, ok, gW);
                    for (int a = 0; a < 3; ++a) bxp[a] += -W * AtB[a] + bW * gW[a];
                }
        /* A = -kappa P F^T + m C */
        double bP[9], bAt[9], bAtP[9], bAF[9];
        matmul3(bA, Fp, bAF);
        for (int k = 0; k < 9; ++k) bP[k] = -kappa * bAF[k];
        transpose3(bA, bAt);
        matmul3(bAt, P, bAtP);
        double bFp[9];
        for (int k = 0; k < 9; ++k) bFp[k] = gF[k * n + p] - kappa * bAtP[k];
        st = orc_stress_adjoint(pr->material, Fp, mu, lam, bP, bFp);
        if (st != ORC_OK) goto done;
        gE_acc += dot9(bP, P) / pr->E;
        for (int a = 0; a < 3; ++a) {
            gx[a * n + p] = bxp[a];
            gvp[a * n + p] = bvp[a];
        }
        for (int k = 0; k < 9; ++k) {
            gC[k * n + p] = pr->p_mass * bA[k];
            gF[k * n + p] = bFp[k];
        }
    }
    if (g_E) *g_E += gE_acc;
    st = ORC_OK;
done:
    free(gm);
    free(gp);
    free(gvg);
    free(bv);
    free(bm);
    free(bp);
    return st;
}

/* Grid-level views for the pins: P2G mass and momentum fields. */
int orc_mpm_p2g_grid(const orc_mpm_params *pr, int64_t n, const double *x, const double *v,
                     const double *C, const double *F, double *gm, double *gp) {
    return orc_mpm_p2g(pr, n, x, v, C, F, gm, gp);
}

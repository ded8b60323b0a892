/*
 * FP64 CPU oracle for the moment-encoded lattice Boltzmann step (HOME-LBM,
 * Sec. 3.4 and App. D of DiffWind, after Li et al. 2023) on the D3Q19 lattice.
 *
 * TEST INFRASTRUCTURE ONLY. Plain restatement used to check the CUDA path;
 * only tests/, the smoke check in __graft_entry__.py and bench.py's
 * cpu_baseline leg may load it. It shares no code, header or table with the
 * CUDA library.
 *
 * State per cell: ten moments (rho, u, S) with S_ab = sum_i H2_ab(c_i) f_i / rho,
 * H2_ab = c_a c_b - cs2 delta_ab, cs2 = 1/3, describing the post-collision
 * populations of the cell. Order: rho, ux, uy, uz, Sxx, Syy, Szz, Sxy, Sxz, Syz.
 *
 * Reconstruction (App. D): the Hermite series of the populations to second
 * order in full, plus the third-order terms the D3Q19 lattice carries,
 *   f_i = w_i rho [1 + c.u / cs2 + H2(c_i) : S / (2 cs2^2)
 *                  + sum over the six (a, a, b), a != b, of
 *                    H3_aab(c_i) A_aab / (2 cs2^3)],
 * H3_aab(c) = c_b (c_a^2 - cs2), and the third-order coefficient closed from
 * the lower moments as A_aab = u_b S_aa + 2 u_a S_ab - 2 u_a u_a u_b (the
 * general closure u_a S_bc + u_b S_ac + u_c S_ab - 2 u_a u_b u_c; it equals
 * the equilibrium value u_a u_a u_b when S = u u). H3_aaa and H3_xyz vanish
 * on every D3Q19 velocity. The printed listing pairs some H3 labels with the
 * wrong coefficients; the labels here follow the closure.
 *
 * Step: pull streaming f_i(x) = f_i^post(x - c_i) (each source population
 * reconstructed from the source cell's moments), with halfway bounce-back
 * (f_i(x) = f_opp(i)^post(x) when x - c_i is solid), periodic y and z, and in x
 * either periodic or an inlet at x = 0 (the reconstruction of rho = 1, u_in,
 * S = u_in u_in) and a zero-gradient outlet at x = nx - 1 (the cell's own
 * post-collision population). Then the collision in moment space, the image
 * of BGK with Guo forcing with the trace of the second moment relaxed at
 * rate 1 (the isotropic part of S is set to its equilibrium, as in the
 * printed diagonal update) and its deviatoric part at rate 1/tau:
 *   rho, j = sum c f, Pi = sum c c f of the streamed populations,
 *   u = (j + F/2) / rho, N = Pi - rho (cs2 I + u u), Phi = u F^T + F u^T,
 *   Pi' = rho (cs2 I + u u) + (1 - 1/tau) dev N + (1 - 1/(2 tau)) dev Phi
 *         + iso Phi / 2,
 *   stored: rho, u' = u + F / (2 rho), S' = Pi' / rho - cs2 I.
 * The printed diagonal update omits the equilibrium term (1/tau) dev(u u); it
 * is restored here (the off-diagonal update and every forcing term of the
 * printed update follow from the same formula). The macroscopic velocity is
 * u = u' - F / (2 rho). Solid cells keep their moments.
 *
 * Layout: m[k * ncell + cell], cell = (z * ny + y) * nx + x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 3

static const int hc[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, 0, 1},  {-1, 0, -1}, {0, 1, 1},  {0, -1, -1}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1}};

static const double CS2 = 1.0 / 3.0;

static double hw(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

static int hopp(int i) { return i == 0 ? 0 : ((i % 2) ? i + 1 : i - 1); }

/* the symmetric tensor S from the six stored components */
static void s_full(const double *m, double S[3][3]) {
    S[0][0] = m[4];
    S[1][1] = m[5];
    S[2][2] = m[6];
    S[0][1] = S[1][0] = m[7];
    S[0][2] = S[2][0] = m[8];
    S[1][2] = S[2][1] = m[9];
}

/* population i of the Hermite reconstruction of the moments m[10] */
static double reconstruct_one(const double *m, int i) {
    const double rho = m[0], u[3] = {m[1], m[2], m[3]};
    double S[3][3];
    s_full(m, S);
    const double c[3] = {hc[i][0], hc[i][1], hc[i][2]};
    double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
    double h2s = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) h2s += (c[a] * c[b] - (a == b ? CS2 : 0.0)) * S[a][b];
    double h3a = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            if (a == b) continue;
            double h3 = c[b] * (c[a] * c[a] - CS2);
            double A = u[b] * S[a][a] + 2.0 * u[a] * S[a][b] - 2.0 * u[a] * u[a] * u[b];
            h3a += h3 * A;
        }
    return hw(i) * rho *
           (1.0 + cu / CS2 + h2s / (2.0 * CS2 * CS2) + h3a / (2.0 * CS2 * CS2 * CS2));
}

void orc_home_reconstruct(const double *m, double *f /*[19]*/) {
    for (int i = 0; i < 19; ++i) f[i] = reconstruct_one(m, i);
}

/* collision in moment space: (rho, j, Pi) of the pre-collision populations
 * -> the stored moments m[10] */
static void collide_moments(double rho, const double j[3], double Pi[3][3], double tau,
                            const double F[3], double *m) {
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
    double N[3][3], Phi[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            N[a][b] = Pi[a][b] - rho * ((a == b ? CS2 : 0.0) + u[a] * u[b]);
            Phi[a][b] = u[a] * F[b] + F[a] * u[b];
        }
    double trN = (N[0][0] + N[1][1] + N[2][2]) / 3.0;
    double trP = (Phi[0][0] + Phi[1][1] + Phi[2][2]) / 3.0;
    double S[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double d = a == b ? 1.0 : 0.0;
            double pp = rho * (d * CS2 + u[a] * u[b]) + (1.0 - 1.0 / tau) * (N[a][b] - d * trN) +
                        (1.0 - 0.5 / tau) * (Phi[a][b] - d * trP) + 0.5 * d * trP;
            S[a][b] = pp / rho - d * CS2;
        }
    m[0] = rho;
    for (int a = 0; a < 3; ++a) m[1 + a] = u[a] + 0.5 * F[a] / rho;
    m[4] = S[0][0];
    m[5] = S[1][1];
    m[6] = S[2][2];
    m[7] = S[0][1];
    m[8] = S[0][2];
    m[9] = S[1][2];
}

static void moments_of(const double f[19], double *rho, double j[3], double Pi[3][3]) {
    *rho = 0.0;
    for (int a = 0; a < 3; ++a) {
        j[a] = 0.0;
        for (int b = 0; b < 3; ++b) Pi[a][b] = 0.0;
    }
    for (int i = 0; i < 19; ++i) {
        *rho += f[i];
        for (int a = 0; a < 3; ++a) {
            j[a] += hc[i][a] * f[i];
            for (int b = 0; b < 3; ++b) Pi[a][b] += hc[i][a] * hc[i][b] * f[i];
        }
    }
}

/* the collision applied to one cell's populations (exported for the pins) */
void orc_home_collide(const double *f, double tau, const double *force, double *m) {
    double rho, j[3], Pi[3][3];
    moments_of(f, &rho, j, Pi);
    collide_moments(rho, j, Pi, tau, force, m);
}

/* the stored moments of the equilibrium f_eq(rho0, u0) taken as the
 * pre-collision state (rho0, j = rho0 u0, Pi = rho0 (cs2 I + u0 u0)) */
void orc_home_init(int64_t ncell, double rho0, const double *u0, double tau, const double *force,
                   double *m) {
    double j[3], Pi[3][3], one[10];
    for (int a = 0; a < 3; ++a) {
        j[a] = rho0 * u0[a];
        for (int b = 0; b < 3; ++b) Pi[a][b] = rho0 * ((a == b ? CS2 : 0.0) + u0[a] * u0[b]);
    }
    collide_moments(rho0, j, Pi, tau, force, one);
    for (int64_t c = 0; c < ncell; ++c)
        for (int k = 0; k < 10; ++k) m[k * ncell + c] = one[k];
}

static int wrapi(int v, int n) { return ((v % n) + n) % n; }

static void load_cell(const double *m, int64_t nc, int64_t c, double *out) {
    for (int k = 0; k < 10; ++k) out[k] = m[k * nc + c];
}

/* Advance the moments m in place by `steps` steps. */
int orc_home_step(int nx, int ny, int nz, double tau, const double *u_in, const double *force,
                  int bc_x, const uint8_t *solid, double *m, int steps) {
    if (nx < 2 || ny < 1 || nz < 1 || !(tau > 0.5) || steps < 0) return ORC_ERR_ARG;
    int64_t nc = (int64_t)nx * ny * nz;
    double *mn = (double *)malloc(sizeof(double) * 10 * nc);
    if (!mn) return ORC_ERR_OOM;
    double m_in[10] = {1.0, u_in[0], u_in[1], u_in[2], u_in[0] * u_in[0], u_in[1] * u_in[1],
                       u_in[2] * u_in[2], u_in[0] * u_in[1], u_in[0] * u_in[2],
                       u_in[1] * u_in[2]};
    for (int s = 0; s < steps; ++s) {
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int64_t c = ((int64_t)z * ny + y) * nx + x;
                    if (solid && solid[c]) {
                        for (int k = 0; k < 10; ++k) mn[k * nc + c] = m[k * nc + c];
                        continue;
                    }
                    double own[10], f[19];
                    load_cell(m, nc, c, own);
                    for (int i = 0; i < 19; ++i) {
                        int sx = x - hc[i][0], sy = wrapi(y - hc[i][1], ny),
                            sz = wrapi(z - hc[i][2], nz);
                        if (bc_x == 1 && sx < 0) {
                            f[i] = reconstruct_one(m_in, i);
                        } else if (bc_x == 1 && sx > nx - 1) {
                            f[i] = reconstruct_one(own, i);
                        } else {
                            sx = wrapi(sx, nx);
                            int64_t src = ((int64_t)sz * ny + sy) * nx + sx;
                            if (solid && solid[src]) {
                                f[i] = reconstruct_one(own, hopp(i));
                            } else {
                                double ms[10];
                                load_cell(m, nc, src, ms);
                                f[i] = reconstruct_one(ms, i);
                            }
                        }
                    }
                    double one[10];
                    orc_home_collide(f, tau, force, one);
                    for (int k = 0; k < 10; ++k) mn[k * nc + c] = one[k];
                }
        memcpy(m, mn, sizeof(double) * 10 * nc);
    }
    free(mn);
    return ORC_OK;
}

/* rho[ncell] and the macroscopic velocity u[3][ncell] = u' - F / (2 rho);
 * solid cells report 0 */
void orc_home_macroscopic(int64_t ncell, const double *force, const uint8_t *solid,
                          const double *m, double *rho, double *u) {
    for (int64_t c = 0; c < ncell; ++c) {
        if (solid && solid[c]) {
            rho[c] = 0.0;
            for (int a = 0; a < 3; ++a) u[a * ncell + c] = 0.0;
            continue;
        }
        double r = m[c];
        rho[c] = r;
        for (int a = 0; a < 3; ++a) u[a * ncell + c] = m[(1 + a) * ncell + c] - 0.5 * force[a] / r;
    }
}

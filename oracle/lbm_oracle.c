/*
 * FP64 CPU oracle for the D3Q19 BGK lattice Boltzmann step of DiffWind and
 * for the particle-to-voxel obstacle mask.
 *
 * TEST INFRASTRUCTURE ONLY. Plain restatement used to check the CUDA path;
 * only tests/, the smoke check in __graft_entry__.py and bench.py's
 * cpu_baseline leg may load it. It shares no code, header or table with the
 * CUDA library.
 *
 * What it computes:
 *   - The lattice Boltzmann equation f_i(x + c_i, t + 1) - f_i(x, t) =
 *     Omega_i + F_oi (Eq. lbe, Sec. 3.1) with the BGK collision operator
 *     Omega_i = -(f_i - f_i^eq) / tau and, when a body force is given, Guo's
 *     forcing term; the moments rho = sum f_i and rho u = sum c_i f_i + F/2
 *     (Eq. lbm_sum_v2, read with the force term outside the sum).
 *   - Equilibrium f_i^eq = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u) for the
 *     D3Q19 lattice (c_s^2 = 1/3).
 *   - Streaming with halfway bounce-back on solid nodes, periodic y and z,
 *     and in x either periodic or an equilibrium inlet at x = 0 (incoming
 *     populations f^eq(1, u_in)) and a zero-gradient outlet at x = nx - 1
 *     (incoming populations copied from the node's own post-collision ones).
 *   - The solid mask of Eq. point2voxel: node w is solid iff some particle
 *     satisfies 0 <= x_p - x_w < dx on every axis, i.e. w = floor(x_p / dx).
 * Plus the hand-derived adjoint of the step (reverse streaming and the
 * transposed collision Jacobian), pinned in the tests by finite differences.
 *
 * Layout: f[q * ncell + cell], cell = (z * ny + y) * nx + x; solid[cell].
 * Velocity set order: rest; +x, -x, +y, -y, +z, -z; then the twelve edge
 * diagonals (+x+y), (-x-y), (+x+z), (-x-z), (+y+z), (-y-z), (+x-y), (-x+y),
 * (+x-z), (-x+z), (+y-z), (-y+z). Direction 2k-1 and 2k are opposite.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 3

static const int cvec[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, 0, 1},  {-1, 0, -1}, {0, 1, 1},  {0, -1, -1}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1}};

static double wq(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

static int opp(int i) { return i == 0 ? 0 : ((i % 2) ? i + 1 : i - 1); }

void orc_lbm_velocity_set(int *c /*[19][3]*/, double *w /*[19]*/, int *op /*[19]*/) {
    for (int i = 0; i < 19; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = cvec[i][a];
        w[i] = wq(i);
        op[i] = opp(i);
    }
}

void orc_lbm_equilibrium(double rho, const double u[3], double feq[19]) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double cu = cvec[i][0] * u[0] + cvec[i][1] * u[1] + cvec[i][2] * u[2];
        feq[i] = wq(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* rho and u of one node (Eq. lbm_sum_v2 with the half-force shift) */
static void moments(const double f[19], const double force[3], double *rho, double u[3]) {
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; ++i) {
        r += f[i];
        for (int a = 0; a < 3; ++a) m[a] += cvec[i][a] * f[i];
    }
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * force[a]) / r;
    *rho = r;
}

/* BGK collision with Guo forcing at one node */
static void collide(const double f[19], double tau, const double force[3], double fp[19]) {
    double rho, u[3], feq[19];
    moments(f, force, &rho, u);
    orc_lbm_equilibrium(rho, u, feq);
    double pre = 1.0 - 0.5 / tau;
    for (int i = 0; i < 19; ++i) {
        double cu = cvec[i][0] * u[0] + cvec[i][1] * u[1] + cvec[i][2] * u[2];
        double src = 0.0;
        for (int a = 0; a < 3; ++a) src += (3.0 * (cvec[i][a] - u[a]) + 9.0 * cu * cvec[i][a]) * force[a];
        fp[i] = f[i] - (f[i] - feq[i]) / tau + pre * wq(i) * src;
    }
}

/* transposed collision Jacobian: gpre = (d fpost / d f)^T gpost at state f */
static void collide_adjoint(const double f[19], double tau, const double force[3],
                            const double gpost[19], double gpre[19]) {
    double rho, u[3], feq[19];
    moments(f, force, &rho, u);
    orc_lbm_equilibrium(rho, u, feq);
    double pre = 1.0 - 0.5 / tau;
    double alpha = 0.0, beta[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; ++i) {
        double cu = cvec[i][0] * u[0] + cvec[i][1] * u[1] + cvec[i][2] * u[2];
        double cF = cvec[i][0] * force[0] + cvec[i][1] * force[1] + cvec[i][2] * force[2];
        alpha += gpost[i] * feq[i];
        for (int a = 0; a < 3; ++a) {
            double dfeq = wq(i) * rho * (3.0 * cvec[i][a] + 9.0 * cu * cvec[i][a] - 3.0 * u[a]);
            double dsrc = pre * wq(i) * (-3.0 * force[a] + 9.0 * cF * cvec[i][a]);
            beta[a] += gpost[i] * (dfeq / tau + dsrc);
        }
    }
    alpha /= (tau * rho);
    for (int j = 0; j < 19; ++j) {
        double bc = 0.0;
        for (int a = 0; a < 3; ++a) bc += beta[a] * (cvec[j][a] - u[a]);
        gpre[j] = (1.0 - 1.0 / tau) * gpost[j] + alpha + bc / rho;
    }
}

typedef struct {
    int nx, ny, nz;
    double tau;
    double u_in[3];
    double force[3];
    int bc_x; /* 0 periodic, 1 equilibrium inlet at x = 0 and zero-gradient outlet */
} lat;

static int64_t cell_of(const lat *L, int x, int y, int z) {
    return ((int64_t)z * L->ny + y) * L->nx + x;
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* one collide + stream step; f (pre-collision at t) -> fn (pre-collision at t+1) */
static void step_once(const lat *L, const uint8_t *solid, const double *f, double *fp, double *fn) {
    int64_t nc = (int64_t)L->nx * L->ny * L->nz;
    double feq_in[19];
    orc_lbm_equilibrium(1.0, L->u_in, feq_in);
    for (int64_t c = 0; c < nc; ++c) {
        double fl[19], po[19];
        for (int i = 0; i < 19; ++i) fl[i] = f[i * nc + c];
        if (solid && solid[c]) {
            memcpy(po, fl, sizeof po);
        } else {
            collide(fl, L->tau, L->force, po);
        }
        for (int i = 0; i < 19; ++i) fp[i * nc + c] = po[i];
    }
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                int64_t c = cell_of(L, x, y, z);
                if (solid && solid[c]) {
                    for (int i = 0; i < 19; ++i) fn[i * nc + c] = f[i * nc + c];
                    continue;
                }
                for (int i = 0; i < 19; ++i) {
                    int sx = x - cvec[i][0], sy = wrap(y - cvec[i][1], L->ny),
                        sz = wrap(z - cvec[i][2], L->nz);
                    double val;
                    if (L->bc_x == 1 && sx < 0) {
                        val = feq_in[i];
                    } else if (L->bc_x == 1 && sx > L->nx - 1) {
                        val = fp[i * nc + c];
                    } else {
                        sx = wrap(sx, L->nx);
                        int64_t s = cell_of(L, sx, sy, sz);
                        if (solid && solid[s])
                            val = fp[opp(i) * nc + c];
                        else
                            val = fp[i * nc + s];
                    }
                    fn[i * nc + c] = val;
                }
            }
}

/* Advance f in place by `steps` lattice steps. */
int orc_lbm_step(int nx, int ny, int nz, double tau, const double *u_in, const double *force,
                 int bc_x, const uint8_t *solid, double *f, int steps) {
    if (nx < 2 || ny < 1 || nz < 1 || !(tau > 0.5) || steps < 0) return ORC_ERR_ARG;
    lat L = {nx, ny, nz, tau, {u_in[0], u_in[1], u_in[2]}, {force[0], force[1], force[2]}, bc_x};
    int64_t nc = (int64_t)nx * ny * nz;
    double *fp = (double *)malloc(sizeof(double) * 19 * nc);
    double *fn = (double *)malloc(sizeof(double) * 19 * nc);
    if (!fp || !fn) {
        free(fp);
        free(fn);
        return ORC_ERR_OOM;
    }
    for (int s = 0; s < steps; ++s) {
        step_once(&L, solid, f, fp, fn);
        memcpy(f, fn, sizeof(double) * 19 * nc);
    }
    free(fp);
    free(fn);
    return ORC_OK;
}

/* Reverse mode of orc_lbm_step. f0 is the state the forward started from;
 * g holds dL/df(t + steps) on entry and dL/df(t) on return. */
int orc_lbm_step_adjoint(int nx, int ny, int nz, double tau, const double *u_in,
                         const double *force, int bc_x, const uint8_t *solid, const double *f0,
                         double *g, int steps) {
    if (nx < 2 || ny < 1 || nz < 1 || !(tau > 0.5) || steps < 0) return ORC_ERR_ARG;
    lat L = {nx, ny, nz, tau, {u_in[0], u_in[1], u_in[2]}, {force[0], force[1], force[2]}, bc_x};
    int64_t nc = (int64_t)nx * ny * nz;
    size_t sz = sizeof(double) * 19 * (size_t)nc;
    double *hist = (double *)malloc(sz * (size_t)(steps > 0 ? steps : 1));
    double *fp = (double *)malloc(sz);
    double *gp = (double *)malloc(sz);
    if (!hist || !fp || !gp) {
        free(hist);
        free(fp);
        free(gp);
        return ORC_ERR_OOM;
    }
    if (steps > 0) memcpy(hist, f0, sz);
    for (int s = 1; s < steps; ++s) step_once(&L, solid, hist + (size_t)(s - 1) * 19 * nc, fp, hist + (size_t)s * 19 * nc);
    for (int s = steps - 1; s >= 0; --s) {
        const double *fs = hist + (size_t)s * 19 * nc;
        /* reverse streaming: gp_i(y) collects every read of fpost_i(y) */
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int64_t c = cell_of(&L, x, y, z);
                    if (solid && solid[c]) continue;
                    for (int i = 0; i < 19; ++i) {
                        double acc = 0.0;
                        int tx = x + cvec[i][0], ty = wrap(y + cvec[i][1], ny),
                            tz = wrap(z + cvec[i][2], nz);
                        int inside = 1;
                        if (bc_x == 1 && (tx < 0 || tx > nx - 1)) inside = 0;
                        if (inside) {
                            tx = wrap(tx, nx);
                            int64_t t = cell_of(&L, tx, ty, tz);
                            if (solid && solid[t])
                                acc += g[opp(i) * nc + c]; /* bounced back into y as opp(i) */
                            else
                                acc += g[i * nc + t];
                        }
                        if (bc_x == 1 && x - cvec[i][0] > nx - 1) acc += g[i * nc + c]; /* outlet copy */
                        gp[i * nc + c] = acc;
                    }
                }
        /* transposed collision */
        for (int64_t c = 0; c < nc; ++c) {
            if (solid && solid[c]) continue; /* solid populations pass through unchanged */
            double fl[19], go[19], gi[19];
            for (int i = 0; i < 19; ++i) {
                fl[i] = fs[i * nc + c];
                go[i] = gp[i * nc + c];
            }
            collide_adjoint(fl, tau, L.force, go, gi);
            for (int i = 0; i < 19; ++i) g[i * nc + c] = gi[i];
        }
    }
    free(hist);
    free(fp);
    free(gp);
    return ORC_OK;
}

/* rho[ncell] and u[3][ncell] by Eq. lbm_sum_v2; solid nodes report rho = 0, u = 0 */
void orc_lbm_macroscopic(int nx, int ny, int nz, const double *force, const uint8_t *solid,
                         const double *f, double *rho, double *u) {
    int64_t nc = (int64_t)nx * ny * nz;
    for (int64_t c = 0; c < nc; ++c) {
        if (solid && solid[c]) {
            rho[c] = 0.0;
            u[c] = u[nc + c] = u[2 * nc + c] = 0.0;
            continue;
        }
        double fl[19], r, uu[3];
        for (int i = 0; i < 19; ++i) fl[i] = f[i * nc + c];
        moments(fl, force, &r, uu);
        rho[c] = r;
        for (int a = 0; a < 3; ++a) u[a * nc + c] = uu[a];
    }
}

/* single-node collision, exported for the pins */
void orc_lbm_collide(const double *f, double tau, const double *force, double *fpost) {
    collide(f, tau, force, fpost);
}

void orc_lbm_collide_adjoint(const double *f, double tau, const double *force,
                             const double *gpost, double *gpre) {
    collide_adjoint(f, tau, force, gpost, gpre);
}

/* Eq. point2voxel: solid[cell] = 1 iff a particle lies in [x_w, x_w + dx)^3.
 * The mask is cleared first. pos is [3][n]. */
void orc_voxelize(const double *pos, int64_t n, int nx, int ny, int nz, double dx, uint8_t *solid) {
    int64_t nc = (int64_t)nx * ny * nz;
    memset(solid, 0, (size_t)nc);
    for (int64_t p = 0; p < n; ++p) {
        double q[3] = {pos[p], pos[n + p], pos[2 * n + p]};
        int w[3], dims[3] = {nx, ny, nz}, ok = 1;
        for (int a = 0; a < 3; ++a) {
            double s = floor(q[a] / dx);
            if (!(s >= 0.0 && s < (double)dims[a])) ok = 0;
            w[a] = ok ? (int)s : 0;
        }
        if (ok) solid[((int64_t)w[2] * ny + w[1]) * nx + w[0]] = 1;
    }
}

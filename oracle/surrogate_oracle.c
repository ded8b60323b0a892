/*
 * FP64 CPU oracle for the learned wind-constraint surrogate: a 4-layer 3D
 * convolutional network on a coarse n^3 grid (channels 16 -> 32 -> 32 -> 32
 * -> 16, kernel 3, zero padding, GELU after the first three layers), its
 * reverse mode, the coarse features taken from an LBM lattice, and the
 * upsample + re-equilibration back onto the lattice.
 *
 * TEST INFRASTRUCTURE ONLY. Plain direct sums in FP64 that the CUDA path is
 * checked against; only tests/, the smoke check and bench.py's cpu_baseline
 * leg may load it. It shares no code with the CUDA library.
 *
 * The paper has no learned component; the network is the surrogate of the
 * LBM wind constraint (Sec. 3.4 uses the LBM velocity as the guide) that
 * advances the velocity field by a block of lattice steps at once.
 *
 * Layouts (the same the C-ABI documents):
 *   activations channels-last: a[((z*n + y)*n + x)*C + c]
 *   layer weights W[tap][co][ci], tap = (dz+1)*9 + (dy+1)*3 + (dx+1), the
 *   input voxel of output voxel v at tap (dx,dy,dz) being v + (dx,dy,dz);
 *   parameters packed layer by layer as W then bias[co].
 *   GELU(z) = z * Phi(z) = 0.5 z (1 + erf(z / sqrt 2)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const int CH[5] = {16, 32, 32, 32, 16};
static const double PI = 3.14159265358979323846;

int64_t orc_surr_num_params(void) {
    int64_t s = 0;
    for (int l = 0; l < 4; ++l) s += 27LL * CH[l] * CH[l + 1] + CH[l + 1];
    return s;
}

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }

static double gelu_grad(double z) {
    return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * PI);
}

/* out[v][co] = b[co] + sum_{tap, ci} W[tap][co][ci] in[v + tap][ci] (zero outside) */
static void conv3(int n, int cin, int cout, const double *W, const double *b, const double *in,
                  double *out) {
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                double *o = out + (((int64_t)z * n + y) * n + x) * cout;
                for (int co = 0; co < cout; ++co) o[co] = b ? b[co] : 0.0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int sx = x + dx, sy = y + dy, sz = z + dz;
                            if (sx < 0 || sy < 0 || sz < 0 || sx >= n || sy >= n || sz >= n) continue;
                            int tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                            const double *a = in + (((int64_t)sz * n + sy) * n + sx) * cin;
                            for (int co = 0; co < cout; ++co) {
                                const double *w = W + ((int64_t)tap * cout + co) * cin;
                                double s = 0.0;
                                for (int ci = 0; ci < cin; ++ci) s += w[ci] * a[ci];
                                o[co] += s;
                            }
                        }
            }
}

/* Forward pass. feats [n^3][16]; z_out / a_out (optional) receive, layer by
 * layer, the pre-activations and activations of layers 1..3 ([3][n^3][32]);
 * out [n^3][16] is the last layer's output (channels 0..2 carry du). */
void orc_surr_forward(int n, const double *params, const double *feats, double *z_out,
                      double *a_out, double *out) {
    int64_t nv = (int64_t)n * n * n;
    const double *cur = feats;
    double *bufz = (double *)malloc(sizeof(double) * nv * 32);
    double *bufa[2] = {(double *)malloc(sizeof(double) * nv * 32),
                       (double *)malloc(sizeof(double) * nv * 32)};
    const double *p = params;
    for (int l = 0; l < 4; ++l) {
        int cin = CH[l], cout = CH[l + 1];
        const double *W = p;
        const double *b = p + 27LL * cin * cout;
        p = b + cout;
        if (l < 3) {
            conv3(n, cin, cout, W, b, cur, bufz);
            double *a = bufa[l & 1];
            for (int64_t i = 0; i < nv * cout; ++i) a[i] = gelu(bufz[i]);
            if (z_out) memcpy(z_out + (int64_t)l * nv * 32, bufz, sizeof(double) * nv * 32);
            if (a_out) memcpy(a_out + (int64_t)l * nv * 32, a, sizeof(double) * nv * 32);
            cur = a;
        } else {
            conv3(n, cin, cout, W, b, cur, out);
        }
    }
    free(bufz);
    free(bufa[0]);
    free(bufa[1]);
}

/* Reverse mode: given g_out = dL/d(out) [n^3][16], accumulates dL/dparams
 * into g_params (same packing as params). */
void orc_surr_backward(int n, const double *params, const double *feats, const double *g_out,
                       double *g_params) {
    int64_t nv = (int64_t)n * n * n;
    double *z = (double *)malloc(sizeof(double) * 3 * nv * 32);
    double *a = (double *)malloc(sizeof(double) * 3 * nv * 32);
    double *out = (double *)malloc(sizeof(double) * nv * 16);
    orc_surr_forward(n, params, feats, z, a, out);
    /* offsets of each layer's parameters */
    int64_t off[4], o = 0;
    for (int l = 0; l < 4; ++l) {
        off[l] = o;
        o += 27LL * CH[l] * CH[l + 1] + CH[l + 1];
    }
    double *g = (double *)malloc(sizeof(double) * nv * 32);  /* dL/dz of the current layer */
    double *gin = (double *)malloc(sizeof(double) * nv * 32); /* dL/d(input) */
    memcpy(g, g_out, sizeof(double) * nv * 16);
    for (int l = 3; l >= 0; --l) {
        int cin = CH[l], cout = CH[l + 1];
        const double *W = params + off[l];
        double *gW = g_params + off[l];
        double *gb = gW + 27LL * cin * cout;
        const double *in = l == 0 ? feats : a + (int64_t)(l - 1) * nv * 32;
        /* parameter gradients */
        for (int z0 = 0; z0 < n; ++z0)
            for (int y0 = 0; y0 < n; ++y0)
                for (int x0 = 0; x0 < n; ++x0) {
                    const double *gv = g + (((int64_t)z0 * n + y0) * n + x0) * cout;
                    for (int co = 0; co < cout; ++co) gb[co] += gv[co];
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int sx = x0 + dx, sy = y0 + dy, sz = z0 + dz;
                                if (sx < 0 || sy < 0 || sz < 0 || sx >= n || sy >= n || sz >= n) continue;
                                int tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                                const double *av = in + (((int64_t)sz * n + sy) * n + sx) * cin;
                                for (int co = 0; co < cout; ++co)
                                    for (int ci = 0; ci < cin; ++ci)
                                        gW[((int64_t)tap * cout + co) * cin + ci] += gv[co] * av[ci];
                            }
                }
        if (l == 0) break;
        /* input gradient: gin[u][ci] = sum_{tap, co} W[tap][co][ci] g[u - tap][co] */
        memset(gin, 0, sizeof(double) * nv * cin);
        for (int z0 = 0; z0 < n; ++z0)
            for (int y0 = 0; y0 < n; ++y0)
                for (int x0 = 0; x0 < n; ++x0) {
                    const double *gv = g + (((int64_t)z0 * n + y0) * n + x0) * cout;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int sx = x0 + dx, sy = y0 + dy, sz = z0 + dz;
                                if (sx < 0 || sy < 0 || sz < 0 || sx >= n || sy >= n || sz >= n) continue;
                                int tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                                double *gi = gin + (((int64_t)sz * n + sy) * n + sx) * cin;
                                for (int co = 0; co < cout; ++co) {
                                    const double *w = W + ((int64_t)tap * cout + co) * cin;
                                    for (int ci = 0; ci < cin; ++ci) gi[ci] += w[ci] * gv[co];
                                }
                            }
                }
        /* through the GELU of the previous layer */
        const double *zp = z + (int64_t)(l - 1) * nv * 32;
        for (int64_t i = 0; i < nv * cin; ++i) g[i] = gin[i] * gelu_grad(zp[i]);
    }
    free(z);
    free(a);
    free(out);
    free(g);
    free(gin);
}

static const int CV[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, 0, 1},  {-1, 0, -1}, {0, 1, 1},  {0, -1, -1}, {1, -1, 0},
    {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1}};

/* Coarse features of a fine lattice of 2n^3 cells (plain populations f[19][cells]):
 * per coarse voxel, the 2x2x2 average of rho - 1 over its fluid cells, the
 * average of u over its fluid cells minus the reference velocity uref
 * (0 when the voxel has no fluid cell), the solid fraction, and uref itself
 * in channels 5..7; channels 8..15 are zero. Also returns the fine rho and u
 * (solid cells: rho = 1, u = 0). */
void orc_surr_features(int n, const double *f, const uint8_t *solid, const double *uref,
                       double *feats, double *rho_fine, double *u_fine) {
    int N = 2 * n;
    int64_t nc = (int64_t)N * N * N;
    for (int64_t c = 0; c < nc; ++c) {
        double r = 0.0, m[3] = {0.0, 0.0, 0.0};
        if (!(solid && solid[c])) {
            for (int i = 0; i < 19; ++i) {
                double fi = f[i * nc + c];
                r += fi;
                for (int a = 0; a < 3; ++a) m[a] += CV[i][a] * fi;
            }
            rho_fine[c] = r;
            for (int a = 0; a < 3; ++a) u_fine[a * nc + c] = m[a] / r;
        } else {
            rho_fine[c] = 1.0;
            for (int a = 0; a < 3; ++a) u_fine[a * nc + c] = 0.0;
        }
    }
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                double s[4] = {0, 0, 0, 0};
                int fluid = 0;
                for (int k = 0; k < 8; ++k) {
                    int fx = 2 * x + (k & 1), fy = 2 * y + ((k >> 1) & 1), fz = 2 * z + (k >> 2);
                    int64_t c = ((int64_t)fz * N + fy) * N + fx;
                    if (solid && solid[c]) continue;
                    ++fluid;
                    s[0] += rho_fine[c] - 1.0;
                    for (int a = 0; a < 3; ++a) s[1 + a] += u_fine[a * nc + c];
                }
                double *o = feats + (((int64_t)z * n + y) * n + x) * 16;
                for (int ch = 0; ch < 16; ++ch) o[ch] = 0.0;
                if (fluid > 0) {
                    o[0] = s[0] / fluid;
                    for (int a = 0; a < 3; ++a) o[1 + a] = s[1 + a] / fluid - uref[a];
                }
                o[4] = (8 - fluid) / 8.0;
                for (int a = 0; a < 3; ++a) o[5 + a] = uref[a];
            }
}

/* Coarse-to-fine trilinear upsampling of du [n^3][16] (channels 0..2), the
 * fine cell i sitting at coarse coordinate i/2 - 1/4 (cell-centred, clamped),
 * and re-equilibration f = f_eq(rho, u + du) on fluid cells (solid cells keep
 * f). f is [19][cells] plain populations, overwritten. */
void orc_surr_apply(int n, const double *du, const double *rho_fine, const double *u_fine,
                    const uint8_t *solid, double *f) {
    int N = 2 * n;
    int64_t nc = (int64_t)N * N * N;
    for (int fz = 0; fz < N; ++fz)
        for (int fy = 0; fy < N; ++fy)
            for (int fx = 0; fx < N; ++fx) {
                int64_t c = ((int64_t)fz * N + fy) * N + fx;
                if (solid && solid[c]) continue;
                int i0[3];
                double t[3];
                int fi[3] = {fx, fy, fz};
                for (int a = 0; a < 3; ++a) {
                    double s = fi[a] * 0.5 - 0.25;
                    if (s < 0.0) s = 0.0;
                    if (s > n - 1) s = n - 1;
                    int i = (int)floor(s);
                    if (i > n - 2) i = n - 2;
                    i0[a] = i;
                    t[a] = s - i;
                }
                double d[3] = {0, 0, 0};
                for (int k = 0; k < 8; ++k) {
                    int cx = k & 1, cy = (k >> 1) & 1, cz = k >> 2;
                    double w = (cx ? t[0] : 1 - t[0]) * (cy ? t[1] : 1 - t[1]) * (cz ? t[2] : 1 - t[2]);
                    const double *v = du + ((((int64_t)(i0[2] + cz)) * n + (i0[1] + cy)) * n + (i0[0] + cx)) * 16;
                    for (int a = 0; a < 3; ++a) d[a] += w * v[a];
                }
                double u[3], rho = rho_fine[c];
                for (int a = 0; a < 3; ++a) u[a] = u_fine[a * nc + c] + d[a];
                double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                for (int i = 0; i < 19; ++i) {
                    double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
                    double w = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
                    f[i * nc + c] = w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
                }
            }
}

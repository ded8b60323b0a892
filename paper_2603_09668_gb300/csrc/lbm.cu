// D3Q19 BGK lattice Boltzmann step (Eq. lbe, moments of Eq. lbm_sum_v2), its
// reverse mode, macroscopic fields and the particle-to-voxel mask
// (Eq. point2voxel).
//
// Forward steps run in pairs as the in-place AA pattern on one lattice:
//   even kernel: read the natural slots of the own cell, collide, write each
//                post-collision population f*_i into the own cell's opposite
//                slot (no neighbour access);
//   odd kernel:  pull f_i from slot opp(i) of cell x - c_i, collide, push the
//                result into slot i of cell x + c_i, which leaves the lattice
//                in natural order again.
// Every (cell, slot) pair read by the odd kernel is written only by the same
// thread, which makes the update race-free in place. Boundary handling folded
// into the two kernels:
//   solid neighbour  -> halfway bounce-back (own cell's opposite population);
//   beyond x = 0     -> inlet equilibrium f_eq(1, u_inlet) (bc_x = 1);
//   beyond x = nx-1  -> the own post-collision population of the same
//                       direction; the even kernel saves those five values of
//                       the outlet face in a side buffer so that the odd kernel
//                       does not read a slot its upstream neighbour pushes into.
// Populations are stored shifted, f_i - w_i, for float32 resolution.
#include <stdio.h>

#include <new>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace dw {

// D3Q19 velocity set; with the loops unrolled every lookup folds to a constant.
struct D3Q19 {
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    __host__ __device__ static constexpr float w(int i) {
        return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
    }
};

// Directions leaving through -x (c_x = -1) in slot order of the outlet side buffer.
__host__ __device__ constexpr int outlet_slot(int i) {
    return i == 2 ? 0 : i == 8 ? 1 : i == 10 ? 2 : i == 14 ? 3 : i == 16 ? 4 : -1;
}

struct LbmParams {
    int nx, ny, nz;
    int ncell;
    float inv_tau;
    float pre;         // 1 - 1/(2 tau), Guo forcing prefactor
    float Fx, Fy, Fz;  // body force
    int has_force;
    int bc_x;
    float feq_in[19];  // shifted inlet equilibrium f_eq(1, u_inlet) - w
};

// Cell of this thread in a lattice-row launch (lattice_launch): x from the
// block's position along the row, y and z from the block indices, so that
// no division is needed; false past the end of the row.
__device__ __forceinline__ bool lattice_cell(const LbmParams &L, int &x, int &y, int &z, int &cell) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y;
    z = blockIdx.z;
    cell = (z * L.ny + y) * L.nx + x;
    return x < L.nx;
}

// BGK collision (+ Guo forcing) of one node, shifted populations, in place.
__device__ __forceinline__ void collide(const LbmParams &L, float f[19]) {
    float rs = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        rs += f[i];
        jx += (float)D3Q19::cx(i) * f[i];
        jy += (float)D3Q19::cy(i) * f[i];
        jz += (float)D3Q19::cz(i) * f[i];
    }
    float rho = 1.0f + rs;
    float inv_rho = 1.0f / rho;
    float ux = (jx + 0.5f * L.Fx) * inv_rho, uy = (jy + 0.5f * L.Fy) * inv_rho,
          uz = (jz + 0.5f * L.Fz) * inv_rho;
    float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        float cu = (float)D3Q19::cx(i) * ux + (float)D3Q19::cy(i) * uy + (float)D3Q19::cz(i) * uz;
        float feq = D3Q19::w(i) * (rs + rho * (3.0f * cu + 4.5f * cu * cu - uu));
        float fi = f[i] - (f[i] - feq) * L.inv_tau;
        if (L.has_force) {
            float cF = (float)D3Q19::cx(i) * L.Fx + (float)D3Q19::cy(i) * L.Fy + (float)D3Q19::cz(i) * L.Fz;
            float uF = ux * L.Fx + uy * L.Fy + uz * L.Fz;
            fi += L.pre * D3Q19::w(i) * (3.0f * (cF - uF) + 9.0f * cu * cF);
        }
        f[i] = fi;
    }
}

// Transposed collision Jacobian at state f: g <- (d f* / d f)^T g.
__device__ __forceinline__ void collide_adjoint(const LbmParams &L, const float f[19], float g[19]) {
    float rs = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        rs += f[i];
        jx += (float)D3Q19::cx(i) * f[i];
        jy += (float)D3Q19::cy(i) * f[i];
        jz += (float)D3Q19::cz(i) * f[i];
    }
    float rho = 1.0f + rs;
    float inv_rho = 1.0f / rho;
    float u[3] = {(jx + 0.5f * L.Fx) * inv_rho, (jy + 0.5f * L.Fy) * inv_rho,
                  (jz + 0.5f * L.Fz) * inv_rho};
    float uu = 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    float alpha = 0.0f, beta[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        float c[3] = {(float)D3Q19::cx(i), (float)D3Q19::cy(i), (float)D3Q19::cz(i)};
        float cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        float feq = D3Q19::w(i) * rho * (1.0f + 3.0f * cu + 4.5f * cu * cu - uu);
        alpha += g[i] * feq;
        float cF = c[0] * L.Fx + c[1] * L.Fy + c[2] * L.Fz;
        float F3[3] = {L.Fx, L.Fy, L.Fz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float dfeq = D3Q19::w(i) * rho * (3.0f * c[a] + 9.0f * cu * c[a] - 3.0f * u[a]);
            float dsrc = L.pre * D3Q19::w(i) * (-3.0f * F3[a] + 9.0f * cF * c[a]);
            beta[a] += g[i] * (dfeq * L.inv_tau + dsrc);
        }
    }
    alpha *= L.inv_tau * inv_rho;
#pragma unroll
    for (int j = 0; j < 19; ++j) {
        float bc = beta[0] * ((float)D3Q19::cx(j) - u[0]) + beta[1] * ((float)D3Q19::cy(j) - u[1]) +
                   beta[2] * ((float)D3Q19::cz(j) - u[2]);
        g[j] = (1.0f - L.inv_tau) * g[j] + alpha + bc * inv_rho;
    }
}

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ int cell_index(const LbmParams &L, int x, int y, int z) {
    return (z * L.ny + y) * L.nx + x;
}

// ---------------------------------------------------------------- forward --

__global__ void __launch_bounds__(256, 5) k_lbm_aa_even(LbmParams L, float *f,
                                                    const uint8_t *__restrict__ solid,
                                                    float *__restrict__ outlet) {
    pdl_wait();  // every thread, before anything of the previous step is touched
    pdl_trigger();
    int x, y, z, cell;
    if (!lattice_cell(L, x, y, z, cell)) return;
    if (solid && solid[cell]) return;
    const int nc = L.ncell;  // 19 * ncell < 2^31 is checked at create
    float fl[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = f[i * nc + cell];
    collide(L, fl);
#pragma unroll
    for (int i = 0; i < 19; ++i) f[D3Q19::opp(i) * nc + cell] = fl[i];
    if (L.bc_x == 1) {
        if (x == L.nx - 1) {
            int face = z * L.ny + y;
            int nface = L.ny * L.nz;
#pragma unroll
            for (int i = 0; i < 19; ++i)
                if (outlet_slot(i) >= 0) outlet[outlet_slot(i) * nface + face] = fl[i];
        }
    }
}

// Offsets of the neighbours with the periodic wraps folded in: the neighbour
// x + c is cell + off(c) (m = -1 side, p = +1 side of each axis).
struct NbrOffsets {
    int xm, xp, ym, yp, zm, zp;
    __device__ __forceinline__ int off(int cx, int cy, int cz) const {
        return (cx < 0 ? xm : (cx > 0 ? xp : 0)) + (cy < 0 ? ym : (cy > 0 ? yp : 0)) +
               (cz < 0 ? zm : (cz > 0 ? zp : 0));
    }
};

__device__ __forceinline__ NbrOffsets nbr_offsets(const LbmParams &L, int x, int y, int z) {
    NbrOffsets o;
    const int sy = L.nx, sz = L.nx * L.ny;
    o.xm = x == 0 ? L.nx - 1 : -1;
    o.xp = x == L.nx - 1 ? -(L.nx - 1) : 1;
    o.ym = y == 0 ? (L.ny - 1) * sy : -sy;
    o.yp = y == L.ny - 1 ? -(L.ny - 1) * sy : sy;
    o.zm = z == 0 ? (L.nz - 1) * sz : -sz;
    o.zp = z == L.nz - 1 ? -(L.nz - 1) * sz : sz;
    return o;
}

// Per-cell link mask for the odd kernel: bit 0 = the cell is solid, bit i =
// the neighbour x + c_i (after the periodic wraps) is solid, so that the
// kernels read 4 bytes instead of 18 masks. Lattice-row launch: the 19 mask
// bytes of a cell come from three rows of three planes, shared by the
// neighbouring threads through L1.
__global__ void __launch_bounds__(256) k_lbm_links(LbmParams L, const uint8_t *__restrict__ solid,
                                                   uint32_t *__restrict__ links) {
    pdl_wait();  // the mask may come from the previous kernel (voxelize)
    pdl_trigger();
    int x, y, z, cell;
    if (!lattice_cell(L, x, y, z, cell)) return;
    const NbrOffsets o = nbr_offsets(L, x, y, z);
    uint32_t m = solid[cell] ? 1u : 0u;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int cx = D3Q19::cx(i);
        if (L.bc_x == 1 && ((cx < 0 && x == 0) || (cx > 0 && x == L.nx - 1))) continue;  // no solid bit outside
        if (solid[cell + o.off(cx, D3Q19::cy(i), D3Q19::cz(i))]) m |= 1u << i;
    }
    links[cell] = m;
}

__global__ void __launch_bounds__(256, 5) k_lbm_aa_odd(LbmParams L, float *f,
                                                      const uint32_t *__restrict__ links,
                                                      const float *__restrict__ outlet) {
    pdl_wait();
    pdl_trigger();
    int x, y, z, cell;
    if (!lattice_cell(L, x, y, z, cell)) return;
    const uint32_t lk = links ? links[cell] : 0u;
    if (lk & 1u) return;
    const int nc = L.ncell;  // 19 * ncell < 2^31 is checked at create
    const NbrOffsets o = nbr_offsets(L, x, y, z);
    float fl[19];
    fl[0] = f[cell];  // rest population: own slot 0 in both orders
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int j = D3Q19::opp(i);  // f_i arrives from x + c_j, stored in its slot j
        const int idx = ((lk >> j) & 1u)
                            ? i * nc + cell  // bounce-back: own f*_j, in slot i since the even step
                            : j * nc + cell + o.off(D3Q19::cx(j), D3Q19::cy(j), D3Q19::cz(j));
        fl[i] = f[idx];
    }
    if (L.bc_x == 1) {
        const int nface = L.ny * L.nz, face = z * L.ny + y;
        if (x == 0) {
#pragma unroll
            for (int i = 1; i < 19; ++i)
                if (D3Q19::cx(i) == 1) fl[i] = L.feq_in[i];
        }
        if (x == L.nx - 1) {
#pragma unroll
            for (int i = 1; i < 19; ++i)
                if (D3Q19::cx(i) == -1) fl[i] = outlet[outlet_slot(i) * nface + face];
        }
    }
    collide(L, fl);
    f[cell] = fl[0];
    const bool inlet_face = L.bc_x == 1 && x == 0, outlet_face = L.bc_x == 1 && x == L.nx - 1;
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        if (inlet_face && D3Q19::cx(i) == -1) continue;   // leaves through x = 0
        if (outlet_face && D3Q19::cx(i) == 1) continue;   // leaves through x = nx - 1
        const int idx = ((lk >> i) & 1u)
                            ? D3Q19::opp(i) * nc + cell
                            : i * nc + cell + o.off(D3Q19::cx(i), D3Q19::cy(i), D3Q19::cz(i));
        f[idx] = fl[i];
    }
    if (inlet_face) {
#pragma unroll
        for (int i = 1; i < 19; ++i)
            if (D3Q19::cx(i) == 1) f[i * nc + cell] = L.feq_in[i];
    }
    if (outlet_face) {
#pragma unroll
        for (int i = 1; i < 19; ++i)
            if (D3Q19::cx(i) == -1) f[i * nc + cell] = fl[i];
    }
}

// One collide + push step between two lattices in natural order. Solid cells
// are copied so that fout holds a complete lattice. links (or NULL without a
// mask) gives the solid neighbours, so every target index is computed without
// a dependent load.
__global__ void __launch_bounds__(256, 4) k_lbm_push(LbmParams L, const float *__restrict__ fin,
                                                 float *__restrict__ fout,
                                                 const uint32_t *__restrict__ links) {
    pdl_wait();
    pdl_trigger();
    int x, y, z, cell;
    if (!lattice_cell(L, x, y, z, cell)) return;
    const int nc = L.ncell;  // 19 * ncell < 2^31 is checked at create
    const uint32_t lk = links ? links[cell] : 0u;
    if (lk & 1u) {
#pragma unroll
        for (int i = 0; i < 19; ++i) fout[i * nc + cell] = fin[i * nc + cell];
        return;
    }
    const NbrOffsets o = nbr_offsets(L, x, y, z);
    float fl[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = fin[i * nc + cell];
    collide(L, fl);
    const bool inlet_face = L.bc_x == 1 && x == 0, outlet_face = L.bc_x == 1 && x == L.nx - 1;
    fout[cell] = fl[0];
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        if (inlet_face && D3Q19::cx(i) == -1) continue;   // leaves through x = 0
        if (outlet_face && D3Q19::cx(i) == 1) continue;   // leaves through x = nx - 1
        const int idx = ((lk >> i) & 1u)
                            ? D3Q19::opp(i) * nc + cell
                            : i * nc + cell + o.off(D3Q19::cx(i), D3Q19::cy(i), D3Q19::cz(i));
        fout[idx] = fl[i];
    }
    if (inlet_face) {
#pragma unroll
        for (int i = 1; i < 19; ++i)
            if (D3Q19::cx(i) == 1) fout[i * nc + cell] = L.feq_in[i];
    }
    if (outlet_face) {
#pragma unroll
        for (int i = 1; i < 19; ++i)
            if (D3Q19::cx(i) == -1) fout[i * nc + cell] = fl[i];
    }
}

// ---------------------------------------------------------------- reverse --

// One reverse step: g_prev = C^T S^T g_next at the pre-collision state f_t.
// The transposed streaming pulls g_next from where the forward pushed f*:
// slot i of x + c_i, or slot opp(i) of x itself where x + c_i is solid
// (bounce-back), nothing where the population leaves the domain, plus the
// cell's own slot i at the outlet face for the populations it re-injects.
__global__ void __launch_bounds__(256, 4) k_lbm_adjoint(LbmParams L, const float *__restrict__ f_t,
                                                    const float *__restrict__ g_next,
                                                    float *__restrict__ g_prev,
                                                    const uint32_t *__restrict__ links) {
    pdl_wait();
    pdl_trigger();
    int x, y, z, cell;
    if (!lattice_cell(L, x, y, z, cell)) return;
    const int nc = L.ncell;
    const uint32_t lk = links ? links[cell] : 0u;
    if (lk & 1u) {
#pragma unroll
        for (int i = 0; i < 19; ++i) g_prev[i * nc + cell] = g_next[i * nc + cell];
        return;
    }
    const NbrOffsets o = nbr_offsets(L, x, y, z);
    const bool inlet_face = L.bc_x == 1 && x == 0, outlet_face = L.bc_x == 1 && x == L.nx - 1;
    float g[19];
    g[0] = g_next[cell];
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        const int idx = ((lk >> i) & 1u)
                            ? D3Q19::opp(i) * nc + cell
                            : i * nc + cell + o.off(D3Q19::cx(i), D3Q19::cy(i), D3Q19::cz(i));
        float v = g_next[idx];
        if ((inlet_face && D3Q19::cx(i) == -1) || (outlet_face && D3Q19::cx(i) == 1)) v = 0.0f;
        if (outlet_face && D3Q19::cx(i) == -1) v += g_next[i * nc + cell];
        g[i] = v;
    }
    float fl[19];
#pragma unroll
    for (int i = 0; i < 19; ++i) fl[i] = f_t[i * nc + cell];
    collide_adjoint(L, fl, g);
#pragma unroll
    for (int i = 0; i < 19; ++i) g_prev[i * nc + cell] = g[i];
}

// ------------------------------------------------------------ auxiliaries --

// rho and u of one cell by Eq. lbm_sum_v2 (shifted populations: rho = 1 +
// sum f, rho u = sum c f + F/2); solid cells report rho = 0, u = 0.
__device__ __forceinline__ void cell_moments(const LbmParams &L, const float *__restrict__ f,
                                             const uint8_t *__restrict__ solid, int cell,
                                             float &r, float &ux, float &uy, float &uz) {
    const size_t nc = (size_t)L.ncell;
    r = ux = uy = uz = 0.0f;
    if (!(solid && solid[cell])) {
        float rs = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            float fi = f[i * nc + cell];
            rs += fi;
            jx += (float)D3Q19::cx(i) * fi;
            jy += (float)D3Q19::cy(i) * fi;
            jz += (float)D3Q19::cz(i) * fi;
        }
        r = 1.0f + rs;
        ux = (jx + 0.5f * L.Fx) / r;
        uy = (jy + 0.5f * L.Fy) / r;
        uz = (jz + 0.5f * L.Fz) / r;
    }
}

// The same from HOME-LBM moments m (planes rho - 1, u' = u + F/(2 rho), ...).
__device__ __forceinline__ void home_cell_velocity(const LbmParams &L, const float *__restrict__ m,
                                                   const uint8_t *__restrict__ solid, int cell,
                                                   float &r, float &ux, float &uy, float &uz) {
    const size_t nc = (size_t)L.ncell;
    r = ux = uy = uz = 0.0f;
    if (!(solid && solid[cell])) {
        r = 1.0f + m[cell];
        const float h = 0.5f / r;
        ux = m[nc + cell] - h * L.Fx;
        uy = m[2 * nc + cell] - h * L.Fy;
        uz = m[3 * nc + cell] - h * L.Fz;
    }
}

__global__ void k_lbm_macroscopic(LbmParams L, const float *__restrict__ f,
                                  const uint8_t *__restrict__ solid, float *__restrict__ rho,
                                  float *__restrict__ u) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.ncell) return;
    const size_t nc = (size_t)L.ncell;
    float r, ux, uy, uz;
    cell_moments(L, f, solid, cell, r, ux, uy, uz);
    if (rho) rho[cell] = r;
    if (u) {
        u[cell] = ux;
        u[nc + cell] = uy;
        u[2 * nc + cell] = uz;
    }
}

// The velocity at points pos[3][n] of the unit cube: trilinear between the
// cell centres ((c + 1/2) / n per axis, clamped to their box) of the cells'
// velocities (solid cells at rest); f holds populations or, with HOME, the
// HOME-LBM moments.
template <bool HOME>
__global__ void k_lbm_sample_velocity(LbmParams L, const float *__restrict__ f,
                                      const uint8_t *__restrict__ solid,
                                      const float *__restrict__ pos, int64_t n,
                                      float *__restrict__ u_out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int dims[3] = {L.nx, L.ny, L.nz};
    int i0[3];
    float t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float sc = pos[a * n + p] * (float)dims[a] - 0.5f;
        sc = fminf(fmaxf(sc, 0.0f), (float)(dims[a] - 1));  // NaN -> 0
        const int i = min((int)floorf(sc), dims[a] - 2);
        i0[a] = i;
        t[a] = sc - (float)i;
    }
    float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int cx = q & 1, cy = (q >> 1) & 1, cz = q >> 2;
        const float w = (cx ? t[0] : 1.0f - t[0]) * (cy ? t[1] : 1.0f - t[1]) *
                        (cz ? t[2] : 1.0f - t[2]);
        const int cell = ((i0[2] + cz) * L.ny + (i0[1] + cy)) * L.nx + (i0[0] + cx);
        float r, ux, uy, uz;
        if (HOME)
            home_cell_velocity(L, f, solid, cell, r, ux, uy, uz);
        else
            cell_moments(L, f, solid, cell, r, ux, uy, uz);
        acc[0] += w * ux;
        acc[1] += w * uy;
        acc[2] += w * uz;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) u_out[a * n + p] = acc[a];
}

__global__ void k_lbm_fill_eq(LbmParams L, float *__restrict__ f, float rho0, float ux, float uy,
                              float uz) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.ncell) return;
    const size_t nc = (size_t)L.ncell;
    float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        float cu = (float)D3Q19::cx(i) * ux + (float)D3Q19::cy(i) * uy + (float)D3Q19::cz(i) * uz;
        f[i * nc + cell] = D3Q19::w(i) * ((rho0 - 1.0f) + rho0 * (3.0f * cu + 4.5f * cu * cu - uu));
    }
}

__global__ void k_voxel_clear(uint8_t *__restrict__ solid, int64_t nbytes) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nbytes) solid[i] = 0;
}

// Eq. point2voxel: the node whose cell [x_w, x_w + dx)^3 holds the particle.
__global__ void k_voxelize(const float *__restrict__ pos, int64_t n, int nx, int ny, int nz,
                           float inv_dx, uint8_t *__restrict__ solid) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float sx = floorf(pos[p] * inv_dx), sy = floorf(pos[n + p] * inv_dx),
          sz = floorf(pos[2 * n + p] * inv_dx);
    if (!(sx >= 0.0f && sx < (float)nx && sy >= 0.0f && sy < (float)ny && sz >= 0.0f && sz < (float)nz))
        return;
    solid[((int64_t)sz * ny + (int64_t)sy) * nx + (int64_t)sx] = 1;
}

struct LbmHandle {
    dw_lbm_desc desc;
    LbmParams L;
    float *outlet = nullptr;  // [5][ny*nz]
    float *tape = nullptr;    // [max_tape][19][ncell]
    float *gtmp = nullptr;    // [19][ncell]
    uint32_t *links = nullptr;  // [ncell]
    const uint8_t *links_for = nullptr;  // mask whose link words lbm_cache_mask keeps in links
    bool home_attr_set = false;  // k_home_step's shared-memory limit raised, tz chosen
    int home_tz = 16;            // planes per block of k_home_step
};

static void fill_lbm_params(LbmHandle *h) {
    const dw_lbm_desc &d = h->desc;
    LbmParams &L = h->L;
    L.nx = d.nx;
    L.ny = d.ny;
    L.nz = d.nz;
    L.ncell = d.nx * d.ny * d.nz;
    L.inv_tau = 1.0f / d.tau;
    L.pre = 1.0f - 0.5f / d.tau;
    L.Fx = d.force[0];
    L.Fy = d.force[1];
    L.Fz = d.force[2];
    L.has_force = (d.force[0] != 0.0f || d.force[1] != 0.0f || d.force[2] != 0.0f) ? 1 : 0;
    L.bc_x = d.bc_x;
    double ux = d.u_inlet[0], uy = d.u_inlet[1], uz = d.u_inlet[2];
    double uu = ux * ux + uy * uy + uz * uz;
    for (int i = 0; i < 19; ++i) {
        double cu = D3Q19::cx(i) * ux + D3Q19::cy(i) * uy + D3Q19::cz(i) * uz;
        L.feq_in[i] = (float)(D3Q19::w(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
    }
}

}  // namespace dw

using namespace dw;

struct dw_lbm_s : LbmHandle {};

extern "C" dw_status lbm_create(const dw_lbm_desc *desc, dw_lbm *out) {
    DW_REQUIRE(desc && out, "desc/out must not be NULL");
    *out = nullptr;
    DW_REQUIRE(desc->nx >= 2 && desc->ny >= 2 && desc->nz >= 2, "lattice sizes must be >= 2");
    DW_REQUIRE(19ll * desc->nx * desc->ny * desc->nz < (1ll << 31), "lattice too large (19 nx ny nz must be < 2^31)");
    DW_REQUIRE(desc->ny <= 65535 && desc->nz <= 65535, "ny and nz must be <= 65535");
    DW_REQUIRE(desc->tau > 0.5f, "tau must be > 0.5");
    DW_REQUIRE(desc->bc_x == 0 || desc->bc_x == 1, "bc_x must be 0 or 1");
    DW_REQUIRE(desc->max_tape >= 1 && desc->max_tape <= 4096, "max_tape must be in [1, 4096]");
    dw_lbm h = new (std::nothrow) dw_lbm_s();
    if (!h) {
        set_error("out of host memory");
        return DW_ERR_OOM;
    }
    h->desc = *desc;
    fill_lbm_params(h);
    size_t lat = sizeof(float) * 19 * (size_t)h->L.ncell;
    cudaError_t e = cudaMalloc((void **)&h->outlet, sizeof(float) * 5 * (size_t)desc->ny * desc->nz);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->tape, lat * (size_t)desc->max_tape);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->gtmp, lat);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->links, sizeof(uint32_t) * (size_t)h->L.ncell);
    if (e != cudaSuccess) {
        dw_status st = cuda_fail(e, "lbm_create");
        lbm_destroy(h);
        return st;
    }
    *out = h;
    return DW_OK;
}

extern "C" dw_status lbm_destroy(dw_lbm h) {
    if (!h) return DW_OK;
    cudaFree(h->outlet);
    cudaFree(h->tape);
    cudaFree(h->gtmp);
    cudaFree(h->links);
    delete h;
    return DW_OK;
}

namespace dw {

// Launch shape of the lattice-row kernels (lattice_cell): one block row of up
// to 256 threads along x per (y, z).
static void lattice_launch(const LbmParams &L, dim3 &grid, dim3 &block) {
    const int bx = std::min(256, (L.nx + 31) / 32 * 32);
    block = dim3((unsigned)bx);
    grid = dim3((unsigned)((L.nx + bx - 1) / bx), (unsigned)L.ny, (unsigned)L.nz);
}

// Link words for a call with mask `solid`: the cached words when the mask is
// the one registered by lbm_cache_mask, else rebuilt into the handle's
// buffer (which drops a registered mask). NULL without a mask.
static dw_status links_for_call(LbmHandle *h, const uint8_t *solid, cudaStream_t s,
                                const uint32_t **links) {
    *links = nullptr;
    if (!solid) return DW_OK;
    if (solid != h->links_for) {
        h->links_for = nullptr;
        dim3 rg, rb;
        lattice_launch(h->L, rg, rb);
        DW_CUDA(launch_pdl3(k_lbm_links, rg, rb, s, h->L, solid, h->links));
    }
    *links = h->links;
    return DW_OK;
}

}  // namespace dw

extern "C" dw_status lbm_cache_mask(dw_lbm h, const uint8_t *solid, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    h->links_for = nullptr;
    if (!solid) return DW_OK;
    const uint32_t *links = nullptr;
    dw_status st = links_for_call(h, solid, as_stream(stream), &links);
    if (st != DW_OK) return st;
    h->links_for = solid;
    DW_LAUNCHED("lbm_cache_mask");
    return DW_OK;
}

extern "C" dw_status lbm_step(dw_lbm h, float *f, const uint8_t *solid, int32_t steps,
                              dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(f, "f must not be NULL");
    DW_REQUIRE(steps >= 0, "steps must be >= 0");
    cudaStream_t s = as_stream(stream);
    const LbmParams &L = h->L;
    const uint32_t *links = nullptr;
    dw_status st = links_for_call(h, solid, s, &links);
    if (st != DW_OK) return st;
    dim3 rg, rb;
    lattice_launch(L, rg, rb);
    for (int k = 0; k + 1 < steps; k += 2) {
        DW_CUDA(launch_pdl3(k_lbm_aa_even, rg, rb, s, L, f, solid, h->outlet));
        DW_CUDA(launch_pdl3(k_lbm_aa_odd, rg, rb, s, L, f, links, h->outlet));
    }
    if (steps & 1) {
        DW_CUDA(launch_pdl3(k_lbm_push, rg, rb, s, L, (const float *)f, h->tape, links));
        DW_CUDA(cudaMemcpyAsync(f, h->tape, sizeof(float) * 19 * (size_t)L.ncell,
                                cudaMemcpyDeviceToDevice, s));
    }
    DW_LAUNCHED("lbm_step");
    return DW_OK;
}

extern "C" dw_status lbm_step_adjoint(dw_lbm h, const float *f_in, float *g_f,
                                      const uint8_t *solid, int32_t steps, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(f_in && g_f, "f_in/g_f must not be NULL");
    DW_REQUIRE(steps >= 0 && steps <= h->desc.max_tape, "steps=%d must be in [0, max_tape=%d]",
               steps, h->desc.max_tape);
    if (steps == 0) return DW_OK;
    cudaStream_t s = as_stream(stream);
    const LbmParams &L = h->L;
    const size_t lat = 19 * (size_t)L.ncell;
    const uint32_t *links = nullptr;
    dw_status st = links_for_call(h, solid, s, &links);
    if (st != DW_OK) return st;
    dim3 rg, rb;
    lattice_launch(L, rg, rb);
    // states f(1) .. f(steps-1) into tape[0 .. steps-2]
    for (int k = 1; k < steps; ++k) {
        const float *src = k == 1 ? f_in : h->tape + (size_t)(k - 2) * lat;
        DW_CUDA(launch_pdl3(k_lbm_push, rg, rb, s, L, src, h->tape + (size_t)(k - 1) * lat, links));
    }
    float *cur = g_f, *other = h->gtmp;
    for (int k = steps - 1; k >= 0; --k) {
        const float *state = k == 0 ? f_in : h->tape + (size_t)(k - 1) * lat;
        DW_CUDA(launch_pdl3(k_lbm_adjoint, rg, rb, s, L, state, (const float *)cur, other, links));
        float *tmp = cur;
        cur = other;
        other = tmp;
    }
    if (cur != g_f)
        DW_CUDA(cudaMemcpyAsync(g_f, cur, sizeof(float) * lat, cudaMemcpyDeviceToDevice, s));
    DW_LAUNCHED("lbm_step_adjoint");
    return DW_OK;
}

extern "C" dw_status lbm_macroscopic(dw_lbm h, const float *f, const uint8_t *solid, float *rho,
                                     float *u, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(f, "f must not be NULL");
    if (!rho && !u) return DW_OK;
    k_lbm_macroscopic<<<grid_for(h->L.ncell, 256), 256, 0, as_stream(stream)>>>(h->L, f, solid, rho, u);
    DW_LAUNCHED("k_lbm_macroscopic");
    return DW_OK;
}

extern "C" dw_status lbm_sample_velocity(dw_lbm h, const float *f, const uint8_t *solid,
                                         const float *pos, int64_t n, float *u_out,
                                         dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(f && pos && u_out, "f, pos and u_out must not be NULL");
    k_lbm_sample_velocity<false><<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(
        h->L, f, solid, pos, n, u_out);
    DW_LAUNCHED("k_lbm_sample_velocity");
    return DW_OK;
}

extern "C" dw_status lbm_home_sample_velocity(dw_lbm h, const float *m, const uint8_t *solid,
                                              const float *pos, int64_t n, float *u_out,
                                              dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(m && pos && u_out, "m, pos and u_out must not be NULL");
    k_lbm_sample_velocity<true><<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(
        h->L, m, solid, pos, n, u_out);
    DW_LAUNCHED("k_lbm_sample_velocity<home>");
    return DW_OK;
}

extern "C" dw_status lbm_init_equilibrium(dw_lbm h, float *f, float rho0, const float u0[3],
                                          dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(f && u0, "f/u0 must not be NULL");
    DW_REQUIRE(rho0 > 0.0f, "rho0 must be > 0");
    k_lbm_fill_eq<<<grid_for(h->L.ncell, 256), 256, 0, as_stream(stream)>>>(h->L, f, rho0, u0[0],
                                                                            u0[1], u0[2]);
    DW_LAUNCHED("k_lbm_fill_eq");
    return DW_OK;
}

extern "C" dw_status voxelize_particles(const float *pos, int64_t n, int32_t nx, int32_t ny,
                                        int32_t nz, float dx, uint8_t *solid, dw_stream stream) {
    DW_REQUIRE(solid, "solid must not be NULL");
    DW_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1, "lattice sizes must be >= 1");
    DW_REQUIRE(dx > 0.0f, "dx must be > 0");
    DW_REQUIRE(n >= 0 && (n == 0 || pos), "pos must not be NULL with n > 0");
    cudaStream_t s = as_stream(stream);
    int64_t nb = (int64_t)nx * ny * nz;
    k_voxel_clear<<<grid_for(nb, 256), 256, 0, s>>>(solid, nb);
    if (n > 0) k_voxelize<<<grid_for(n, 256), 256, 0, s>>>(pos, n, nx, ny, nz, 1.0f / dx, solid);
    DW_LAUNCHED("voxelize");
    return DW_OK;
}

// ================================================================ HOME-LBM
// Moment-encoded lattice Boltzmann step (App. D, after Li et al. 2023): each
// cell stores ten moments of its post-collision populations instead of the
// nineteen populations, m = [10][ncell] with planes
//   0: rho - 1, 1-3: u' (momentum / rho after the collision), 4-9: S (Sxx, Syy,
//   Szz, Sxy, Sxz, Syz; S = sum H2(c_i) f_i / rho, H2 = c c - I/3).
// A step pulls f_i(x) = f_i^post(x - c_i), each population rebuilt from the
// source cell's moments by the Hermite series to second order plus the six
// third-order terms D3Q19 carries (H3_aab(c) = c_b (c_a^2 - 1/3), coefficient
// A_aab = u_b S_aa + 2 u_a S_ab - 2 u_a^2 u_b), with the same boundaries as the
// BGK step (bounce-back from the own cell's opposite population, inlet, outlet),
// then collides in moment space: the deviatoric part of the second moment
// relaxes at 1/tau, its trace to equilibrium, Guo forcing per part. Arithmetic
// on deviations (f_i - w_i) keeps float32 resolution. Two moment lattices are
// used in turn (pull streaming is not in place); the handle's tape serves as
// the second one.

namespace dw {

struct HomeParams {
    float g_in[19];  // inlet populations (deviations): rebuilt from rho = 1, u_in, S = u_in u_in
};

// f_i - w_i rebuilt from one cell's moments (a[0] = rho - 1). Every velocity
// component is a compile-time constant once the direction loop is unrolled,
// and the guards drop the terms that vanish for it.
__host__ __device__ __forceinline__ float home_rebuild(int i, const float a[10]) {
    const int cx = D3Q19::cx(i), cy = D3Q19::cy(i), cz = D3Q19::cz(i);
    const float ux = a[1], uy = a[2], uz = a[3];
    const float sxx = a[4], syy = a[5], szz = a[6], sxy = a[7], sxz = a[8], syz = a[9];
    float p = 0.0f;
    if (cx) p += 3.0f * (float)cx * ux;
    if (cy) p += 3.0f * (float)cy * uy;
    if (cz) p += 3.0f * (float)cz * uz;
    // 4.5 H2 : S
    p += (cx ? 3.0f : -1.5f) * sxx;
    p += (cy ? 3.0f : -1.5f) * syy;
    p += (cz ? 3.0f : -1.5f) * szz;
    if (cx && cy) p += 9.0f * (float)(cx * cy) * sxy;
    if (cx && cz) p += 9.0f * (float)(cx * cz) * sxz;
    if (cy && cz) p += 9.0f * (float)(cy * cz) * syz;
    // 13.5 sum H3_aab A_aab, H3_aab = c_b (c_a^2 - 1/3): 13.5 * 2/3 = 9, 13.5 * -1/3 = -4.5
    if (cy) p += (float)cy * (cx ? 9.0f : -4.5f) * (uy * sxx + 2.0f * ux * sxy - 2.0f * ux * ux * uy);
    if (cz) p += (float)cz * (cx ? 9.0f : -4.5f) * (uz * sxx + 2.0f * ux * sxz - 2.0f * ux * ux * uz);
    if (cx) p += (float)cx * (cy ? 9.0f : -4.5f) * (ux * syy + 2.0f * uy * sxy - 2.0f * uy * uy * ux);
    if (cz) p += (float)cz * (cy ? 9.0f : -4.5f) * (uz * syy + 2.0f * uy * syz - 2.0f * uy * uy * uz);
    if (cx) p += (float)cx * (cz ? 9.0f : -4.5f) * (ux * szz + 2.0f * uz * sxz - 2.0f * uz * uz * ux);
    if (cy) p += (float)cy * (cz ? 9.0f : -4.5f) * (uy * szz + 2.0f * uz * syz - 2.0f * uz * uz * uy);
    return D3Q19::w(i) * (a[0] + (1.0f + a[0]) * p);
}

// All nineteen f_i - w_i of one cell at once. Grouping each direction's terms
// into an even part (shared by opposite directions) and odd parts makes the
// closure coefficients A_aab count once per cell instead of once per
// population; the result equals home_rebuild(i, a) for every i.
__host__ __device__ __forceinline__ void home_rebuild_all(const float a[10], float g[19]) {
    const float dr = a[0], rho = 1.0f + a[0];
    const float ux = a[1], uy = a[2], uz = a[3];
    const float sxx = a[4], syy = a[5], szz = a[6], sxy = a[7], sxz = a[8], syz = a[9];
    const float Axxy = uy * sxx + 2.0f * ux * sxy - 2.0f * ux * ux * uy;
    const float Axxz = uz * sxx + 2.0f * ux * sxz - 2.0f * ux * ux * uz;
    const float Axyy = ux * syy + 2.0f * uy * sxy - 2.0f * uy * uy * ux;
    const float Ayyz = uz * syy + 2.0f * uy * syz - 2.0f * uy * uy * uz;
    const float Axzz = ux * szz + 2.0f * uz * sxz - 2.0f * uz * uz * ux;
    const float Ayzz = uy * szz + 2.0f * uz * syz - 2.0f * uz * uz * uy;
    const float w0 = 1.0f / 3.0f, w1 = 1.0f / 18.0f, w2 = 1.0f / 36.0f;
    g[0] = w0 * (dr + rho * (-1.5f * (sxx + syy + szz)));
    // axis directions: p = E_a +- O_a
    const float Ex = 3.0f * sxx - 1.5f * (syy + szz), Ox = 3.0f * ux - 4.5f * (Axyy + Axzz);
    const float Ey = 3.0f * syy - 1.5f * (sxx + szz), Oy = 3.0f * uy - 4.5f * (Axxy + Ayzz);
    const float Ez = 3.0f * szz - 1.5f * (sxx + syy), Oz = 3.0f * uz - 4.5f * (Axxz + Ayyz);
    g[1] = w1 * (dr + rho * (Ex + Ox));
    g[2] = w1 * (dr + rho * (Ex - Ox));
    g[3] = w1 * (dr + rho * (Ey + Oy));
    g[4] = w1 * (dr + rho * (Ey - Oy));
    g[5] = w1 * (dr + rho * (Ez + Oz));
    g[6] = w1 * (dr + rho * (Ez - Oz));
    // edge directions (s, t) in a plane: p = E + 9 s t S_ab + s P + t Q
    {
        const float E = 3.0f * (sxx + syy) - 1.5f * szz, D = 9.0f * sxy;
        const float P = 3.0f * ux + 9.0f * Axyy - 4.5f * Axzz;
        const float Q = 3.0f * uy + 9.0f * Axxy - 4.5f * Ayzz;
        g[7] = w2 * (dr + rho * (E + D + P + Q));
        g[8] = w2 * (dr + rho * (E + D - P - Q));
        g[13] = w2 * (dr + rho * (E - D + P - Q));
        g[14] = w2 * (dr + rho * (E - D - P + Q));
    }
    {
        const float E = 3.0f * (sxx + szz) - 1.5f * syy, D = 9.0f * sxz;
        const float P = 3.0f * ux + 9.0f * Axzz - 4.5f * Axyy;
        const float Q = 3.0f * uz + 9.0f * Axxz - 4.5f * Ayyz;
        g[9] = w2 * (dr + rho * (E + D + P + Q));
        g[10] = w2 * (dr + rho * (E + D - P - Q));
        g[15] = w2 * (dr + rho * (E - D + P - Q));
        g[16] = w2 * (dr + rho * (E - D - P + Q));
    }
    {
        const float E = 3.0f * (syy + szz) - 1.5f * sxx, D = 9.0f * syz;
        const float P = 3.0f * uy + 9.0f * Ayzz - 4.5f * Axxy;
        const float Q = 3.0f * uz + 9.0f * Ayyz - 4.5f * Axxz;
        g[11] = w2 * (dr + rho * (E + D + P + Q));
        g[12] = w2 * (dr + rho * (E + D - P - Q));
        g[17] = w2 * (dr + rho * (E - D + P - Q));
        g[18] = w2 * (dr + rho * (E - D - P + Q));
    }
}

// Moment-space collision from the pulled deviations' sums: dr = sum g,
// j = sum c g, P = sum c c g (= Pi - I/3); writes the ten stored moments.
__host__ __device__ __forceinline__ void home_collide(const LbmParams &L, float dr, const float j[3],
                                             const float P[6], float out[10]) {
    const float rho = 1.0f + dr, inv_rho = 1.0f / rho;
    const float u[3] = {(j[0] + 0.5f * L.Fx) * inv_rho, (j[1] + 0.5f * L.Fy) * inv_rho,
                        (j[2] + 0.5f * L.Fz) * inv_rho};
    // N = Pi - rho (I/3 + u u) = P - dr/3 I - rho u u
    const float third = 1.0f / 3.0f;
    float N[6] = {P[0] - third * dr - rho * u[0] * u[0], P[1] - third * dr - rho * u[1] * u[1],
                  P[2] - third * dr - rho * u[2] * u[2], P[3] - rho * u[0] * u[1],
                  P[4] - rho * u[0] * u[2], P[5] - rho * u[1] * u[2]};
    const float trN = third * (N[0] + N[1] + N[2]);
    const float k = 1.0f - L.inv_tau;
    float S[6];
    S[0] = k * (N[0] - trN);
    S[1] = k * (N[1] - trN);
    S[2] = k * (N[2] - trN);
    S[3] = k * N[3];
    S[4] = k * N[4];
    S[5] = k * N[5];
    if (L.has_force) {
        // Phi = u F + F u: deviatoric part with 1 - 1/(2 tau), trace part with 1/2
        const float F[3] = {L.Fx, L.Fy, L.Fz};
        const float pd[3] = {2.0f * u[0] * F[0], 2.0f * u[1] * F[1], 2.0f * u[2] * F[2]};
        const float trP = third * (pd[0] + pd[1] + pd[2]);
        S[0] += L.pre * (pd[0] - trP) + 0.5f * trP;
        S[1] += L.pre * (pd[1] - trP) + 0.5f * trP;
        S[2] += L.pre * (pd[2] - trP) + 0.5f * trP;
        S[3] += L.pre * (u[0] * F[1] + F[0] * u[1]);
        S[4] += L.pre * (u[0] * F[2] + F[0] * u[2]);
        S[5] += L.pre * (u[1] * F[2] + F[1] * u[2]);
    }
    out[0] = dr;
    out[1] = u[0] + 0.5f * L.Fx * inv_rho;
    out[2] = u[1] + 0.5f * L.Fy * inv_rho;
    out[3] = u[2] + 0.5f * L.Fz * inv_rho;
    out[4] = u[0] * u[0] + S[0] * inv_rho;
    out[5] = u[1] * u[1] + S[1] * inv_rho;
    out[6] = u[2] * u[2] + S[2] * inv_rho;
    out[7] = u[0] * u[1] + S[3] * inv_rho;
    out[8] = u[0] * u[2] + S[4] * inv_rho;
    out[9] = u[1] * u[2] + S[5] * inv_rho;
}

// Tiles of the streaming HOME kernel: 30 x 6 cells of a z-plane per block,
// walking tz planes along z (chosen per lattice, below). Each plane of the
// tile plus a one-cell halo (32 x 8 = 256 cells, one per thread) has its cells' nineteen
// post-collision populations rebuilt once into a shared-memory ring of three
// planes; every cell of the middle plane then pulls its populations from the
// ring, so a cell's closure terms are evaluated about 1.6 times per step
// (halo and the two extra planes of each z range) instead of once per pulling
// neighbour, and its moments are read from global memory about as often.
constexpr int HOME_TX = 30, HOME_TY = 6;
constexpr int HOME_HX = HOME_TX + 2, HOME_HY = HOME_TY + 2;
constexpr int HOME_PLANE = HOME_HX * HOME_HY;          // 256 cells: one per thread
// The ring keeps each plane's populations only as long as they are pulled:
// in-plane directions (c_z = 0, nine of them) while the plane is the current
// one, upward ones (c_z = +1, five) until the plane above is done, downward
// ones (c_z = -1, five) from the plane below's step through the plane's own
// (bounce-back reads them). Buffers, in units of 340 floats: in-plane
// [2 planes][9] at 0, upward [3][5] at 18, downward [2][5] at 33 (units of one plane).
constexpr size_t HOME_SMEM = 43 * HOME_PLANE * sizeof(float);  // 44,032 bytes

// Index of direction i within its group (in-plane 0 1 2 3 4 7 8 13 14,
// upward 5 9 11 16 18, downward 6 10 12 15 17).
__host__ __device__ constexpr int home_k(int i) {
    constexpr int t[19] = {0, 1, 2, 3, 4, 0, 0, 5, 6, 1, 1, 2, 2, 7, 8, 3, 3, 4, 4};
    return t[i];
}
// Ring offsets of plane q's group buffers (q counts the block's planes from
// z0 - 1).
__host__ __device__ __forceinline__ int home_in_base(int q) { return (q & 1) * 9 * HOME_PLANE; }
__host__ __device__ __forceinline__ int home_up_base(int q) { return (18 + (q % 3) * 5) * HOME_PLANE; }
__host__ __device__ __forceinline__ int home_dn_base(int q) { return (33 + (q & 1) * 5) * HOME_PLANE; }

__host__ __device__ __forceinline__ int wrap_full(int v, int n) { return ((v % n) + n) % n; }

__host__ __device__ __forceinline__ float ld_ro(const float *p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}

// The moments of one halo-plane cell, loaded ahead of their use. ok is false
// for cells whose populations no fluid cell of the tile pulls: solid cells
// (bounce-back uses the puller's own populations) and, with the x inlet and
// outlet, cells beyond the x faces (nothing is loaded for those).
struct HomeHalo {
    float a[10];
    bool ok;
};

// Where halo-plane cell c (0..339) of the tile at (x0, y0) sits in every
// plane: xy = y * nx + x after the periodic wraps, or -1 beyond an x face
// with the inlet and outlet. Fixed for a thread, so computed once.
__host__ __device__ __forceinline__ int home_halo_xy(const LbmParams &L, int x0, int y0, int c) {
    const int hx = c % HOME_HX, hy = c / HOME_HX;
    int gx = x0 + hx - 1;
    if (gx < 0 || gx >= L.nx) {
        if (L.bc_x == 1) return -1;
        gx = wrap_full(gx, L.nx);
    }
    return wrap_full(y0 + hy - 1, L.ny) * L.nx + gx;
}

// Load the moments of the halo cell at xy in plane gz (0 <= gz < nz).
__host__ __device__ __forceinline__ void home_halo_load(const LbmParams &L,
                                                        const float *__restrict__ m_in,
                                                        const uint8_t *__restrict__ solid, int xy,
                                                        int gz, HomeHalo &h) {
    h.ok = xy >= 0;
    if (!h.ok) return;
    const int cell = gz * (L.nx * L.ny) + xy;
    const int nc = L.ncell;
#pragma unroll
    for (int k = 0; k < 10; ++k) h.a[k] = ld_ro(m_in + k * nc + cell);
    if (solid && solid[cell]) h.ok = false;
}

// Plane z wrapped periodically for z in [-1, nz].
__host__ __device__ __forceinline__ int home_wrap_z(const LbmParams &L, int z) {
    return z < 0 ? z + L.nz : (z >= L.nz ? z - L.nz : z);
}

// Rebuild the nineteen populations of a loaded halo cell c of plane q into
// the ring sm.
__host__ __device__ __forceinline__ void home_halo_store(const HomeHalo &h, float *sm, int q, int c) {
    if (!h.ok) return;
    float g[19];
    home_rebuild_all(h.a, g);
    const int bi = home_in_base(q) + c, bu = home_up_base(q) + c, bd = home_dn_base(q) + c;
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const int cz = D3Q19::cz(i);
        sm[(cz == 0 ? bi : (cz == 1 ? bu : bd)) + home_k(i) * HOME_PLANE] = g[i];
    }
}

// Pull, collide and store cell (x0 + tx, y0 + ty, z) from the ring; z is the
// block's plane q; lk is the cell's link word (bit 0 solid, bit i the
// neighbour x + c_i solid; 0 without a mask).
__host__ __device__ __forceinline__ void home_tile_cell(const LbmParams &L, const HomeParams &H,
                                                        const float *__restrict__ m_in,
                                                        float *__restrict__ mout, uint32_t lk,
                                                        const float *sm, int q, int x0, int y0,
                                                        int z, int tx, int ty) {
    const int x = x0 + tx, y = y0 + ty;
    if (x >= L.nx || y >= L.ny) return;
    const int nc = L.ncell;
    const int cell = (z * L.ny + y) * L.nx + x;
    if (lk & 1u) {  // solid: keep the moments
#pragma unroll
        for (int k = 0; k < 10; ++k) mout[k * nc + cell] = ld_ro(m_in + k * nc + cell);
        return;
    }
    const bool inlet_face = L.bc_x == 1 && x == 0, outlet_face = L.bc_x == 1 && x == L.nx - 1;
    const int oc = (ty + 1) * HOME_HX + (tx + 1);
    // pulled direction i comes from plane q - c_z; the own cell's from plane q
    const int in_q = home_in_base(q) + oc, up_qm = home_up_base(q - 1) + oc,
              dn_qp = home_dn_base(q + 1) + oc;
    const int up_q = home_up_base(q) + oc, dn_q = home_dn_base(q) + oc;
    float g[19];
    if (lk == 0u && !inlet_face && !outlet_face) {
        // no solid neighbour, no open face: every population comes from the ring
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int cx = D3Q19::cx(i), cy = D3Q19::cy(i), cz = D3Q19::cz(i);
            const int b = cz == 0 ? in_q : (cz == 1 ? up_qm : dn_qp);
            g[i] = sm[b + home_k(i) * HOME_PLANE - cy * HOME_HX - cx];
        }
    } else {
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const int cx = D3Q19::cx(i), cy = D3Q19::cy(i), cz = D3Q19::cz(i);
            const int jo = D3Q19::opp(i), czo = D3Q19::cz(jo);
            const int own_i = (cz == 0 ? in_q : (cz == 1 ? up_q : dn_q)) + home_k(i) * HOME_PLANE;
            const int own_jo =
                (czo == 0 ? in_q : (czo == 1 ? up_q : dn_q)) + home_k(jo) * HOME_PLANE;
            if (i == 0) {
                g[i] = sm[own_i];
            } else if (inlet_face && cx == 1) {
                g[i] = H.g_in[i];
            } else if (outlet_face && cx == -1) {
                g[i] = sm[own_i];
            } else if ((lk >> jo) & 1u) {
                g[i] = sm[own_jo];  // halfway bounce-back
            } else {
                const int b = cz == 0 ? in_q : (cz == 1 ? up_qm : dn_qp);
                g[i] = sm[b + home_k(i) * HOME_PLANE - cy * HOME_HX - cx];
            }
        }
    }
    // moments over pairs of opposite directions (2k - 1, 2k): s = g + g_opp
    // carries the even moments, d = g - g_opp the odd ones
    float dr = g[0], j[3] = {0.0f, 0.0f, 0.0f}, P[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
        const int cx = D3Q19::cx(i), cy = D3Q19::cy(i), cz = D3Q19::cz(i);
        const float sp = g[i] + g[i + 1], dp = g[i] - g[i + 1];
        dr += sp;
        if (cx) j[0] += (float)cx * dp;
        if (cy) j[1] += (float)cy * dp;
        if (cz) j[2] += (float)cz * dp;
        if (cx) P[0] += sp;
        if (cy) P[1] += sp;
        if (cz) P[2] += sp;
        if (cx && cy) P[3] += (float)(cx * cy) * sp;
        if (cx && cz) P[4] += (float)(cx * cz) * sp;
        if (cy && cz) P[5] += (float)(cy * cz) * sp;
    }
    float out[10];
    home_collide(L, dr, j, P, out);
#pragma unroll
    for (int k = 0; k < 10; ++k) mout[k * nc + cell] = out[k];
}

// One HOME-LBM step m_in -> mout. Grid (ceil(nx/32), ceil(ny/8),
// ceil(nz/tz)), 256 threads, HOME_SMEM bytes of dynamic shared memory.
// The moments of plane z + 2 and the link words of plane z + 1 are loaded
// while plane z is pulled and collided, so their latency overlaps the work.
// Interior cell of thread t (t < 180) of a tile: (t mod 30, t div 30).
__host__ __device__ __forceinline__ bool home_interior(int t, int &ix, int &iy) {
    ix = t % HOME_TX;
    iy = t / HOME_TX;
    return t < HOME_TX * HOME_TY;
}

__global__ void __launch_bounds__(256, 4) k_home_step(LbmParams L, HomeParams H,
                                                  const float *__restrict__ m_in,
                                                  float *__restrict__ mout,
                                                  const uint8_t *__restrict__ solid,
                                                  const uint32_t *__restrict__ links, int tz) {
    extern __shared__ float home_sm[];
    pdl_wait();
    pdl_trigger();
    const int x0 = blockIdx.x * HOME_TX, y0 = blockIdx.y * HOME_TY, z0 = blockIdx.z * tz;
    const int z1 = min(z0 + tz, L.nz);
    const int tid = threadIdx.x;
    int ix, iy;
    const bool worker = home_interior(tid, ix, iy);
    const bool inside = worker && x0 + ix < L.nx && y0 + iy < L.ny;
    const int col = (y0 + iy) * L.nx + (x0 + ix), plane = L.nx * L.ny;
    const int xy = home_halo_xy(L, x0, y0, tid);
    HomeHalo h;
    // planes z0 - 1 and z0 (q = 0, 1), then plane z0 + 1 loaded ahead
    home_halo_load(L, m_in, solid, xy, home_wrap_z(L, z0 - 1), h);
    home_halo_store(h, home_sm, 0, tid);
    home_halo_load(L, m_in, solid, xy, z0, h);
    home_halo_store(h, home_sm, 1, tid);
    home_halo_load(L, m_in, solid, xy, home_wrap_z(L, z0 + 1), h);
    uint32_t lk_next = (links && inside) ? links[z0 * plane + col] : 0u;
    for (int z = z0; z < z1; ++z) {
        const int q = z - z0 + 1;
        home_halo_store(h, home_sm, q + 1, tid);
        if (z + 1 < z1) home_halo_load(L, m_in, solid, xy, home_wrap_z(L, z + 2), h);
        const uint32_t lk = lk_next;
        if (links && inside && z + 1 < z1) lk_next = links[(z + 1) * plane + col];
        __syncthreads();
        if (worker) home_tile_cell(L, H, m_in, mout, lk, home_sm, q, x0, y0, z, ix, iy);
        __syncthreads();
    }
}

__global__ void k_home_fill(int nc, float *__restrict__ m, float v0, float v1,
                            float v2, float v3, float v4, float v5, float v6, float v7, float v8,
                            float v9) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= nc) return;
    const float v[10] = {v0, v1, v2, v3, v4, v5, v6, v7, v8, v9};
#pragma unroll
    for (int k = 0; k < 10; ++k) m[k * nc + cell] = v[k];
}

__global__ void k_home_macroscopic(LbmParams L, const float *__restrict__ m,
                                   const uint8_t *__restrict__ solid, float *__restrict__ rho,
                                   float *__restrict__ u) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= L.ncell) return;
    const int nc = L.ncell;
    const bool sol = solid && solid[cell];
    const float r = 1.0f + m[cell];
    const float hr = 0.5f / r;
    if (rho) rho[cell] = sol ? 0.0f : r;
    if (u) {
        u[cell] = sol ? 0.0f : m[nc + cell] - hr * L.Fx;
        u[nc + cell] = sol ? 0.0f : m[2 * nc + cell] - hr * L.Fy;
        u[2 * nc + cell] = sol ? 0.0f : m[3 * nc + cell] - hr * L.Fz;
    }
}

// Host copy of the moment-space collision in double (inlet and fill values).
static void home_collide_host(const dw_lbm_desc &d, double rho, const double j[3],
                              const double Pi[3][3], double out[10]) {
    const double F[3] = {d.force[0], d.force[1], d.force[2]}, tau = d.tau;
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
    double N[3][3], Phi[3][3], trN = 0.0, trP = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            N[a][b] = Pi[a][b] - rho * ((a == b ? 1.0 / 3.0 : 0.0) + u[a] * u[b]);
            Phi[a][b] = u[a] * F[b] + F[a] * u[b];
        }
    for (int a = 0; a < 3; ++a) {
        trN += N[a][a] / 3.0;
        trP += Phi[a][a] / 3.0;
    }
    double S[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double dl = a == b ? 1.0 : 0.0;
            S[a][b] = u[a] * u[b] + ((1.0 - 1.0 / tau) * (N[a][b] - dl * trN) +
                                     (1.0 - 0.5 / tau) * (Phi[a][b] - dl * trP) + 0.5 * dl * trP) /
                                        rho;
        }
    out[0] = rho - 1.0;
    for (int a = 0; a < 3; ++a) out[1 + a] = u[a] + 0.5 * F[a] / rho;
    out[4] = S[0][0];
    out[5] = S[1][1];
    out[6] = S[2][2];
    out[7] = S[0][1];
    out[8] = S[0][2];
    out[9] = S[1][2];
}

static HomeParams home_params(const dw_lbm_desc &d) {
    HomeParams H;
    const double u[3] = {d.u_inlet[0], d.u_inlet[1], d.u_inlet[2]};
    const double S[3][3] = {{u[0] * u[0], u[0] * u[1], u[0] * u[2]},
                            {u[1] * u[0], u[1] * u[1], u[1] * u[2]},
                            {u[2] * u[0], u[2] * u[1], u[2] * u[2]}};
    for (int i = 0; i < 19; ++i) {
        const double c[3] = {(double)D3Q19::cx(i), (double)D3Q19::cy(i), (double)D3Q19::cz(i)};
        double p = 0.0;
        for (int a = 0; a < 3; ++a) p += 3.0 * c[a] * u[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                p += 4.5 * (c[a] * c[b] - (a == b ? 1.0 / 3.0 : 0.0)) * S[a][b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                if (a == b) continue;
                const double A = u[b] * S[a][a] + 2.0 * u[a] * S[a][b] - 2.0 * u[a] * u[a] * u[b];
                p += 13.5 * c[b] * (c[a] * c[a] - 1.0 / 3.0) * A;
            }
        H.g_in[i] = (float)(D3Q19::w(i) * p);  // rho = 1: w (rho - 1) + w rho p
    }
    return H;
}

// Planes per block: each block also rebuilds the two planes beyond its z
// range, so tall ranges waste less; the blocks run in waves of `slots`
// (resident blocks on the GPU), so a block count just under a whole number of
// waves wastes less. Take the tz in [8, 32] with the best product.
static int home_pick_tz(const LbmParams &L, int slots) {
    const long cols = (long)((L.nx + HOME_TX - 1) / HOME_TX) * ((L.ny + HOME_TY - 1) / HOME_TY);
    int best = 16;
    double best_eff = -1.0;
    for (int tz = 8; tz <= 32; ++tz) {
        const long blocks = cols * ((L.nz + tz - 1) / tz);
        const double waves = (double)blocks / slots;
        const double eff = waves / std::ceil(waves) * (double)tz / (tz + 2);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = tz;
        }
    }
    return best;
}

}  // namespace dw

extern "C" dw_status lbm_home_init(dw_lbm h, float *m, float rho0, const float u0[3],
                                   dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(m && u0, "m/u0 must not be NULL");
    DW_REQUIRE(rho0 > 0.0f, "rho0 must be > 0");
    const double r = rho0, u[3] = {u0[0], u0[1], u0[2]};
    const double j[3] = {r * u[0], r * u[1], r * u[2]};
    double Pi[3][3], v[10];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Pi[a][b] = r * ((a == b ? 1.0 / 3.0 : 0.0) + u[a] * u[b]);
    home_collide_host(h->desc, r, j, Pi, v);
    k_home_fill<<<grid_for(h->L.ncell, 256), 256, 0, as_stream(stream)>>>(
        h->L.ncell, m, (float)v[0], (float)v[1], (float)v[2], (float)v[3], (float)v[4],
        (float)v[5], (float)v[6], (float)v[7], (float)v[8], (float)v[9]);
    DW_LAUNCHED("k_home_fill");
    return DW_OK;
}

extern "C" dw_status lbm_home_step(dw_lbm h, float *m, const uint8_t *solid, int32_t steps,
                                   dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(m, "m must not be NULL");
    DW_REQUIRE(steps >= 0, "steps must be >= 0");
    if (steps == 0) return DW_OK;
    cudaStream_t s = as_stream(stream);
    const LbmParams &L = h->L;
    const HomeParams H = home_params(h->desc);
    const uint32_t *links = nullptr;
    dw_status st = links_for_call(h, solid, s, &links);
    if (st != DW_OK) return st;
    if (!h->home_attr_set) {
        DW_CUDA(cudaFuncSetAttribute(k_home_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)HOME_SMEM));
        int dev = 0, sms = 0, per_sm = 0;
        DW_CUDA(cudaGetDevice(&dev));
        DW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        DW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_home_step, 256, HOME_SMEM));
        h->home_tz = home_pick_tz(L, std::max(1, sms * per_sm));
        h->home_attr_set = true;
    }
    const int tz = h->home_tz;
    const dim3 grid((unsigned)((L.nx + HOME_TX - 1) / HOME_TX),
                    (unsigned)((L.ny + HOME_TY - 1) / HOME_TY), (unsigned)((L.nz + tz - 1) / tz));
    float *a = m, *b = h->tape;  // the tape holds >= 19 ncell floats; 10 are used
    for (int k = 0; k < steps; ++k) {
        DW_CUDA(launch_pdl_smem(k_home_step, grid, dim3(256), HOME_SMEM, s, L, H,
                                (const float *)a, b, solid, links, tz));
        std::swap(a, b);
    }
    if (a != m)
        DW_CUDA(cudaMemcpyAsync(m, a, sizeof(float) * 10 * (size_t)L.ncell,
                                cudaMemcpyDeviceToDevice, s));
    DW_LAUNCHED("lbm_home_step");
    return DW_OK;
}

extern "C" dw_status lbm_home_macroscopic(dw_lbm h, const float *m, const uint8_t *solid,
                                          float *rho, float *u, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(m, "m must not be NULL");
    if (!rho && !u) return DW_OK;
    k_home_macroscopic<<<grid_for(h->L.ncell, 256), 256, 0, as_stream(stream)>>>(h->L, m, solid,
                                                                                 rho, u);
    DW_LAUNCHED("k_home_macroscopic");
    return DW_OK;
}

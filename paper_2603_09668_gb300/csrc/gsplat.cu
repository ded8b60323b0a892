// Particle-bound 3D Gaussians: the covariance update under the MPM
// deformation gradient (Sec. 3.2, Sigma_p(t) = F_p Sigma_p F_p^T) and the
// alpha-blended splatting renderer of Eq. rendering (the 3D Gaussian
// representation: Sigma' = J W Sigma W^T J^T, C = sum T_i c_i alpha_i), with
// its reverse mode down to the particle positions and deformation gradients,
// so that an image loss differentiates through the MPM adjoint.
//
// Pipeline of gs_render (one camera):
//   k_gs_preprocess  per Gaussian: Sigma, camera-space centre, projected
//                    centre mu', the inverse 2D covariance (conic), the pixel
//                    rectangle of the 3-sigma ellipse, depth key;
//   radix sort       stable LSD sort of the depth keys (four 8-bit passes:
//                    block histograms, one scan, order-keeping scatter);
//   tile lists       in depth order, each Gaussian is listed once per 16 x 16
//                    pixel tile its rectangle meets (counts, scan, copies);
//                    a stable sort of the list by tile keeps the depth order
//                    within each tile, and each tile's range is marked;
//   k_gs_render_fwd  one tile per block: its Gaussians are read front to back
//                    in batches of 256 into shared memory, then every pixel
//                    composites them.
// gs_render_backward walks the same ranges front to back again with the
// final colour known (dC/dalpha_i = T_i c_i - (C - C_<=i) / (1 - alpha_i)),
// reduces each Gaussian's pixel contributions per warp before one atomic,
// and k_gs_preprocess_bwd carries the 2D gradients back to x and F.
#include <math.h>
#include <string.h>

#include <new>

#include <algorithm>

#include "common.cuh"

namespace dw {

constexpr int GS_TILE = 16;
constexpr int GS_THREADS = GS_TILE * GS_TILE;  // one pixel per thread
constexpr int RS_THREADS = 256;
constexpr int RS_TILE = RS_THREADS * 16;  // keys per sort block

struct GsCam {
    float R[9], T[3];
    float fx, fy, cx, cy;
    int width, height;
    float near_z;
};

// Per-Gaussian forward quantities recomputed identically by both passes.
struct GsProj {
    float S[6];       // Sigma = F Sigma0 F^T (xx, yy, zz, xy, xz, yz)
    float t[3];       // camera-space centre
    float J[6];       // rows (J00 J01 J02), (J10 J11 J12); J01 = J10 = 0
    float V[6];       // R Sigma R^T
    float s2[3];      // Sigma' (xx, xy, yy)
    float mu[2];
    float conic[3];   // inverse of Sigma' (a, b, c)
    bool visible;
};

__device__ __forceinline__ void sym_full(const float s[6], float M[3][3]) {
    M[0][0] = s[0];
    M[1][1] = s[1];
    M[2][2] = s[2];
    M[0][1] = M[1][0] = s[3];
    M[0][2] = M[2][0] = s[4];
    M[1][2] = M[2][1] = s[5];
}

__device__ __forceinline__ void load_F(const float *__restrict__ F, int64_t n, int64_t i,
                                       float Fm[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Fm[a][b] = F[(3 * a + b) * n + i];
}

__device__ __forceinline__ void cov_update(const float Fm[3][3], const float s0[6], float S[6]) {
    float S0[3][3], FS[3][3];
    sym_full(s0, S0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            FS[a][b] = Fm[a][0] * S0[0][b] + Fm[a][1] * S0[1][b] + Fm[a][2] * S0[2][b];
    float M[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            M[a][b] = FS[a][0] * Fm[b][0] + FS[a][1] * Fm[b][1] + FS[a][2] * Fm[b][2];
    S[0] = M[0][0];
    S[1] = M[1][1];
    S[2] = M[2][2];
    S[3] = M[0][1];
    S[4] = M[0][2];
    S[5] = M[1][2];
}

__device__ __forceinline__ void gs_project(const GsCam &c, const float x[3], const float S[6],
                                           GsProj &p) {
#pragma unroll
    for (int k = 0; k < 6; ++k) p.S[k] = S[k];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        p.t[a] = c.R[3 * a] * x[0] + c.R[3 * a + 1] * x[1] + c.R[3 * a + 2] * x[2] + c.T[a];
    p.visible = p.t[2] > c.near_z;
    const float tz = p.visible ? p.t[2] : 1.0f;
    const float iz = 1.0f / tz;
    p.J[0] = c.fx * iz;
    p.J[1] = 0.0f;
    p.J[2] = -c.fx * p.t[0] * iz * iz;
    p.J[3] = 0.0f;
    p.J[4] = c.fy * iz;
    p.J[5] = -c.fy * p.t[1] * iz * iz;
    float Sm[3][3], RS[3][3], Vm[3][3];
    sym_full(S, Sm);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            RS[a][b] = c.R[3 * a] * Sm[0][b] + c.R[3 * a + 1] * Sm[1][b] + c.R[3 * a + 2] * Sm[2][b];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Vm[a][b] = RS[a][0] * c.R[3 * b] + RS[a][1] * c.R[3 * b + 1] + RS[a][2] * c.R[3 * b + 2];
    p.V[0] = Vm[0][0];
    p.V[1] = Vm[1][1];
    p.V[2] = Vm[2][2];
    p.V[3] = Vm[0][1];
    p.V[4] = Vm[0][2];
    p.V[5] = Vm[1][2];
    // Sigma' = J V J^T with J = [[j0, 0, j2], [0, j4, j5]]
    const float j0 = p.J[0], j2 = p.J[2], j4 = p.J[4], j5 = p.J[5];
    const float JV0[3] = {j0 * Vm[0][0] + j2 * Vm[2][0], j0 * Vm[0][1] + j2 * Vm[2][1],
                          j0 * Vm[0][2] + j2 * Vm[2][2]};
    const float JV1[3] = {j4 * Vm[1][0] + j5 * Vm[2][0], j4 * Vm[1][1] + j5 * Vm[2][1],
                          j4 * Vm[1][2] + j5 * Vm[2][2]};
    p.s2[0] = JV0[0] * j0 + JV0[2] * j2;  // xx
    p.s2[1] = JV0[1] * j4 + JV0[2] * j5;  // xy
    p.s2[2] = JV1[1] * j4 + JV1[2] * j5;  // yy
    const float det = p.s2[0] * p.s2[2] - p.s2[1] * p.s2[1];
    p.visible = p.visible && det > 0.0f;
    const float idet = p.visible ? 1.0f / det : 0.0f;
    p.conic[0] = p.s2[2] * idet;
    p.conic[1] = -p.s2[1] * idet;
    p.conic[2] = p.s2[0] * idet;
    p.mu[0] = c.fx * p.t[0] * iz + c.cx;
    p.mu[1] = c.fy * p.t[1] * iz + c.cy;
}

// ------------------------------------------------------------ covariance --

__global__ void k_gs_covariance(const float *__restrict__ F, const float *__restrict__ s0,
                                int64_t n, float *__restrict__ sigma) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float Fm[3][3], a[6], S[6];
    load_F(F, n, i, Fm);
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = s0[k * n + i];
    cov_update(Fm, a, S);
#pragma unroll
    for (int k = 0; k < 6; ++k) sigma[k * n + i] = S[k];
}

// ------------------------------------------------------------ preprocess --

// Per Gaussian: mu'(2), conic(3), the pixel rectangle [x0, x1] x [y0, y1] of
// the pixel centres inside the 3-sigma ellipse (empty when x1 < x0), and the
// depth key (float bits of t_z, or all ones when not drawn).
__global__ void k_gs_preprocess(GsCam c, const float *__restrict__ x, const float *__restrict__ F,
                                const float *__restrict__ s0, int n, float *__restrict__ mu,
                                float *__restrict__ conic, int4 *__restrict__ rect,
                                uint32_t *__restrict__ key, uint32_t *__restrict__ idx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float Fm[3][3], a[6], S[6];
    load_F(F, n, i, Fm);
#pragma unroll
    for (int k = 0; k < 6; ++k) a[k] = s0[(int64_t)k * n + i];
    cov_update(Fm, a, S);
    const float xp[3] = {x[i], x[(int64_t)n + i], x[2 * (int64_t)n + i]};
    GsProj p;
    gs_project(c, xp, S, p);
    int4 r = make_int4(0, 0, -1, -1);
    if (p.visible) {
        const float rx = 3.0f * sqrtf(p.s2[0]), ry = 3.0f * sqrtf(p.s2[2]);
        // pixel px has its centre at px + 1/2
        const float lx = ceilf(p.mu[0] - rx - 0.5f), hx = floorf(p.mu[0] + rx - 0.5f);
        const float ly = ceilf(p.mu[1] - ry - 0.5f), hy = floorf(p.mu[1] + ry - 0.5f);
        r.x = (int)fmaxf(lx, 0.0f);
        r.y = (int)fmaxf(ly, 0.0f);
        r.z = (int)fminf(hx, (float)(c.width - 1));
        r.w = (int)fminf(hy, (float)(c.height - 1));
        if (!(lx <= hx && ly <= hy)) r = make_int4(0, 0, -1, -1);  // also NaN
    }
    const bool drawn = r.z >= r.x && r.w >= r.y;
    mu[i] = p.mu[0];
    mu[n + i] = p.mu[1];
    conic[i] = p.conic[0];
    conic[n + i] = p.conic[1];
    conic[2 * n + i] = p.conic[2];
    rect[i] = r;
    key[i] = drawn ? __float_as_uint(p.t[2]) : 0xffffffffu;  // t_z > 0: bits order as floats
    idx[i] = (uint32_t)i;
}

// ------------------------------------------------------------ radix sort --

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint32_t *__restrict__ key, int n,
                                                        int shift, int nblocks,
                                                        uint32_t *__restrict__ counts) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * RS_TILE;
    const int end = min(base + RS_TILE, n);
    for (int i = base + threadIdx.x; i < end; i += RS_THREADS)
        atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
    __syncthreads();
    counts[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of counts[0..m) in one block (digit-major, block-minor, so
// the offsets keep the blocks' order within a digit).
__global__ void __launch_bounds__(1024) k_rs_scan(uint32_t *__restrict__ counts, int m) {
    __shared__ uint32_t part[1024];
    const int per = (m + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(b + per, m);
    uint32_t s = 0;
    for (int i = b; i < e; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;  // exclusive prefix of this thread's range
    for (int i = b; i < e; ++i) {
        const uint32_t c = counts[i];
        counts[i] = run;
        run += c;
    }
}

// Stable scatter: each block walks its tile 256 keys at a time in order; a
// key's slot is its digit's running base in the block, plus the same-digit
// keys of earlier warps of the chunk, plus the same-digit lanes before it.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t *__restrict__ kin,
                                                           const uint32_t *__restrict__ vin,
                                                           uint32_t *__restrict__ kout,
                                                           uint32_t *__restrict__ vout, int n,
                                                           int shift, int nblocks,
                                                           const uint32_t *__restrict__ offsets) {
    constexpr int WARPS = RS_THREADS / 32;
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcount[WARPS][257];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    base[threadIdx.x] = offsets[threadIdx.x * nblocks + blockIdx.x];
    const int tile0 = blockIdx.x * RS_TILE;
    const int tile1 = min(tile0 + RS_TILE, n);
    for (int c0 = tile0; c0 < tile1; c0 += RS_THREADS) {
        for (int k = threadIdx.x; k < WARPS * 257; k += RS_THREADS) (&wcount[0][0])[k] = 0u;
        __syncthreads();
        const int i = c0 + threadIdx.x;
        const bool valid = i < tile1;
        const uint32_t kv = valid ? kin[i] : 0u;
        const uint32_t d = valid ? ((kv >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned below = peers & ((1u << lane) - 1u);
        if (below == 0u) wcount[warp][d] = (uint32_t)__popc(peers);  // the lowest lane of a group
        __syncthreads();
        if (valid) {
            uint32_t pos = base[d] + (uint32_t)__popc(below);
            for (int w = 0; w < warp; ++w) pos += wcount[w][d];
            kout[pos] = kv;
            vout[pos] = vin[i];
        }
        __syncthreads();
        {  // advance every digit's base by its count in this chunk
            const int dd = threadIdx.x;
            uint32_t add = 0;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) add += wcount[w][dd];
            base[dd] += add;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ tile lists --

// Tiles met by Gaussian order[k] (its pixel rectangle in 16 x 16 tiles).
__global__ void k_gs_tile_count(const uint32_t *__restrict__ order, const int4 *__restrict__ rect,
                                int n, uint32_t *__restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int4 r = rect[order[k]];
    uint32_t c = 0;
    if (r.z >= r.x && r.w >= r.y)
        c = (uint32_t)((r.z / GS_TILE - r.x / GS_TILE + 1) * (r.w / GS_TILE - r.y / GS_TILE + 1));
    cnt[k] = c;
}

// Exclusive scan of 1024 values per block (256 threads x 4), block totals out.
__global__ void __launch_bounds__(256) k_scan1024(const uint32_t *__restrict__ in, int n,
                                                  uint32_t *__restrict__ out,
                                                  uint32_t *__restrict__ sums) {
    __shared__ uint32_t part[256];
    const int base = blockIdx.x * 1024 + threadIdx.x * 4;
    uint32_t v[4], t = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[j] = base + j < n ? in[base + j] : 0u;
        t += v[j];
    }
    part[threadIdx.x] = t;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        const uint32_t a = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += a;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - t;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == 255) sums[blockIdx.x] = part[255];
}

// out += the scanned block offsets; the total goes to *total.
__global__ void k_scan_finish(uint32_t *__restrict__ out, const uint32_t *__restrict__ cnt, int n,
                              const uint32_t *__restrict__ block_off, uint32_t *__restrict__ total) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t o = out[i] + block_off[i / 1024];
    out[i] = o;
    if (i == n - 1) *total = o + cnt[i];
}

// One entry (tile id, Gaussian) per tile met, written in depth order.
__global__ void k_gs_duplicate(const uint32_t *__restrict__ order, const int4 *__restrict__ rect,
                               const uint32_t *__restrict__ off, int n, int tiles_x,
                               uint32_t *__restrict__ tile_key, uint32_t *__restrict__ gid) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t g = order[k];
    const int4 r = rect[g];
    if (!(r.z >= r.x && r.w >= r.y)) return;
    uint32_t o = off[k];
    for (int ty = r.y / GS_TILE; ty <= r.w / GS_TILE; ++ty)
        for (int tx = r.x / GS_TILE; tx <= r.z / GS_TILE; ++tx) {
            tile_key[o] = (uint32_t)(ty * tiles_x + tx);
            gid[o] = g;
            ++o;
        }
}

// ranges[tile] = [first, last + 1) of the tile's entries in the sorted list.
__global__ void k_gs_tile_ranges(const uint32_t *__restrict__ tile_key, int m,
                                 int2 *__restrict__ ranges) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    const uint32_t t = tile_key[p];
    if (p == 0 || tile_key[p - 1] != t) ranges[t].x = p;
    if (p == m - 1 || tile_key[p + 1] != t) ranges[t].y = p + 1;
}

// ---------------------------------------------------------------- render --

// Load the batch [b0, b0 + 256) of the tile's range of the tile list into
// shared memory (mu', conic, opacity, colour per Gaussian); returns its size.
__device__ __forceinline__ int gs_load_batch(int b0, int end, int n,
                                             const uint32_t *__restrict__ list,
                                             const float *__restrict__ mu,
                                             const float *__restrict__ conic,
                                             const float *__restrict__ color,
                                             const float *__restrict__ opacity, int *s_id,
                                             float (*s_g)[9]) {
    const int cnt = min(GS_THREADS, end - b0);
    if ((int)threadIdx.x < cnt) {
        const int g = (int)list[b0 + threadIdx.x];
        float *r = s_g[threadIdx.x];
        s_id[threadIdx.x] = g;
        r[0] = mu[g];
        r[1] = mu[n + g];
        r[2] = conic[g];
        r[3] = conic[n + g];
        r[4] = conic[2 * n + g];
        r[5] = opacity[g];
        r[6] = color[g];
        r[7] = color[n + g];
        r[8] = color[2 * n + g];
    }
    __syncthreads();
    return cnt;
}

__global__ void __launch_bounds__(GS_THREADS) k_gs_render_fwd(
    GsCam c, int n, const uint32_t *__restrict__ list, const int2 *__restrict__ ranges,
    const float *__restrict__ mu, const float *__restrict__ conic,
    const float *__restrict__ color, const float *__restrict__ opacity,
    float *__restrict__ image, float *__restrict__ image_keep) {
    __shared__ int s_id[GS_THREADS];
    __shared__ float s_g[GS_THREADS][9];  // mu(2) conic(3) opacity color(3)
    const int tx0 = blockIdx.x * GS_TILE, ty0 = blockIdx.y * GS_TILE;
    const int px = tx0 + (threadIdx.x & (GS_TILE - 1)), py = ty0 + threadIdx.x / GS_TILE;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const int2 rg = ranges[blockIdx.y * gridDim.x + blockIdx.x];
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    for (int b0 = rg.x; b0 < rg.y; b0 += GS_THREADS) {
        const int cnt = gs_load_batch(b0, rg.y, n, list, mu, conic, color, opacity, s_id, s_g);
        for (int k = 0; k < cnt; ++k) {
            const float *r = s_g[k];
            const float dx = fx - r[0], dy = fy - r[1];
            const float q = r[2] * dx * dx + 2.0f * r[3] * dx * dy + r[4] * dy * dy;
            if (q <= 9.0f) {
                const float a = r[5] * expf(-0.5f * q);
                const float w = T * a;
                C0 += w * r[6];
                C1 += w * r[7];
                C2 += w * r[8];
                T *= 1.0f - a;
            }
        }
        __syncthreads();
    }
    if (px < c.width && py < c.height) {
        const int64_t hw = (int64_t)c.width * c.height, pix = (int64_t)py * c.width + px;
        image[pix] = C0;
        image[hw + pix] = C1;
        image[2 * hw + pix] = C2;
        image_keep[pix] = C0;
        image_keep[hw + pix] = C1;
        image_keep[2 * hw + pix] = C2;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per pixel, front to back: w = T alpha, dL/dc += g w, dL/dalpha = g . (T c -
// (C - C_<=i) / (1 - alpha)), then dL/do, dL/dmu', dL/dconic; each Gaussian's
// nine sums over a warp's pixels go to memory from nine lanes at once.
__global__ void __launch_bounds__(GS_THREADS) k_gs_render_bwd(
    GsCam c, int n, const uint32_t *__restrict__ list, const int2 *__restrict__ ranges,
    const float *__restrict__ mu, const float *__restrict__ conic,
    const float *__restrict__ color, const float *__restrict__ opacity,
    const float *__restrict__ image_keep, const float *__restrict__ g_image,
    float *__restrict__ g2d) {
    __shared__ int s_id[GS_THREADS];
    __shared__ float s_g[GS_THREADS][9];
    const int tx0 = blockIdx.x * GS_TILE, ty0 = blockIdx.y * GS_TILE;
    const int px = tx0 + (threadIdx.x & (GS_TILE - 1)), py = ty0 + threadIdx.x / GS_TILE;
    const bool inside = px < c.width && py < c.height;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const int64_t hw = (int64_t)c.width * c.height, pix = (int64_t)py * c.width + px;
    float Cf[3] = {0.0f, 0.0f, 0.0f}, gC[3] = {0.0f, 0.0f, 0.0f};
    if (inside) {
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            Cf[ch] = image_keep[ch * hw + pix];
            gC[ch] = g_image[ch * hw + pix];
        }
    }
    float T = 1.0f, Cl[3] = {0.0f, 0.0f, 0.0f};
    const int lane = threadIdx.x & 31;
    const int2 rg = ranges[blockIdx.y * gridDim.x + blockIdx.x];
    for (int b0 = rg.x; b0 < rg.y; b0 += GS_THREADS) {
        const int cnt = gs_load_batch(b0, rg.y, n, list, mu, conic, color, opacity, s_id, s_g);
        for (int k = 0; k < cnt; ++k) {
            const float *r = s_g[k];
            const float dx = fx - r[0], dy = fy - r[1];
            const float q = r[2] * dx * dx + 2.0f * r[3] * dx * dy + r[4] * dy * dy;
            float v[9] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            const bool hit = inside && q <= 9.0f;
            if (hit) {
                const float e = expf(-0.5f * q);
                const float a = r[5] * e;
                const float w = T * a;
                float dA = 0.0f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    Cl[ch] += w * r[6 + ch];
                    dA += gC[ch] * (T * r[6 + ch] - (Cf[ch] - Cl[ch]) / (1.0f - a));
                    v[6 + ch] = gC[ch] * w;  // dL/dcolor
                }
                v[5] = dA * e;                 // dL/dopacity
                const float dq = -0.5f * a * dA;  // dL/dq
                v[0] = -2.0f * dq * (r[2] * dx + r[3] * dy);  // dL/dmu'
                v[1] = -2.0f * dq * (r[3] * dx + r[4] * dy);
                v[2] = dq * dx * dx;           // dL/dconic a, b, c
                v[3] = dq * 2.0f * dx * dy;
                v[4] = dq * dy * dy;
                T *= 1.0f - a;
            }
            if (__any_sync(0xffffffffu, hit)) {
                // the xor sums leave all nine totals in every lane: lane j adds total j
                float mine = 0.0f;
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    const float sj = warp_sum(v[j]);
                    mine = lane == j ? sj : mine;
                }
                if (lane < 9 && mine != 0.0f) atomicAdd(&g2d[(int64_t)lane * n + s_id[k]], mine);
            }
        }
        __syncthreads();
    }
}

// dL/d(mu', conic, opacity, color) of each Gaussian -> dL/dx, dL/dF (and the
// colour and opacity gradients), accumulated into the caller's buffers.
__global__ void k_gs_preprocess_bwd(GsCam c, const float *__restrict__ x,
                                    const float *__restrict__ F, const float *__restrict__ s0,
                                    int n, const float *__restrict__ g2d, float *__restrict__ g_x,
                                    float *__restrict__ g_F, float *__restrict__ g_color,
                                    float *__restrict__ g_opacity) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t nn = n;
    float gv[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) gv[j] = g2d[j * nn + i];
    if (g_opacity) g_opacity[i] += gv[5];
    if (g_color) {
        g_color[i] += gv[6];
        g_color[nn + i] += gv[7];
        g_color[2 * nn + i] += gv[8];
    }
    float Fm[3][3], a6[6], S[6];
    load_F(F, nn, i, Fm);
#pragma unroll
    for (int k = 0; k < 6; ++k) a6[k] = s0[k * nn + i];
    cov_update(Fm, a6, S);
    const float xp[3] = {x[i], x[nn + i], x[2 * nn + i]};
    GsProj p;
    gs_project(c, xp, S, p);
    if (!p.visible) return;
    // conic A = Sigma'^-1: dL/dSigma' = -A Abar A, Abar = [[ga, gb/2], [gb/2, gc]]
    const float A00 = p.conic[0], A01 = p.conic[1], A11 = p.conic[2];
    const float b00 = gv[2], b01 = 0.5f * gv[3], b11 = gv[4];
    const float M00 = b00 * A00 + b01 * A01, M01 = b00 * A01 + b01 * A11;  // Abar A
    const float M10 = b01 * A00 + b11 * A01, M11 = b01 * A01 + b11 * A11;
    const float G00 = -(A00 * M00 + A01 * M10), G01 = -(A00 * M01 + A01 * M11);
    const float G11 = -(A01 * M01 + A11 * M11);
    const float G[2][2] = {{G00, G01}, {G01, G11}};
    const float J[2][3] = {{p.J[0], p.J[1], p.J[2]}, {p.J[3], p.J[4], p.J[5]}};
    float V[3][3];
    sym_full(p.V, V);
    // dL/dV = J^T G J ; dL/dJ = 2 G J V
    float GJ[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int b = 0; b < 3; ++b) GJ[r][b] = G[r][0] * J[0][b] + G[r][1] * J[1][b];
    float dV[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) dV[a][b] = J[0][a] * GJ[0][b] + J[1][a] * GJ[1][b];
    float dJ[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            dJ[r][b] = 2.0f * (GJ[r][0] * V[0][b] + GJ[r][1] * V[1][b] + GJ[r][2] * V[2][b]);
    // dL/dSigma = R^T dV R
    float RtdV[3][3], dS[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            RtdV[a][b] = c.R[a] * dV[0][b] + c.R[3 + a] * dV[1][b] + c.R[6 + a] * dV[2][b];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            dS[a][b] = RtdV[a][0] * c.R[b] + RtdV[a][1] * c.R[3 + b] + RtdV[a][2] * c.R[6 + b];
    // dL/dF = 2 dS F Sigma0
    float S0[3][3], FS0[3][3];
    sym_full(a6, S0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            FS0[a][b] = Fm[a][0] * S0[0][b] + Fm[a][1] * S0[1][b] + Fm[a][2] * S0[2][b];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            g_F[(3 * a + b) * nn + i] +=
                2.0f * (dS[a][0] * FS0[0][b] + dS[a][1] * FS0[1][b] + dS[a][2] * FS0[2][b]);
    // camera-space centre: from mu' and from J
    const float iz = 1.0f / p.t[2], iz2 = iz * iz, iz3 = iz2 * iz;
    float gt[3];
    gt[0] = gv[0] * c.fx * iz + dJ[0][2] * (-c.fx * iz2);
    gt[1] = gv[1] * c.fy * iz + dJ[1][2] * (-c.fy * iz2);
    gt[2] = -gv[0] * c.fx * p.t[0] * iz2 - gv[1] * c.fy * p.t[1] * iz2 +
            dJ[0][0] * (-c.fx * iz2) + dJ[0][2] * (2.0f * c.fx * p.t[0] * iz3) +
            dJ[1][1] * (-c.fy * iz2) + dJ[1][2] * (2.0f * c.fy * p.t[1] * iz3);
#pragma unroll
    for (int b = 0; b < 3; ++b)
        g_x[b * nn + i] += c.R[b] * gt[0] + c.R[3 + b] * gt[1] + c.R[6 + b] * gt[2];
}

__global__ void __launch_bounds__(256) k_image_l1(const float *__restrict__ img,
                                                  const float *__restrict__ target, int64_t n,
                                                  float weight, float *__restrict__ loss,
                                                  float *__restrict__ g) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float term = 0.0f;
    if (i < n) {
        const float d = img[i] - target[i];
        term = fabsf(d);
        if (g) g[i] += weight * (d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f));
    }
    __shared__ float red[8];
    term = warp_sum(term);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x < 32) {
        float s = threadIdx.x < 8 ? red[threadIdx.x] : 0.0f;
        s = warp_sum(s);
        if (threadIdx.x == 0) atomicAdd(loss, weight * s);
    }
}

// ----------------------------------------------------------------- D-SSIM --
// The structural term of L_render: 1 - mean SSIM with local statistics under
// an 11 x 11 Gaussian window (sigma 1.5, zero outside the image), computed as
// separable blurs: horizontal sums of the five maps x, y, x^2, y^2, x y, then
// vertical sums; the gradient blurs the per-pixel partials back the same way
// (the window is symmetric, so the transposed blur is the blur).

struct SsimWin {
    float w[11];
};

__global__ void k_ssim_h5(const float *__restrict__ x, const float *__restrict__ y, int C, int H,
                          int W, SsimWin k, float *__restrict__ out) {
    const int64_t plane = (int64_t)C * H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= plane) return;
    const int px = (int)(i % W);
    const int64_t row = i - px;
    float s[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int d = -5; d <= 5; ++d) {
        const int q = px + d;
        if (q < 0 || q >= W) continue;
        const float a = x[row + q], b = y[row + q], w = k.w[d + 5];
        s[0] += w * a;
        s[1] += w * b;
        s[2] += w * a * a;
        s[3] += w * b * b;
        s[4] += w * a * b;
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) out[m * plane + i] = s[m];
}

// One-direction blur of `maps` planes of H x W (horizontal: dir 0, vertical: 1).
__global__ void k_blur(const float *__restrict__ in, int64_t maps, int H, int W, int dir, SsimWin k,
                       float *__restrict__ out) {
    const int64_t total = maps * H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int px = (int)(i % W), py = (int)((i / W) % H);
    const int64_t base = i - px - (int64_t)py * W;  // start of this plane
    float s = 0.0f;
#pragma unroll
    for (int d = -5; d <= 5; ++d) {
        const int qx = dir == 0 ? px + d : px, qy = dir == 0 ? py : py + d;
        if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
        s += k.w[d + 5] * in[base + (int64_t)qy * W + qx];
    }
    out[i] = s;
}

// SSIM per pixel from the blurred maps (mu_x, mu_y, <x^2>, <y^2>, <x y>);
// loss += weight (1 - mean SSIM); part = weight * dD/d(mu_x, <x^2>, <x y>).
__global__ void __launch_bounds__(256) k_ssim_map(const float *__restrict__ v5, int64_t n,
                                                  float weight, float *__restrict__ loss,
                                                  float *__restrict__ part) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    const float scale = -weight / (float)n;
    float term = 0.0f;
    if (i < n) {
        const float A = v5[i], Ay = v5[n + i], B = v5[2 * n + i], Byy = v5[3 * n + i],
                    Cxy = v5[4 * n + i];
        const float n1 = 2.0f * A * Ay + C1, n2 = 2.0f * (Cxy - A * Ay) + C2;
        const float d1 = A * A + Ay * Ay + C1, d2 = (B - A * A) + (Byy - Ay * Ay) + C2;
        const float dd = d1 * d2;
        const float S = n1 * n2 / dd;
        term = S;
        if (part) {
            const float dA = 2.0f * Ay * (n2 - n1) / dd - 2.0f * A * n1 * n2 * (d2 - d1) / (dd * dd);
            const float dB = -S / d2;
            const float dC = 2.0f * n1 / dd;
            part[i] = scale * dA;
            part[n + i] = scale * dB;
            part[2 * n + i] = scale * dC;
        }
    }
    __shared__ float red[8];
    term = warp_sum(term);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < 8 ? red[threadIdx.x] : 0.0f;
        t = warp_sum(t);
        if (threadIdx.x == 0) atomicAdd(loss, scale * t + (blockIdx.x == 0 ? weight : 0.0f));
    }
}

// g += blur(p_mu) + 2 x blur(p_xx) + y blur(p_xy)
__global__ void k_ssim_grad(const float *__restrict__ x, const float *__restrict__ y,
                            const float *__restrict__ bp, int64_t n, float *__restrict__ g) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    g[i] += bp[i] + 2.0f * x[i] * bp[n + i] + y[i] * bp[2 * n + i];
}

static SsimWin ssim_window() {
    SsimWin k;
    double w[11], sum = 0.0;
    for (int i = 0; i < 11; ++i) {
        w[i] = exp(-((i - 5.0) * (i - 5.0)) / (2.0 * 1.5 * 1.5));
        sum += w[i];
    }
    for (int i = 0; i < 11; ++i) k.w[i] = (float)(w[i] / sum);
    return k;
}

struct GsHandle {
    int64_t cap = 0;
    int width = 0, height = 0;
    float *mu = nullptr, *conic = nullptr, *g2d = nullptr, *image = nullptr;
    int4 *rect = nullptr;
    uint32_t *key = nullptr, *idx = nullptr, *key2 = nullptr, *idx2 = nullptr, *counts = nullptr;
    uint32_t *tcnt = nullptr, *toff = nullptr, *bsum = nullptr, *total = nullptr;
    int2 *ranges = nullptr;  // [tiles]
    // tile list: (tile key, Gaussian) entries and their sort buffers
    int64_t list_cap = 0;
    uint32_t *lkey = nullptr, *lgid = nullptr, *lkey2 = nullptr, *lgid2 = nullptr,
             *lcounts = nullptr;
    const uint32_t *list = nullptr;  // the sorted Gaussian column of the last gs_render
    int tiles_x = 0, tiles_y = 0;
    int last_n = -1;  // Gaussians of the last gs_render
    // inputs and camera of the last gs_render (the backward must see the same)
    const void *last_in[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    dw_camera last_cam{};
};

static GsCam to_cam(const dw_camera &c) {
    GsCam g;
    for (int k = 0; k < 9; ++k) g.R[k] = c.R[k];
    for (int k = 0; k < 3; ++k) g.T[k] = c.T[k];
    g.fx = c.fx;
    g.fy = c.fy;
    g.cx = c.cx;
    g.cy = c.cy;
    g.width = c.width;
    g.height = c.height;
    g.near_z = c.near_z;
    return g;
}

// Stable LSD radix sort of (k, v) by the low 8 * passes bits of k; the
// result ends in (k, v) (the pointers are swapped as the passes alternate).
static void radix_sort(uint32_t *&k, uint32_t *&v, uint32_t *&k2, uint32_t *&v2, int n,
                       int passes, uint32_t *counts, cudaStream_t s) {
    const int nb = (n + RS_TILE - 1) / RS_TILE;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<nb, RS_THREADS, 0, s>>>(k, n, shift, nb, counts);
        k_rs_scan<<<1, 1024, 0, s>>>(counts, 256 * nb);
        k_rs_scatter<<<nb, RS_THREADS, 0, s>>>(k, v, k2, v2, n, shift, nb, counts);
        std::swap(k, k2);
        std::swap(v, v2);
    }
}

}  // namespace dw

using namespace dw;

struct dw_gs_s : GsHandle {};

// Grow the tile-list buffers to hold m entries.
static dw_status gs_list_reserve(dw_gs h, int64_t m) {
    if (m <= h->list_cap) return DW_OK;
    const int64_t cap = std::max<int64_t>(m, h->list_cap * 3 / 2);
    DW_REQUIRE(cap < (1ll << 31), "tile list too long (Gaussians x tiles met >= 2^31)");
    cudaFree(h->lkey);
    cudaFree(h->lgid);
    cudaFree(h->lkey2);
    cudaFree(h->lgid2);
    cudaFree(h->lcounts);
    h->lkey = h->lgid = h->lkey2 = h->lgid2 = h->lcounts = nullptr;
    h->list_cap = 0;
    const size_t c = (size_t)cap, nb = (c + RS_TILE - 1) / RS_TILE;
    cudaError_t e = cudaMalloc((void **)&h->lkey, sizeof(uint32_t) * c);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->lgid, sizeof(uint32_t) * c);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->lkey2, sizeof(uint32_t) * c);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->lgid2, sizeof(uint32_t) * c);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->lcounts, sizeof(uint32_t) * 256 * nb);
    if (e != cudaSuccess) return cuda_fail(e, "gs_render (tile list)");
    h->list_cap = cap;
    return DW_OK;
}

extern "C" dw_status gs_create(int64_t max_gaussians, int32_t width, int32_t height, dw_gs *out) {
    DW_REQUIRE(out, "out must not be NULL");
    *out = nullptr;
    DW_REQUIRE(max_gaussians >= 1 && max_gaussians < (1ll << 30), "max_gaussians must be in [1, 2^30)");
    DW_REQUIRE(width >= 1 && height >= 1 && (int64_t)width * height < (1ll << 31),
               "image size must be positive and below 2^31 pixels");
    dw_gs h = new (std::nothrow) dw_gs_s();
    if (!h) {
        set_error("out of host memory");
        return DW_ERR_OOM;
    }
    h->cap = max_gaussians;
    h->width = width;
    h->height = height;
    const size_t n = (size_t)max_gaussians, nb = (n + RS_TILE - 1) / RS_TILE;
    cudaError_t e = cudaMalloc((void **)&h->mu, sizeof(float) * 2 * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->conic, sizeof(float) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->g2d, sizeof(float) * 9 * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->rect, sizeof(int4) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->key, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->idx, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->key2, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->idx2, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->counts, sizeof(uint32_t) * 256 * nb);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&h->image, sizeof(float) * 3 * (size_t)width * height);
    h->tiles_x = (width + GS_TILE - 1) / GS_TILE;
    h->tiles_y = (height + GS_TILE - 1) / GS_TILE;
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->tcnt, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->toff, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->bsum, sizeof(uint32_t) * ((n + 1023) / 1024));
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->total, sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&h->ranges, sizeof(int2) * (size_t)h->tiles_x * h->tiles_y);
    if (e != cudaSuccess) {
        dw_status st = cuda_fail(e, "gs_create");
        gs_destroy(h);
        return st;
    }
    *out = h;
    return DW_OK;
}

extern "C" dw_status gs_destroy(dw_gs h) {
    if (!h) return DW_OK;
    cudaFree(h->mu);
    cudaFree(h->conic);
    cudaFree(h->g2d);
    cudaFree(h->rect);
    cudaFree(h->key);
    cudaFree(h->idx);
    cudaFree(h->key2);
    cudaFree(h->idx2);
    cudaFree(h->counts);
    cudaFree(h->image);
    cudaFree(h->tcnt);
    cudaFree(h->toff);
    cudaFree(h->bsum);
    cudaFree(h->total);
    cudaFree(h->ranges);
    cudaFree(h->lkey);
    cudaFree(h->lgid);
    cudaFree(h->lkey2);
    cudaFree(h->lgid2);
    cudaFree(h->lcounts);
    delete h;
    return DW_OK;
}

extern "C" dw_status gs_covariance(const float *F, const float *sigma0, int64_t n, float *sigma,
                                   dw_stream stream) {
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(F && sigma0 && sigma, "F, sigma0 and sigma must not be NULL");
    k_gs_covariance<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(F, sigma0, n, sigma);
    DW_LAUNCHED("k_gs_covariance");
    return DW_OK;
}

static dw_status gs_check(dw_gs h, const dw_camera *cam, const float *x, const float *F,
                          const float *sigma0, const float *color, const float *opacity,
                          int64_t n) {
    DW_REQUIRE(h && cam, "handle and camera must not be NULL");
    DW_REQUIRE(n >= 0 && n <= h->cap, "n must be in [0, max_gaussians]");
    DW_REQUIRE(cam->width == h->width && cam->height == h->height,
               "camera image size differs from the handle's");
    DW_REQUIRE(cam->fx > 0.0f && cam->fy > 0.0f && cam->near_z > 0.0f,
               "focal lengths and near must be > 0");
    DW_REQUIRE(n == 0 || (x && F && sigma0 && color && opacity), "inputs must not be NULL");
    return DW_OK;
}

extern "C" dw_status gs_render(dw_gs h, const dw_camera *cam, const float *x, const float *F,
                               const float *sigma0, const float *color, const float *opacity,
                               int64_t n, float *image, dw_stream stream) {
    dw_status st = gs_check(h, cam, x, F, sigma0, color, opacity, n);
    if (st != DW_OK) return st;
    DW_REQUIRE(image, "image must not be NULL");
    cudaStream_t s = as_stream(stream);
    const GsCam c = to_cam(*cam);
    const int nn = (int)n;
    const int ntiles = h->tiles_x * h->tiles_y;
    DW_CUDA(cudaMemsetAsync(h->ranges, 0, sizeof(int2) * (size_t)ntiles, s));
    h->list = h->lgid;
    if (nn > 0) {
        k_gs_preprocess<<<grid_for(nn, 256), 256, 0, s>>>(c, x, F, sigma0, nn, h->mu, h->conic,
                                                          h->rect, h->key, h->idx);
        uint32_t *ka = h->key, *va = h->idx, *kb = h->key2, *vb = h->idx2;
        radix_sort(ka, va, kb, vb, nn, 4, h->counts, s);  // depth order in (ka, va)
        // tile list: counts in depth order, offsets, total
        k_gs_tile_count<<<grid_for(nn, 256), 256, 0, s>>>(va, h->rect, nn, h->tcnt);
        const int nsb = (nn + 1023) / 1024;
        k_scan1024<<<nsb, 256, 0, s>>>(h->tcnt, nn, h->toff, h->bsum);
        k_rs_scan<<<1, 1024, 0, s>>>(h->bsum, nsb);
        k_scan_finish<<<grid_for(nn, 256), 256, 0, s>>>(h->toff, h->tcnt, nn, h->bsum, h->total);
        uint32_t m = 0;
        DW_CUDA(cudaMemcpyAsync(&m, h->total, sizeof m, cudaMemcpyDeviceToHost, s));
        DW_CUDA(cudaStreamSynchronize(s));
        if (m > 0) {
            dw_status st2 = gs_list_reserve(h, (int64_t)m);
            if (st2 != DW_OK) return st2;
            k_gs_duplicate<<<grid_for(nn, 256), 256, 0, s>>>(va, h->rect, h->toff, nn, h->tiles_x,
                                                             h->lkey, h->lgid);
            int bits = 1;
            while ((1 << bits) < ntiles) ++bits;
            uint32_t *lk = h->lkey, *lv = h->lgid, *lk2 = h->lkey2, *lv2 = h->lgid2;
            radix_sort(lk, lv, lk2, lv2, (int)m, (bits + 7) / 8, h->lcounts, s);
            k_gs_tile_ranges<<<grid_for(m, 256), 256, 0, s>>>(lk, (int)m, h->ranges);
            h->list = lv;
        }
    }
    const dim3 grid((unsigned)h->tiles_x, (unsigned)h->tiles_y);
    k_gs_render_fwd<<<grid, GS_THREADS, 0, s>>>(c, nn, h->list, h->ranges, h->mu, h->conic, color,
                                                 opacity, image, h->image);
    h->last_n = nn;
    const void *in[5] = {x, F, sigma0, color, opacity};
    memcpy(h->last_in, in, sizeof in);
    h->last_cam = *cam;
    DW_LAUNCHED("gs_render");
    return DW_OK;
}

extern "C" dw_status gs_render_backward(dw_gs h, const dw_camera *cam, const float *x,
                                        const float *F, const float *sigma0, const float *color,
                                        const float *opacity, int64_t n, const float *g_image,
                                        float *g_x, float *g_F, float *g_color, float *g_opacity,
                                        dw_stream stream) {
    dw_status st = gs_check(h, cam, x, F, sigma0, color, opacity, n);
    if (st != DW_OK) return st;
    DW_REQUIRE(g_image && g_x && g_F, "g_image, g_x and g_F must not be NULL");
    const void *in[5] = {x, F, sigma0, color, opacity};
    DW_REQUIRE(h->last_n == (int)n && memcmp(h->last_in, in, sizeof in) == 0 &&
                   memcmp(&h->last_cam, cam, sizeof *cam) == 0,
               "gs_render_backward must follow gs_render of the same Gaussians and camera");
    if (n == 0) return DW_OK;
    cudaStream_t s = as_stream(stream);
    const GsCam c = to_cam(*cam);
    const int nn = (int)n;
    DW_CUDA(cudaMemsetAsync(h->g2d, 0, sizeof(float) * 9 * (size_t)nn, s));
    const dim3 grid((unsigned)h->tiles_x, (unsigned)h->tiles_y);
    k_gs_render_bwd<<<grid, GS_THREADS, 0, s>>>(c, nn, h->list, h->ranges, h->mu, h->conic, color,
                                                 opacity, h->image, g_image, h->g2d);
    k_gs_preprocess_bwd<<<grid_for(nn, 256), 256, 0, s>>>(c, x, F, sigma0, nn, h->g2d, g_x, g_F,
                                                           g_color, g_opacity);
    DW_LAUNCHED("gs_render_backward");
    return DW_OK;
}

extern "C" dw_status image_l1_loss(const float *image, const float *target, int64_t n,
                                   float weight, float *loss, float *g_image, dw_stream stream) {
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(image && target && loss, "image, target and loss must not be NULL");
    k_image_l1<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(image, target, n, weight, loss,
                                                                 g_image);
    DW_LAUNCHED("k_image_l1");
    return DW_OK;
}

extern "C" dw_status image_dssim_loss(const float *image, const float *target, int32_t channels,
                                      int32_t height, int32_t width, float weight, float *loss,
                                      float *g_image, float *workspace, dw_stream stream) {
    DW_REQUIRE(channels >= 1 && height >= 1 && width >= 1, "image sizes must be >= 1");
    const int64_t n = (int64_t)channels * height * width;
    DW_REQUIRE(10 * n < (1ll << 31), "image too large (10 C H W must be < 2^31)");
    DW_REQUIRE(image && target && loss && workspace, "image, target, loss and workspace must not be NULL");
    cudaStream_t s = as_stream(stream);
    const SsimWin k = ssim_window();
    float *h5 = workspace, *v5 = workspace + 5 * n;
    k_ssim_h5<<<grid_for(n, 256), 256, 0, s>>>(image, target, channels, height, width, k, h5);
    k_blur<<<grid_for(5 * n, 256), 256, 0, s>>>(h5, 5 * (int64_t)channels, height, width, 1, k, v5);
    float *part = g_image ? workspace : nullptr;  // h5 is free again
    k_ssim_map<<<grid_for(n, 256), 256, 0, s>>>(v5, n, weight, loss, part);
    if (g_image) {
        k_blur<<<grid_for(3 * n, 256), 256, 0, s>>>(part, 3 * (int64_t)channels, height, width, 0,
                                                     k, v5);
        k_blur<<<grid_for(3 * n, 256), 256, 0, s>>>(v5, 3 * (int64_t)channels, height, width, 1,
                                                     k, part);
        k_ssim_grad<<<grid_for(n, 256), 256, 0, s>>>(image, target, part, n, g_image);
    }
    DW_LAUNCHED("image_dssim_loss");
    return DW_OK;
}

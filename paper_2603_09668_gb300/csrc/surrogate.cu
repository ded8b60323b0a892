// Learned surrogate of the LBM wind constraint: a 4-layer 3D conv network on
// a coarse n^3 grid (channels 16 -> 32 -> 32 -> 32 -> 16, kernel 3, GELU after
// layers 1-3) that maps the coarse state (rho - 1, u, solid fraction) of a
// (2n)^3 lattice to the change du of the coarse velocity over a block of
// lattice steps. Training and inference run in the library's kernels: BF16
// tensor-core convolutions with FP32 accumulation (surrogate_conv.cuh), FP32
// master weights and Adam. The paper has no learned component; Sec. 3.4 uses
// the LBM velocity field as the guide that this network stands in for.
#include <cudaTypedefs.h>

#include <algorithm>
#include <new>

#include "surrogate_tc.cuh"
#include "surrogate_wgrad_tc.cuh"

namespace dw {

static const int SCH[5] = {16, 32, 32, 32, 16};

struct SurrHandle {
    int n = 0;           // coarse grid per axis
    int64_t nv = 0;      // n^3
    int64_t nparams = 0;
    int64_t off_w[4] = {0, 0, 0, 0}, off_b[4] = {0, 0, 0, 0};
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wf = nullptr;  // forward weights, per layer [9][cin/8][3][cout][8]
    bf16 *wd = nullptr;  // input-gradient weights, per layer [9][cout/8][3][cin][8], taps mirrored
    int64_t woff[4] = {0, 0, 0, 0};
    bf16 *feats = nullptr;          // [nv][16]
    bf16 *z[3] = {nullptr, nullptr, nullptr}, *a[3] = {nullptr, nullptr, nullptr};  // [nv][32]
    float *out = nullptr;           // [nv][16]
    float *out4 = nullptr;          // [nv][4]: channels 0-3 of out (the chained update's input)
    bf16 *g4 = nullptr;             // [nv][16]: dL/d(out)
    bf16 *gz[3] = {nullptr, nullptr, nullptr};  // [nv][32]: dL/dz of layers 1..3
    float *part = nullptr, *part_b = nullptr;   // weight-gradient partials
    int nchunks = 0, tiles_per_chunk = 0;
    float *fine = nullptr;          // [4][(2n)^3]: rho, ux, uy, uz of the last surr_features
    float *corr = nullptr;          // [3][(2n)^3] defect correction of the chained update
    float uref[3] = {0.f, 0.f, 0.f};  // reference (inlet) velocity of the features
    bool corr_on = false;           // corr is added by surr_advance_fine
    double *red = nullptr;          // reduction scratch
    int *err = nullptr;             // device status bits (bounded waits of the conv kernels)
    unsigned *gbar = nullptr;       // grid barrier of the one-launch forward (arrivals, generation)
    bool fused = true;              // the one-launch forward can be launched (cooperatively)
    bool fused_attr_set = false;
    int conv_ctas = 0;
    int sms = 0;
    // the BF16 weights were rewritten since the last forward: its first layer,
    // which copies them before its dependency wait, is then launched normally
    bool weights_dirty = true;
    // TMA descriptors of the conv inputs: features, a1..a3, dL/d(out), dL/dz1..dz3
    CUtensorMap tm_feats, tm_a[3], tm_g4, tm_gz[3];
    // and of the weight-gradient kernel's operands: layer l's input (features,
    // a1..a3) and its output gradient (dL/dz1..dz3, dL/d(out))
    CUtensorMap tmw_in[4], tmw_g[4];
    int part_chunks = 0;            // capacity of part / part_b in CTA partials
};

// ------------------------------------------------------------- kernels ----

// BF16 copies of the layer weights in the tensor-core operand layout
// [9 (dy, dx)][cin/8][3 (dz)][cout][8] (core matrices of 8 output channels x 8
// input channels; the three dz taps of one (dx, dy) form one operand): wf for
// the forward convolution, wd for the input gradient (taps mirrored, input
// and output channels swapped).
__global__ void k_surr_weights(const float *__restrict__ params, bf16 *__restrict__ wf,
                               bf16 *__restrict__ wd, int64_t off_w, int64_t woff, int cin,
                               int cout) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t cnt = 27LL * cin * cout;
    if (i >= cnt) return;
    const int ci = (int)(i % cin), co = (int)((i / cin) % cout), t = (int)(i / ((int64_t)cin * cout));
    const bf16 w = __float2bfloat16_rn(params[off_w + i]);
    const int t2 = 26 - t;  // tap of the input-gradient convolution
    wf[woff + ((((int64_t)(t % 9) * (cin / 8) + ci / 8) * 3 + t / 9) * cout + co) * 8 + (ci & 7)] = w;
    wd[woff + ((((int64_t)(t2 % 9) * (cout / 8) + co / 8) * 3 + t2 / 9) * cin + ci) * 8 + (co & 7)] = w;
}

__device__ __constant__ int kCX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0};
__device__ __constant__ int kCY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 1, -1};
__device__ __constant__ int kCZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 1, -1, 1};

// Fine rho and u of every cell of a shifted (2n)^3 lattice (solid: rho 1, u 0).
__global__ void k_surr_fine(const float *__restrict__ f, const uint8_t *__restrict__ solid, int N,
                            float *__restrict__ fine) {
    const int64_t nc = (int64_t)N * N * N;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    float r = 1.0f, ux = 0.0f, uy = 0.0f, uz = 0.0f;
    if (!(solid && solid[c])) {
        float rs = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float fi = f[(size_t)i * nc + c];
            rs += fi;
            jx += (float)kCX[i] * fi;
            jy += (float)kCY[i] * fi;
            jz += (float)kCZ[i] * fi;
        }
        r = 1.0f + rs;
        ux = jx / r;
        uy = jy / r;
        uz = jz / r;
    }
    fine[c] = r;
    fine[nc + c] = ux;
    fine[2 * nc + c] = uy;
    fine[3 * nc + c] = uz;
}

// Coarse features: 2x2x2 averages over fluid cells of (rho - 1, u), solid fraction.
__global__ void k_surr_coarse(const float *__restrict__ fine, const uint8_t *__restrict__ solid,
                              int n, float in_scale, float3 uref, bf16 *__restrict__ feats,
                              float *__restrict__ feats32) {
    const int64_t nv = (int64_t)n * n * n;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int N = 2 * n;
    const int64_t nc = (int64_t)N * N * N;
    const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)(v / ((int64_t)n * n));
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    int fluid = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int64_t c = ((int64_t)(2 * z + (k >> 2)) * N + (2 * y + ((k >> 1) & 1))) * N + 2 * x + (k & 1);
        if (solid && solid[c]) continue;
        ++fluid;
        s[0] += fine[c] - 1.0f;
        s[1] += fine[nc + c];
        s[2] += fine[2 * nc + c];
        s[3] += fine[3 * nc + c];
    }
    const float inv = fluid > 0 ? in_scale / (float)fluid : 0.0f;
    // velocity relative to the reference velocity, which itself fills channels 5-7
    const float r1 = fluid > 0 ? s[1] * inv - uref.x * in_scale : 0.0f;
    const float r2 = fluid > 0 ? s[2] * inv - uref.y * in_scale : 0.0f;
    const float r3 = fluid > 0 ? s[3] * inv - uref.z * in_scale : 0.0f;
    __align__(16) bf16 o[16];
#pragma unroll
    for (int ch = 0; ch < 16; ++ch) o[ch] = __float2bfloat16_rn(0.0f);
    o[0] = __float2bfloat16_rn(s[0] * inv);
    o[1] = __float2bfloat16_rn(r1);
    o[2] = __float2bfloat16_rn(r2);
    o[3] = __float2bfloat16_rn(r3);
    o[4] = __float2bfloat16_rn((8 - fluid) * 0.125f);
    o[5] = __float2bfloat16_rn(uref.x * in_scale);
    o[6] = __float2bfloat16_rn(uref.y * in_scale);
    o[7] = __float2bfloat16_rn(uref.z * in_scale);
    reinterpret_cast<uint4 *>(feats)[v] = reinterpret_cast<const uint4 *>(o)[0];       // channels 0-7
    reinterpret_cast<uint4 *>(feats)[nv + v] = reinterpret_cast<const uint4 *>(o)[1];  // channels 8-15
    if (feats32) {
        float4 *d32 = reinterpret_cast<float4 *>(feats32 + v * 16);
        d32[0] = make_float4(s[0] * inv, r1, r2, r3);
        d32[1] = make_float4((8 - fluid) * 0.125f, uref.x * in_scale, uref.y * in_scale,
                             uref.z * in_scale);
        d32[2] = make_float4(0.f, 0.f, 0.f, 0.f);
        d32[3] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Channels-last FP32 [nv][16] -> planar BF16 [2][nv][8] (the layout of the
// network's activations: 8-channel planes, see surrogate_tc.cuh).
__global__ void k_cl16_to_planar(const float *__restrict__ src, bf16 *__restrict__ dst, int64_t nv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (chunk, voxel)
    if (i >= 2 * nv) return;
    const int64_t c = i / nv, v = i - c * nv;
    const float4 a = *reinterpret_cast<const float4 *>(src + v * 16 + c * 8);
    const float4 b = *reinterpret_cast<const float4 *>(src + v * 16 + c * 8 + 4);
    __align__(16) bf16 o[8] = {__float2bfloat16_rn(a.x), __float2bfloat16_rn(a.y),
                               __float2bfloat16_rn(a.z), __float2bfloat16_rn(a.w),
                               __float2bfloat16_rn(b.x), __float2bfloat16_rn(b.y),
                               __float2bfloat16_rn(b.z), __float2bfloat16_rn(b.w)};
    reinterpret_cast<uint4 *>(dst)[i] = *reinterpret_cast<const uint4 *>(o);
}

// Planar BF16 [2][nv][8] -> channels-last BF16 [nv][16].
__global__ void k_planar_to_cl16(const bf16 *__restrict__ src, bf16 *__restrict__ dst, int64_t nv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * nv) return;
    const int64_t c = i / nv, v = i - c * nv;
    reinterpret_cast<uint4 *>(dst)[v * 2 + c] = reinterpret_cast<const uint4 *>(src)[i];
}

// Mean squared error over the coarse voxels that are not fully solid, on
// channels 0..2: L = sum (out - target)^2 / (3 count); g4 = dL/d(out).
__global__ void k_surr_loss(const float *__restrict__ out, const float *__restrict__ target,
                            const bf16 *__restrict__ feats, int64_t nv, const int *__restrict__ count,
                            bf16 *__restrict__ g4, float *__restrict__ loss) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float inv_norm = 1.0f / (3.0f * (float)max(*count, 1));
    float l = 0.0f;
    if (v < nv) {
        const bool fluid = __bfloat162float(feats[v * 8 + 4]) < 1.0f;  // solid fraction, plane 0
        __align__(16) bf16 g[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) g[c] = __float2bfloat16_rn(0.0f);
        if (fluid) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float d = out[v * 16 + c] - target[v * 16 + c];
                l += d * d;
                g[c] = __float2bfloat16_rn(2.0f * d * inv_norm);
            }
        }
        reinterpret_cast<uint4 *>(g4)[v] = reinterpret_cast<const uint4 *>(g)[0];
        reinterpret_cast<uint4 *>(g4)[nv + v] = reinterpret_cast<const uint4 *>(g)[1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l * inv_norm);
}

__global__ void k_count_fluid(const bf16 *__restrict__ feats, int64_t nv, int *__restrict__ count) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int c = (v < nv && __bfloat162float(feats[v * 8 + 4]) < 1.0f) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void k_wgrad_reduce(const float *__restrict__ part, const float *__restrict__ part_b,
                               int nchunks, int64_t nw, int cout, float *__restrict__ gw,
                               float *__restrict__ gb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nw) {
        float s = 0.0f;
        for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * nw + i];
        gw[i] += s;
    } else if (i < nw + cout) {
        const int co = (int)(i - nw);
        float s = 0.0f;
        for (int c = 0; c < nchunks; ++c) s += part_b[(size_t)c * cout + co];
        gb[co] += s;
    }
}

__global__ void k_surr_adam(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t cnt, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    g[i] = 0.0f;
}

// f = f_eq(rho, u + du up-sampled) on fluid cells of the (2n)^3 lattice
// (shifted populations), du trilinear from the cell-centred coarse grid.
__global__ void k_surr_apply(const float *__restrict__ out, float out_scale,
                             const float *__restrict__ fine, const uint8_t *__restrict__ solid,
                             int n, float *__restrict__ f) {
    const int N = 2 * n;
    const int64_t nc = (int64_t)N * N * N;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    if (solid && solid[c]) return;
    const int fi[3] = {(int)(c % N), (int)((c / N) % N), (int)(c / ((int64_t)N * N))};
    int i0[3];
    float t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float s = fminf(fmaxf(fi[a] * 0.5f - 0.25f, 0.0f), (float)(n - 1));
        int i = min((int)floorf(s), n - 2);
        i0[a] = i;
        t[a] = s - (float)i;
    }
    float d[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int cx = k & 1, cy = (k >> 1) & 1, cz = k >> 2;
        const float w = (cx ? t[0] : 1.f - t[0]) * (cy ? t[1] : 1.f - t[1]) * (cz ? t[2] : 1.f - t[2]);
        const float *o = out + ((((int64_t)(i0[2] + cz)) * n + (i0[1] + cy)) * n + (i0[0] + cx)) * 16;
        d[0] += w * o[0];
        d[1] += w * o[1];
        d[2] += w * o[2];
    }
    d[0] *= out_scale;
    d[1] *= out_scale;
    d[2] *= out_scale;
    const float rho = fine[c];
    const float ux = fine[nc + c] + d[0], uy = fine[2 * nc + c] + d[1], uz = fine[3 * nc + c] + d[2];
    const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float cu = (float)kCX[i] * ux + (float)kCY[i] * uy + (float)kCZ[i] * uz;
        const float w = i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
        f[(size_t)i * nc + c] = w * ((rho - 1.0f) + rho * (3.0f * cu + 4.5f * cu * cu - uu));
    }
}

// Chained-mode step after a network call: u += out_scale * du upsampled (the
// interpolation of k_surr_apply; rho kept) on every fluid fine cell, then the
// coarse features of the updated state (the arithmetic and summation order of
// k_surr_coarse), so that the next network call can run directly.
// A block covers ADV_VX x ADV_VY x ADV_VZ coarse voxels; each thread takes two
// of their fine cells, ADV_VZ fine slices apart (x fastest: a warp covers 32
// consecutive cells of one fine row), so that every thread has two
// independent sets of loads in flight; the coarse outputs the block
// interpolates from, (ADV_VX + 2) x (ADV_VY + 2) x (ADV_VZ + 2) voxels, are
// staged in shared memory first.
constexpr int ADV_VX = 16, ADV_VY = 2, ADV_VZ = 4;
constexpr int ADV_THREADS = 4 * ADV_VX * ADV_VY * ADV_VZ;  // two fine cells per thread
__global__ void __launch_bounds__(ADV_THREADS) k_surr_advance_fine(
    const float *__restrict__ out4, float out_scale, float *__restrict__ fine,
    const uint8_t *__restrict__ solid, int n, float in_scale, float3 uref,
    bf16 *__restrict__ feats, const float *__restrict__ corr) {
    constexpr int SX = ADV_VX + 2, SY = ADV_VY + 2, SZ = ADV_VZ + 2;
    constexpr int NV = ADV_VX * ADV_VY * ADV_VZ;
    static_assert(SX * SY * SZ <= ADV_THREADS, "one staged voxel per thread");
    __shared__ float du[SZ][SY][SX][3];   // coarse (z, y, x) around the block
    __shared__ float part[8][NV][4];      // per fine cell k of each voxel: (rho - 1, u) or 0
    __shared__ int isf[8][NV];
    const int bxs = n / ADV_VX, bys = n / ADV_VY;
    const int x0 = (blockIdx.x % bxs) * ADV_VX;
    const int y0 = ((blockIdx.x / bxs) % bys) * ADV_VY;
    const int z0 = (blockIdx.x / (bxs * bys)) * ADV_VZ;
    const int N = 2 * n;
    const int64_t nc = (int64_t)N * N * N;
    const int t = threadIdx.x;
    pdl_wait();  // launched as a programmatic dependent of the network's last layer
    pdl_trigger();
    // the thread's two fine cells: (lx, ly, lz) and (lx, ly, lz + 2 ADV_VZ / 2) of the
    // block's 2 ADV_VX x 2 ADV_VY x 2 ADV_VZ cells
    const int lx = t % (2 * ADV_VX), ly = (t / (2 * ADV_VX)) % (2 * ADV_VY);
    const int lzb = t / (4 * ADV_VX * ADV_VY);  // 0 .. ADV_VZ - 1
    // every load is issued before the first barrier: the staged coarse voxel
    // and both fine cells' rho, u and mask (solid cells hold rho = 1, u = 0 and
    // are read but never written)
    float4 st = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < SX * SY * SZ) {
        const int ex = t % SX, ey = (t / SX) % SY, ez = t / (SX * SY);
        const int cx = min(max(x0 - 1 + ex, 0), n - 1), cy = min(max(y0 - 1 + ey, 0), n - 1);
        const int cz = min(max(z0 - 1 + ez, 0), n - 1);
        st = __ldg(reinterpret_cast<const float4 *>(out4) + ((int64_t)cz * n + cy) * n + cx);
    }
    int fi[2][3];
    int64_t c[2];
    float rho[2], u0[2], u1[2], u2[2];
    bool is_solid[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int lz = lzb + h * ADV_VZ;
        fi[h][0] = 2 * x0 + lx;
        fi[h][1] = 2 * y0 + ly;
        fi[h][2] = 2 * z0 + lz;
        c[h] = ((int64_t)fi[h][2] * N + fi[h][1]) * N + fi[h][0];
        rho[h] = fine[c[h]];
        u0[h] = fine[nc + c[h]];
        u1[h] = fine[2 * nc + c[h]];
        u2[h] = fine[3 * nc + c[h]];
        if (corr) {  // the defect measured at the last check, added every block
            u0[h] += corr[c[h]];
            u1[h] += corr[nc + c[h]];
            u2[h] += corr[2 * nc + c[h]];
        }
        is_solid[h] = solid && solid[c[h]];
    }
    if (t < SX * SY * SZ) {
        const int ex = t % SX, ey = (t / SX) % SY, ez = t / (SX * SY);
        du[ez][ey][ex][0] = st.x;
        du[ez][ey][ex][1] = st.y;
        du[ez][ey][ex][2] = st.z;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int lz = lzb + h * ADV_VZ;
        const int k = (lx & 1) + 2 * (ly & 1) + 4 * (lz & 1);  // the cell's place in its voxel
        const int vl = ((lz >> 1) * ADV_VY + (ly >> 1)) * ADV_VX + (lx >> 1);  // voxel within block
        float contrib[4] = {0.f, 0.f, 0.f, 0.f};
        int fl = 0;
        if (!is_solid[h]) {
            // corner and weight of k_surr_apply's interpolation, in integers:
            // fine cell 2v + b sits at coarse v - 1/4 (b = 0) or v + 1/4 (b = 1),
            // so the lower corner is v - 1 + b with weight 0.25 + 0.5 b on the
            // upper one, clamped at both ends of the axis
            int i0[3];
            float tt[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int v = fi[h][a] >> 1, b = fi[h][a] & 1;
                int i = v - 1 + b;
                float t = b ? 0.25f : 0.75f;
                if (v == 0 && b == 0) {
                    i = 0;
                    t = 0.0f;
                }
                if (v == n - 1 && b == 1) {
                    i = n - 2;
                    t = 1.0f;
                }
                i0[a] = i;
                tt[a] = t;
            }
            float d[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int cx = q & 1, cy = (q >> 1) & 1, cz = q >> 2;
                const float wq = (cx ? tt[0] : 1.f - tt[0]) * (cy ? tt[1] : 1.f - tt[1]) * (cz ? tt[2] : 1.f - tt[2]);
                const float *o = du[i0[2] + cz - (z0 - 1)][i0[1] + cy - (y0 - 1)][i0[0] + cx - (x0 - 1)];
                d[0] += wq * o[0];
                d[1] += wq * o[1];
                d[2] += wq * o[2];
            }
            const float ux = u0[h] + out_scale * d[0];
            const float uy = u1[h] + out_scale * d[1];
            const float uz = u2[h] + out_scale * d[2];
            fine[nc + c[h]] = ux;
            fine[2 * nc + c[h]] = uy;
            fine[3 * nc + c[h]] = uz;
            contrib[0] = rho[h] - 1.0f;
            contrib[1] = ux;
            contrib[2] = uy;
            contrib[3] = uz;
            fl = 1;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) part[k][vl][a] = contrib[a];
        isf[k][vl] = fl;
    }
    __syncthreads();
    if (t < NV) {
        float sum[4] = {0.f, 0.f, 0.f, 0.f};
        int fluid = 0;
        for (int kk = 0; kk < 8; ++kk) {
            if (!isf[kk][t]) continue;
            ++fluid;
#pragma unroll
            for (int a = 0; a < 4; ++a) sum[a] += part[kk][t][a];
        }
        const float inv = fluid > 0 ? in_scale / (float)fluid : 0.0f;
        __align__(16) bf16 o8[8];
        o8[0] = __float2bfloat16_rn(sum[0] * inv);
        o8[1] = __float2bfloat16_rn(fluid > 0 ? sum[1] * inv - uref.x * in_scale : 0.0f);
        o8[2] = __float2bfloat16_rn(fluid > 0 ? sum[2] * inv - uref.y * in_scale : 0.0f);
        o8[3] = __float2bfloat16_rn(fluid > 0 ? sum[3] * inv - uref.z * in_scale : 0.0f);
        o8[4] = __float2bfloat16_rn((8 - fluid) * 0.125f);
        o8[5] = __float2bfloat16_rn(uref.x * in_scale);
        o8[6] = __float2bfloat16_rn(uref.y * in_scale);
        o8[7] = __float2bfloat16_rn(uref.z * in_scale);
        const int64_t nv = (int64_t)n * n * n;
        const int vx = t % ADV_VX, vy = (t / ADV_VX) % ADV_VY, vz = t / (ADV_VX * ADV_VY);
        const int64_t cv = ((int64_t)(z0 + vz) * n + (y0 + vy)) * n + x0 + vx;
        reinterpret_cast<uint4 *>(feats)[cv] = *reinterpret_cast<const uint4 *>(o8);   // channels 0-7
        reinterpret_cast<uint4 *>(feats)[nv + cv] = make_uint4(0u, 0u, 0u, 0u);       // channels 8-15
    }
}

// f = f_eq(rho, u) of the fine state on fluid cells (shifted populations).
__global__ void k_surr_write_lattice(const float *__restrict__ fine, const uint8_t *__restrict__ solid,
                                     int64_t nc, float *__restrict__ f) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    if (solid && solid[c]) return;
    const float rho = fine[c], ux = fine[nc + c], uy = fine[2 * nc + c], uz = fine[3 * nc + c];
    const float uu = 1.5f * (ux * ux + uy * uy + uz * uz);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        const float cu = (float)kCX[i] * ux + (float)kCY[i] * uy + (float)kCZ[i] * uz;
        const float w = i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
        f[(size_t)i * nc + c] = w * ((rho - 1.0f) + rho * (3.0f * cu + 4.5f * cu * cu - uu));
    }
}

// Defect of the chained update: corr (+)= u(f) - u_fine on fluid cells, 0 on
// solid cells (u from the shifted lattice f of the plain LBM).
__global__ void k_surr_correction(const float *__restrict__ fine, const float *__restrict__ f,
                                  const uint8_t *__restrict__ solid, int64_t nc, int accumulate,
                                  float *__restrict__ corr) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    float d[3] = {0.f, 0.f, 0.f};
    if (!(solid && solid[c])) {
        float u[3] = {0.f, 0.f, 0.f}, rb = 1.0f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float b = f[(size_t)i * nc + c];
            rb += b;
            u[0] += kCX[i] * b;
            u[1] += kCY[i] * b;
            u[2] += kCZ[i] * b;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) d[k] = u[k] / rb - fine[(k + 1) * nc + c];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) corr[k * nc + c] = accumulate ? corr[k * nc + c] + d[k] : d[k];
}

// sums over fluid cells of |u_fine - u(f)|^2 and |u(f)|^2
__global__ void k_fine_vel_err(const float *__restrict__ fine, const float *__restrict__ f,
                               const uint8_t *__restrict__ solid, int64_t nc, double *__restrict__ out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, r = 0.0;
    if (c < nc && !(solid && solid[c])) {
        float u[3] = {0.f, 0.f, 0.f}, rb = 1.0f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float b = f[(size_t)i * nc + c];
            rb += b;
            u[0] += kCX[i] * b;
            u[1] += kCY[i] * b;
            u[2] += kCZ[i] * b;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double ub = u[k] / rb;
            const double d = fine[(k + 1) * nc + c] - ub;
            e += d * d;
            r += ub * ub;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, e);
        atomicAdd(out + 1, r);
    }
}

// sums over fluid cells of |u_a - u_b|^2 and |u_b|^2 (u from shifted lattices)
__global__ void k_vel_err(const float *__restrict__ fa, const float *__restrict__ fb,
                          const uint8_t *__restrict__ solid, int64_t nc, double *__restrict__ out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, r = 0.0;
    if (c < nc && !(solid && solid[c])) {
        float ua[3] = {0.f, 0.f, 0.f}, ub[3] = {0.f, 0.f, 0.f}, ra = 1.0f, rb = 1.0f;
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            const float a = fa[(size_t)i * nc + c], b = fb[(size_t)i * nc + c];
            ra += a;
            rb += b;
            ua[0] += kCX[i] * a;
            ua[1] += kCY[i] * a;
            ua[2] += kCZ[i] * a;
            ub[0] += kCX[i] * b;
            ub[1] += kCY[i] * b;
            ub[2] += kCZ[i] * b;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double da = ua[k] / ra - ub[k] / rb;
            e += da * da;
            r += (double)(ub[k] / rb) * (ub[k] / rb);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, e);
        atomicAdd(out + 1, r);
    }
}

// ----------------------------------------------------------- launching ----

// pdl: launch with programmatic dependent launch. The kernel copies its
// weights before its dependency wait, so this is off for the first layer of a
// forward pass right after the weights were rewritten.
template <int CIN, int COUT, int EPI>
static dw_status conv(SurrHandle *h, const CUtensorMap &tm_in, const bf16 *wt, const float *bias,
                      bf16 *oz, bf16 *oa, float *of, const bf16 *zprev, cudaStream_t s,
                      bool pdl = true, float *of4 = nullptr) {
    // The kernel allocates the whole tensor memory of its SM, so the shared
    // memory request is raised above half an SM's to keep one CTA per SM.
    constexpr size_t smem = tc_smem<CIN, COUT>() > 120 * 1024 ? tc_smem<CIN, COUT>() : 120 * 1024;
    static bool attr_set = false;
    if (!attr_set) {
        DW_CUDA(cudaFuncSetAttribute(k_conv3_tc<CIN, COUT, EPI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    const int grid = h->sms;  // one CTA per SM; each takes a contiguous range of output slices
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = pdl ? 1 : 0;
    DW_CUDA(cudaLaunchKernelEx(&cfg, k_conv3_tc<CIN, COUT, EPI>, tm_in, wt, bias, h->n, oz, oa, of,
                               zprev, of4, h->err));
    return DW_OK;
}

// TMA descriptor of a planar [C/8][n][n][n][8] BF16 volume viewed as 4D
// [C/8][z][y][x * 8]; box = bx voxels x by rows x bz slices in all C/8
// planes, zero fill outside.
static dw_status make_box_map(CUtensorMap *tm, const bf16 *base, int n, int C, int bx, int by,
                              int bz) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        DW_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                 cudaEnableDefault, &q));
        if (!fn || q != cudaDriverEntryPointSuccess) {
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            return DW_ERR_CUDA;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t nn = (cuuint64_t)n;
    const cuuint64_t dims[4] = {8 * nn, nn, nn, (cuuint64_t)(C / 8)};
    const cuuint64_t strides[3] = {16 * nn, 16 * nn * nn, 16 * nn * nn * nn};
    const cuuint32_t box[4] = {(cuuint32_t)(8 * bx), (cuuint32_t)by, (cuuint32_t)bz, (cuuint32_t)(C / 8)};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(base), dims,
                              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return DW_ERR_CUDA;
    }
    return DW_OK;
}

// The conv kernels' box: the 10 x 18 halo of one z slice.
static dw_status make_halo_map(CUtensorMap *tm, const bf16 *base, int n, int C) {
    return make_box_map(tm, base, n, C, TC_HX, TC_HY, 1);
}

// The weight-gradient kernel's boxes: an input tile's halo (16 voxels x 6
// rows x 3 slices) and an output-gradient tile (16 x 4 x 1).
static dw_status make_wgrad_maps(CUtensorMap *tm_in, CUtensorMap *tm_g, const bf16 *in, int cin,
                                 const bf16 *g, int cout, int n) {
    dw_status st = make_box_map(tm_in, in, n, cin, WG_TX, WG_HY, 3);
    if (st == DW_OK) st = make_box_map(tm_g, g, n, cout, WG_TX, WG_TY, 1);
    return st;
}

// Weight and bias gradients of one layer on tcgen05: gw += dW, gb += db.
template <int CIN, int COUT>
static dw_status wgrad_tc(SurrHandle *h, const CUtensorMap &tm_in, const CUtensorMap &tm_g,
                          const bf16 *g, float *gw, float *gb, cudaStream_t s) {
    constexpr size_t smem = wg_smem<CIN, COUT>();
    static bool attr_set = false;
    if (!attr_set) {
        DW_CUDA(cudaFuncSetAttribute(k_wgrad_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        attr_set = true;
    }
    const int ntiles = (h->n / WG_TX) * (h->n / WG_TY) * h->n;
    const int grid = std::min(std::min(h->sms, h->part_chunks), ntiles);
    k_wgrad_tc<CIN, COUT><<<grid, WG_THREADS, smem, s>>>(tm_in, tm_g, h->n, h->part, h->err);
    DW_LAUNCHED("k_wgrad_tc");
    k_bias_grad<COUT><<<grid, 256, 0, s>>>(g, h->nv, h->part_b);
    DW_LAUNCHED("k_bias_grad");
    const int64_t nw = 27LL * CIN * COUT;
    k_wgrad_reduce<<<grid_for(nw + COUT, 256), 256, 0, s>>>(h->part, h->part_b, grid, nw, COUT, gw, gb);
    DW_LAUNCHED("k_wgrad_reduce");
    return DW_OK;
}

// The same on the warp-level MMA (mma.sync): kept as a second implementation
// that surr_weight_grad exposes for comparison.
template <int CIN, int COUT>
static dw_status wgrad(SurrHandle *h, const bf16 *in, const bf16 *g, float *gw, float *gb,
                       cudaStream_t s) {
    constexpr size_t smem = wgrad_smem<CIN, COUT>();
    static bool attr_set = false;
    if (!attr_set) {
        DW_CUDA(cudaFuncSetAttribute(k_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        attr_set = true;
    }
    k_wgrad<CIN, COUT><<<dim3(h->nchunks, 3), CV_THREADS, smem, s>>>(in, g, h->n, h->tiles_per_chunk,
                                                                     h->part, h->part_b);
    DW_LAUNCHED("k_wgrad");
    const int64_t nw = 27LL * CIN * COUT;
    k_wgrad_reduce<<<grid_for(nw + COUT, 256), 256, 0, s>>>(h->part, h->part_b, h->nchunks, nw, COUT,
                                                            gw, gb);
    DW_LAUNCHED("k_wgrad_reduce");
    return DW_OK;
}

static dw_status refresh_weights(SurrHandle *h, cudaStream_t s) {
    h->weights_dirty = true;
    for (int l = 0; l < 4; ++l) {
        const int64_t cnt = 27LL * SCH[l] * SCH[l + 1];
        k_surr_weights<<<grid_for(cnt, 256), 256, 0, s>>>(h->params, h->wf, h->wd, h->off_w[l],
                                                          h->woff[l], SCH[l], SCH[l + 1]);
    }
    DW_LAUNCHED("k_surr_weights");
    return DW_OK;
}

}  // namespace dw

using namespace dw;

struct dw_surr_s : SurrHandle {};

static float3 uref_of(const SurrHandle *h) { return make_float3(h->uref[0], h->uref[1], h->uref[2]); }

extern "C" dw_status surr_set_inlet(dw_surr h, const float u[3]) {
    DW_REQUIRE(h && u, "handle and u must not be NULL");
    for (int a = 0; a < 3; ++a) {
        DW_REQUIRE(isfinite(u[a]), "u must be finite");
        h->uref[a] = u[a];
    }
    return DW_OK;
}

extern "C" dw_status surr_create(int32_t n, dw_surr *out) {
    DW_REQUIRE(out, "out must not be NULL");
    *out = nullptr;
    DW_REQUIRE(n >= 16 && n <= 256 && n % 16 == 0, "n=%d must be a multiple of 16 in [16, 256]", n);
    dw_surr h = new (std::nothrow) dw_surr_s();
    if (!h) {
        set_error("out of host memory");
        return DW_ERR_OOM;
    }
    h->n = n;
    h->nv = (int64_t)n * n * n;
    int64_t o = 0, wo = 0;
    for (int l = 0; l < 4; ++l) {
        h->off_w[l] = o;
        h->woff[l] = wo;
        o += 27LL * SCH[l] * SCH[l + 1];
        wo += 27LL * SCH[l] * SCH[l + 1];
        h->off_b[l] = o;
        o += SCH[l + 1];
    }
    h->nparams = o;
    const int ntiles = (n / CV_TX) * (n / CV_TY) * n;
    h->tiles_per_chunk = 16;
    h->nchunks = (ntiles + h->tiles_per_chunk - 1) / h->tiles_per_chunk;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    h->conv_ctas = 2 * (sms > 0 ? sms : 1);
    h->sms = sms > 0 ? sms : 1;
    const size_t nv = (size_t)h->nv, Nc = (size_t)8 * nv;
#define DW_ALLOC(ptr, bytes) \
    if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes))
    DW_ALLOC(h->params, sizeof(float) * o);
    DW_ALLOC(h->grads, sizeof(float) * o);
    DW_ALLOC(h->m, sizeof(float) * o);
    DW_ALLOC(h->v, sizeof(float) * o);
    DW_ALLOC(h->wf, sizeof(bf16) * wo);
    DW_ALLOC(h->wd, sizeof(bf16) * wo);
    DW_ALLOC(h->feats, sizeof(bf16) * nv * 16);
    for (int l = 0; l < 3; ++l) {
        DW_ALLOC(h->z[l], sizeof(bf16) * nv * 32);
        DW_ALLOC(h->a[l], sizeof(bf16) * nv * 32);
        DW_ALLOC(h->gz[l], sizeof(bf16) * nv * 32);
    }
    DW_ALLOC(h->out, sizeof(float) * nv * 16);
    DW_ALLOC(h->out4, sizeof(float) * nv * 4);
    DW_ALLOC(h->g4, sizeof(bf16) * nv * 16);
    h->part_chunks = std::max(h->nchunks, h->sms);
    DW_ALLOC(h->part, sizeof(float) * (size_t)h->part_chunks * 27 * 32 * 32);
    DW_ALLOC(h->part_b, sizeof(float) * (size_t)h->part_chunks * 32);
    DW_ALLOC(h->fine, sizeof(float) * 4 * Nc);
    DW_ALLOC(h->red, sizeof(double) * 4);
    DW_ALLOC(h->err, sizeof(int));
    DW_ALLOC(h->gbar, sizeof(unsigned) * 2);
#undef DW_ALLOC
    if (e == cudaSuccess) e = cudaMemset(h->params, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(h->grads, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(h->m, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(h->v, 0, sizeof(float) * o);
    if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->gbar, 0, sizeof(unsigned) * 2);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        dw_status st = cuda_fail(e, "surr_create");
        surr_destroy(h);
        return st;
    }
    dw_status st = make_halo_map(&h->tm_feats, h->feats, n, 16);
    for (int l = 0; l < 3 && st == DW_OK; ++l) st = make_halo_map(&h->tm_a[l], h->a[l], n, 32);
    if (st == DW_OK) st = make_halo_map(&h->tm_g4, h->g4, n, 16);
    for (int l = 0; l < 3 && st == DW_OK; ++l) st = make_halo_map(&h->tm_gz[l], h->gz[l], n, 32);
    if (st == DW_OK) st = make_wgrad_maps(&h->tmw_in[0], &h->tmw_g[0], h->feats, 16, h->gz[0], 32, n);
    for (int l = 1; l < 3 && st == DW_OK; ++l)
        st = make_wgrad_maps(&h->tmw_in[l], &h->tmw_g[l], h->a[l - 1], 32, h->gz[l], 32, n);
    if (st == DW_OK) st = make_wgrad_maps(&h->tmw_in[3], &h->tmw_g[3], h->a[2], 32, h->g4, 16, n);
    if (st != DW_OK) {
        surr_destroy(h);
        return st;
    }
    *out = h;
    return DW_OK;
}

extern "C" dw_status surr_destroy(dw_surr h) {
    if (!h) return DW_OK;
    cudaFree(h->params);
    cudaFree(h->grads);
    cudaFree(h->m);
    cudaFree(h->v);
    cudaFree(h->wf);
    cudaFree(h->wd);
    cudaFree(h->feats);
    for (int l = 0; l < 3; ++l) {
        cudaFree(h->z[l]);
        cudaFree(h->a[l]);
        cudaFree(h->gz[l]);
    }
    cudaFree(h->out);
    cudaFree(h->out4);
    cudaFree(h->g4);
    cudaFree(h->part);
    cudaFree(h->part_b);
    cudaFree(h->fine);
    cudaFree(h->corr);
    cudaFree(h->red);
    cudaFree(h->err);
    cudaFree(h->gbar);
    delete h;
    return DW_OK;
}

extern "C" dw_status surr_num_params(dw_surr h, int64_t *count) {
    DW_REQUIRE(h && count, "arguments must not be NULL");
    *count = h->nparams;
    return DW_OK;
}

extern "C" dw_status surr_set_params(dw_surr h, const float *src, dw_stream stream) {
    DW_REQUIRE(h && src, "arguments must not be NULL");
    cudaStream_t s = as_stream(stream);
    DW_CUDA(cudaMemcpyAsync(h->params, src, sizeof(float) * h->nparams, cudaMemcpyDeviceToDevice, s));
    return refresh_weights(h, s);
}

extern "C" dw_status surr_get_params(dw_surr h, float *dst, dw_stream stream) {
    DW_REQUIRE(h && dst, "arguments must not be NULL");
    DW_CUDA(cudaMemcpyAsync(dst, h->params, sizeof(float) * h->nparams, cudaMemcpyDeviceToDevice,
                            as_stream(stream)));
    return DW_OK;
}

extern "C" dw_status surr_get_grads(dw_surr h, float *dst, dw_stream stream) {
    DW_REQUIRE(h && dst, "arguments must not be NULL");
    DW_CUDA(cudaMemcpyAsync(dst, h->grads, sizeof(float) * h->nparams, cudaMemcpyDeviceToDevice,
                            as_stream(stream)));
    return DW_OK;
}

extern "C" dw_status surr_zero_grads(dw_surr h, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_CUDA(cudaMemsetAsync(h->grads, 0, sizeof(float) * h->nparams, as_stream(stream)));
    return DW_OK;
}

extern "C" dw_status surr_features(dw_surr h, const float *f, const uint8_t *solid,
                                   float in_scale, float *feats32, dw_stream stream) {
    DW_REQUIRE(h && f, "handle and f must not be NULL");
    cudaStream_t s = as_stream(stream);
    const int N = 2 * h->n;
    const int64_t nc = (int64_t)N * N * N;
    k_surr_fine<<<grid_for(nc, 256), 256, 0, s>>>(f, solid, N, h->fine);
    k_surr_coarse<<<grid_for(h->nv, 256), 256, 0, s>>>(h->fine, solid, h->n, in_scale,
                                                       uref_of(h), h->feats, feats32);
    DW_LAUNCHED("surr_features");
    return DW_OK;
}

extern "C" dw_status surr_set_features(dw_surr h, const float *feats, dw_stream stream) {
    DW_REQUIRE(h && feats, "handle and feats must not be NULL");
    k_cl16_to_planar<<<grid_for(h->nv * 2, 256), 256, 0, as_stream(stream)>>>(feats, h->feats, h->nv);
    DW_LAUNCHED("k_cl16_to_planar");
    return DW_OK;
}

extern "C" dw_status surr_get_features(dw_surr h, void *feats_bf16, dw_stream stream) {
    DW_REQUIRE(h && feats_bf16, "handle and feats must not be NULL");
    k_planar_to_cl16<<<grid_for(h->nv * 2, 256), 256, 0, as_stream(stream)>>>(
        h->feats, static_cast<bf16 *>(feats_bf16), h->nv);
    DW_LAUNCHED("k_planar_to_cl16");
    return DW_OK;
}

extern "C" dw_status surr_forward(dw_surr h, float *out, int32_t keep_activations,
                                  dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    cudaStream_t s = as_stream(stream);
    dw_status st;
    const float *P = h->params;
    if (keep_activations) {
        st = conv<16, 32, EPI_GELU>(h, h->tm_feats, h->wf + h->woff[0], P + h->off_b[0], h->z[0], h->a[0], nullptr, nullptr, s, !h->weights_dirty);
        if (st != DW_OK) return st;
        st = conv<32, 32, EPI_GELU>(h, h->tm_a[0], h->wf + h->woff[1], P + h->off_b[1], h->z[1], h->a[1], nullptr, nullptr, s);
        if (st != DW_OK) return st;
        st = conv<32, 32, EPI_GELU>(h, h->tm_a[1], h->wf + h->woff[2], P + h->off_b[2], h->z[2], h->a[2], nullptr, nullptr, s);
        if (st != DW_OK) return st;
    } else if (h->fused) {
        // the whole inference pass in one cooperative launch
        constexpr size_t smem = tc_forward_smem();
        if (!h->fused_attr_set) {
            DW_CUDA(cudaFuncSetAttribute(k_surr_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
            h->fused_attr_set = true;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)h->sms);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        // programmatic overlap with the previous kernel only while the weights
        // (copied before the dependency wait) are unchanged
        cfg.numAttrs = h->weights_dirty ? 1 : 2;
        cudaError_t e = cudaLaunchKernelEx(
            &cfg, k_surr_forward_tc, h->tm_feats, h->tm_a[0], h->tm_a[1], h->tm_a[2],
            (const bf16 *)(h->wf + h->woff[0]), (const bf16 *)(h->wf + h->woff[1]),
            (const bf16 *)(h->wf + h->woff[2]), (const bf16 *)(h->wf + h->woff[3]),
            (const float *)(P + h->off_b[0]), (const float *)(P + h->off_b[1]),
            (const float *)(P + h->off_b[2]), (const float *)(P + h->off_b[3]), h->a[0], h->a[1],
            h->a[2], h->out, h->out4, h->n, h->gbar, h->err);
        if (e == cudaSuccess) {
            h->weights_dirty = false;
            if (out)
                DW_CUDA(cudaMemcpyAsync(out, h->out, sizeof(float) * h->nv * 16,
                                        cudaMemcpyDeviceToDevice, s));
            return DW_OK;
        }
        // not launchable here (e.g. no cooperative launch): the per-layer kernels from now on
        cudaGetLastError();
        h->fused = false;
        return surr_forward(h, out, keep_activations, stream);
    } else {
        st = conv<16, 32, EPI_GELU_ONLY>(h, h->tm_feats, h->wf + h->woff[0], P + h->off_b[0], nullptr, h->a[0], nullptr, nullptr, s, !h->weights_dirty);
        if (st != DW_OK) return st;
        st = conv<32, 32, EPI_GELU_ONLY>(h, h->tm_a[0], h->wf + h->woff[1], P + h->off_b[1], nullptr, h->a[1], nullptr, nullptr, s);
        if (st != DW_OK) return st;
        st = conv<32, 32, EPI_GELU_ONLY>(h, h->tm_a[1], h->wf + h->woff[2], P + h->off_b[2], nullptr, h->a[2], nullptr, nullptr, s);
        if (st != DW_OK) return st;
    }
    st = conv<32, 16, EPI_F32>(h, h->tm_a[2], h->wf + h->woff[3], P + h->off_b[3], nullptr, nullptr, h->out, nullptr, s, true, h->out4);
    h->weights_dirty = false;
    if (st != DW_OK) return st;
    if (out)
        DW_CUDA(cudaMemcpyAsync(out, h->out, sizeof(float) * h->nv * 16, cudaMemcpyDeviceToDevice, s));
    return DW_OK;
}

extern "C" dw_status surr_device_status(dw_surr h, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    int bits = 0;
    cudaStream_t s = as_stream(stream);
    DW_CUDA(cudaMemcpyAsync(&bits, h->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DW_CUDA(cudaStreamSynchronize(s));
    DW_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int), s));
    DW_CUDA(cudaMemsetAsync(h->gbar, 0, sizeof(unsigned) * 2, s));  // a barrier that gave up
    DW_CUDA(cudaStreamSynchronize(s));
    return status_from_bits(bits);
}

extern "C" dw_status surr_loss(dw_surr h, const float *target, float *loss, dw_stream stream) {
    DW_REQUIRE(h && target, "handle and target must not be NULL");
    cudaStream_t s = as_stream(stream);
    int *cnt = reinterpret_cast<int *>(h->red);
    DW_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
    k_count_fluid<<<grid_for(h->nv, 256), 256, 0, s>>>(h->feats, h->nv, cnt);
    k_surr_loss<<<grid_for(h->nv, 256), 256, 0, s>>>(h->out, target, h->feats, h->nv, cnt, h->g4, loss);
    DW_LAUNCHED("k_surr_loss");
    return DW_OK;
}

extern "C" dw_status surr_set_output_grad(dw_surr h, const float *g_out, dw_stream stream) {
    DW_REQUIRE(h && g_out, "handle and g_out must not be NULL");
    k_cl16_to_planar<<<grid_for(h->nv * 2, 256), 256, 0, as_stream(stream)>>>(g_out, h->g4, h->nv);
    DW_LAUNCHED("k_cl16_to_planar");
    return DW_OK;
}

extern "C" dw_status surr_backward(dw_surr h, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    cudaStream_t s = as_stream(stream);
    dw_status st;
    // layer 4: dW from a3 and g4; dL/dz3 = (W4' * g4) GELU'(z3)
    st = wgrad_tc<32, 16>(h, h->tmw_in[3], h->tmw_g[3], h->g4, h->grads + h->off_w[3],
                          h->grads + h->off_b[3], s);
    if (st != DW_OK) return st;
    st = conv<16, 32, EPI_DGELU>(h, h->tm_g4, h->wd + h->woff[3], nullptr, h->gz[2], nullptr, nullptr, h->z[2], s);
    if (st != DW_OK) return st;
    st = wgrad_tc<32, 32>(h, h->tmw_in[2], h->tmw_g[2], h->gz[2], h->grads + h->off_w[2],
                          h->grads + h->off_b[2], s);
    if (st != DW_OK) return st;
    st = conv<32, 32, EPI_DGELU>(h, h->tm_gz[2], h->wd + h->woff[2], nullptr, h->gz[1], nullptr, nullptr, h->z[1], s);
    if (st != DW_OK) return st;
    st = wgrad_tc<32, 32>(h, h->tmw_in[1], h->tmw_g[1], h->gz[1], h->grads + h->off_w[1],
                          h->grads + h->off_b[1], s);
    if (st != DW_OK) return st;
    st = conv<32, 32, EPI_DGELU>(h, h->tm_gz[1], h->wd + h->woff[1], nullptr, h->gz[0], nullptr, nullptr, h->z[0], s);
    if (st != DW_OK) return st;
    st = wgrad_tc<16, 32>(h, h->tmw_in[0], h->tmw_g[0], h->gz[0], h->grads + h->off_w[0],
                          h->grads + h->off_b[0], s);
    return st;
}

extern "C" dw_status surr_weight_grad(dw_surr h, int32_t cin, int32_t cout, const void *in,
                                      const void *g, float *gw, float *gb, int32_t impl,
                                      dw_stream stream) {
    DW_REQUIRE(h && in && g && gw && gb, "handle and arrays must not be NULL");
    DW_REQUIRE((cin == 16 && cout == 32) || (cin == 32 && cout == 32) || (cin == 32 && cout == 16),
               "(cin, cout) = (%d, %d) is not a layer shape of the network", cin, cout);
    DW_REQUIRE(impl == 0 || impl == 1, "impl must be 0 (tcgen05) or 1 (mma.sync)");
    cudaStream_t s = as_stream(stream);
    const bf16 *bi = static_cast<const bf16 *>(in), *bg = static_cast<const bf16 *>(g);
    if (impl == 1) {
        if (cin == 16) return wgrad<16, 32>(h, bi, bg, gw, gb, s);
        if (cout == 32) return wgrad<32, 32>(h, bi, bg, gw, gb, s);
        return wgrad<32, 16>(h, bi, bg, gw, gb, s);
    }
    CUtensorMap tm_in, tm_g;
    dw_status st = make_wgrad_maps(&tm_in, &tm_g, bi, cin, bg, cout, h->n);
    if (st != DW_OK) return st;
    if (cin == 16) return wgrad_tc<16, 32>(h, tm_in, tm_g, bg, gw, gb, s);
    if (cout == 32) return wgrad_tc<32, 32>(h, tm_in, tm_g, bg, gw, gb, s);
    return wgrad_tc<32, 16>(h, tm_in, tm_g, bg, gw, gb, s);
}

extern "C" dw_status surr_adam(dw_surr h, float lr, float beta1, float beta2, float eps,
                               int32_t step, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(step >= 1, "step counts from 1");
    cudaStream_t s = as_stream(stream);
    const float c1 = 1.0f / (1.0f - powf(beta1, (float)step));
    const float c2 = 1.0f / (1.0f - powf(beta2, (float)step));
    k_surr_adam<<<grid_for(h->nparams, 256), 256, 0, s>>>(h->params, h->grads, h->m, h->v, h->nparams,
                                                          lr, beta1, beta2, eps, c1, c2);
    DW_LAUNCHED("k_surr_adam");
    return refresh_weights(h, s);
}

extern "C" dw_status surr_apply(dw_surr h, const float *out, float out_scale,
                                const uint8_t *solid, float *f, dw_stream stream) {
    DW_REQUIRE(h && f, "handle and f must not be NULL");
    const int N = 2 * h->n;
    const int64_t nc = (int64_t)N * N * N;
    k_surr_apply<<<grid_for(nc, 256), 256, 0, as_stream(stream)>>>(out ? out : h->out, out_scale,
                                                                   h->fine, solid, h->n, f);
    DW_LAUNCHED("k_surr_apply");
    return DW_OK;
}

extern "C" dw_status lbm_velocity_error(const float *fa, const float *fb, const uint8_t *solid,
                                        int64_t ncell, double *sums, dw_stream stream) {
    DW_REQUIRE(fa && fb && sums, "fa, fb and sums must not be NULL");
    DW_REQUIRE(ncell > 0, "ncell must be > 0");
    k_vel_err<<<grid_for(ncell, 256), 256, 0, as_stream(stream)>>>(fa, fb, solid, ncell, sums);
    DW_LAUNCHED("k_vel_err");
    return DW_OK;
}

extern "C" dw_status surr_features_fine(dw_surr h, const uint8_t *solid, float in_scale,
                                        dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    k_surr_coarse<<<grid_for(h->nv, 256), 256, 0, as_stream(stream)>>>(h->fine, solid, h->n, in_scale, uref_of(h),
                                                                       h->feats, nullptr);
    DW_LAUNCHED("k_surr_coarse");
    return DW_OK;
}

extern "C" dw_status surr_advance_fine(dw_surr h, float out_scale, const uint8_t *solid,
                                       float in_scale, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_CUDA(launch_pdl(k_surr_advance_fine, (unsigned)(h->nv / (ADV_VX * ADV_VY * ADV_VZ)),
                       ADV_THREADS, as_stream(stream), (const float *)h->out4, out_scale, h->fine,
                       solid, h->n, in_scale, uref_of(h), h->feats,
                       (const float *)(h->corr_on ? h->corr : nullptr)));
    return DW_OK;
}

extern "C" dw_status surr_write_lattice(dw_surr h, const uint8_t *solid, float *f, dw_stream stream) {
    DW_REQUIRE(h && f, "handle and f must not be NULL");
    const int N = 2 * h->n;
    const int64_t nc = (int64_t)N * N * N;
    k_surr_write_lattice<<<grid_for(nc, 256), 256, 0, as_stream(stream)>>>(h->fine, solid, nc, f);
    DW_LAUNCHED("k_surr_write_lattice");
    return DW_OK;
}

extern "C" dw_status surr_set_correction(dw_surr h, const float *f, const uint8_t *solid,
                                        int32_t mode, dw_stream stream) {
    DW_REQUIRE(h, "handle is NULL");
    DW_REQUIRE(mode >= 0 && mode <= 2, "mode=%d must be 0, 1 or 2", mode);
    if (mode == 0) {
        h->corr_on = false;
        return DW_OK;
    }
    DW_REQUIRE(f, "f must not be NULL");
    DW_REQUIRE(mode == 1 || h->corr_on, "mode 2 accumulates into a correction that is not set");
    const int N = 2 * h->n;
    const int64_t nc = (int64_t)N * N * N;
    if (!h->corr) DW_CUDA(cudaMalloc((void **)&h->corr, sizeof(float) * 3 * (size_t)nc));
    k_surr_correction<<<grid_for(nc, 256), 256, 0, as_stream(stream)>>>(h->fine, f, solid, nc,
                                                                        mode == 2 ? 1 : 0, h->corr);
    DW_LAUNCHED("k_surr_correction");
    h->corr_on = true;
    return DW_OK;
}

extern "C" dw_status surr_fine_velocity_error(dw_surr h, const float *f, const uint8_t *solid,
                                              double *sums, dw_stream stream) {
    DW_REQUIRE(h && f && sums, "arguments must not be NULL");
    const int N = 2 * h->n;
    const int64_t nc = (int64_t)N * N * N;
    k_fine_vel_err<<<grid_for(nc, 256), 256, 0, as_stream(stream)>>>(h->fine, f, solid, nc, sums);
    DW_LAUNCHED("k_fine_vel_err");
    return DW_OK;
}

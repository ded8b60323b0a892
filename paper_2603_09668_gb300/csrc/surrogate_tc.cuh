// 3x3x3 convolutions of the surrogate network on the fifth-generation tensor
// cores: tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator in tensor
// memory), operands in shared memory filled by TMA, one MMA-issuing thread
// per CTA.
//
// Activations are stored planar, [C/8][n^3][8] BF16: plane c holds channels
// 8c..8c+7 of every voxel (16 B per voxel, voxels x fastest), so that a row of
// a tile's halo is one contiguous run of 16-byte voxel records.
//
// The convolution out[v][co] = sum_{tap, ci} W[tap][co][ci] in[v + d(tap)][ci]
// (zero padding) is an implicit GEMM over output tiles of 8 (x) x 16 (y)
// voxels (M = 128 rows). A CTA streams along z through the input slices of
// its output range; for each slice the 10 x 18 halo of all 8-channel planes
// is loaded by one TMA box ({80, 18, 1, C/8} of the 4D view
// [C/8][z][y][x * 8], zero fill outside the volume), so that each plane lands
// as 16-byte voxel rows ordered (y, x). In that layout the A operand of every
// (dx, dy) tap is a plain shared-memory matrix descriptor without swizzling:
// the 8 x-voxels of one tile row form a core matrix (8 rows x 16 B,
// contiguous), tile rows are 10 voxels (160 B) apart (stride-dimension
// offset), and the next 8 channels are one plane further (leading-dimension
// offset); shifting the descriptor's start selects the tap. The B operand
// holds the weights of the three dz taps of that (dx, dy) together, so one
// MMA has N = 3 COUT and delivers the slice's contributions to three output
// slices at once (a 128 x 32 x 16 MMA costs nearly as much as 128 x 96 x 16).
#pragma once


#include <cuda.h>

#include "surrogate_conv.cuh"

namespace dw {

constexpr int TC_TX = 8, TC_TY = 16;                 // output tile (x, y), z = 1
constexpr int TC_HX = TC_TX + 2, TC_HY = TC_TY + 2;  // halo 10 x 18 x 3

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // shared-memory matrix descriptor: start, leading and stride byte offsets
    // (all >> 4), descriptor version 1 (bit 46), no swizzle, base offset 0
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity of an mbarrier; false after about
// a second, or as soon as *abort (if given) is set.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity,
                                        const volatile int *abort) {
    uint64_t t0 = 0;
    for (unsigned it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 0) {
            if (abort && *abort) return false;
            const uint64_t t = globaltimer_ns();
            if (it == 0) t0 = t;
            else if (t - t0 > 1000000000ull) return false;
        }
    }
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// tcgen05.ld of N consecutive 32-bit accumulator columns of this warp's 32
// lanes (one row per thread).
template <int N>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&r)[N]);

template <>
__device__ __forceinline__ void tc_ld<16>(uint32_t taddr, float (&r)[16]) {
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
          "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
          "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}

template <>
__device__ __forceinline__ void tc_ld<4>(uint32_t taddr, float (&r)[4]) {
    uint32_t u[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) r[i] = __uint_as_float(u[i]);
}

template <>
__device__ __forceinline__ void tc_ld<8>(uint32_t taddr, float (&r)[8]) {
    uint32_t u[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]),
                   "=r"(u[6]), "=r"(u[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}

constexpr int TC_NST = 8;        // halo stages (one input slice each)
constexpr int TC_LAG = 3;        // a stage is refilled once the MMAs of slice k - TC_LAG are done
constexpr int TC_EPI_WARPS = 8;  // epilogue warps: lane quarter = warp & 3, column half = warp >> 2
constexpr int TC_THREADS = 32 * (TC_EPI_WARPS + 1);  // + one producer / MMA warp
constexpr int TC_TMEM_COLS = 512;                     // the whole tensor memory of the SM
constexpr int TC_NWIN = 5;       // accumulator windows (one input slice each)
constexpr int TC_RING = 8;       // slice-ready barrier ring (>= TC_NWIN + 2)
constexpr int TC_SLICE_BYTES = TC_HX * TC_HY * 16;    // 2880 B: one plane of a 10 x 18 slice halo
constexpr int TC_SLICE = TC_SLICE_BYTES;              // plane stride: a slice's planes arrive as one box

template <int CIN, int COUT>
constexpr size_t tc_smem() {
    return (size_t)TC_NST * (CIN / 8) * TC_SLICE + (size_t)27 * (CIN / 8) * COUT * 16 + 1024;
}

// TMA load of the halo of input slice z of the xy tile at (x0, y0): one box
// {80 (10 voxels x 8 channels), 18, 1, CIN/8} of the 4D view
// [C/8][z][y][x * 8] that lands as CIN/8 planes of 18 rows x 160 B, one
// after the other (a single copy per slice instead of one per plane; the x
// coordinate 8 (x0 - 1) elements is 16-byte aligned, the zero fill covers the
// volume's faces).
template <int CIN>
__device__ __forceinline__ void tc_load_slice(const CUtensorMap *tm, uint32_t halo, uint32_t bar,
                                              int x0, int y0, int z) {
    constexpr int KCH = CIN / 8;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(KCH * TC_SLICE_BYTES) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];"
        :: "r"(halo), "l"((uint64_t)tm), "r"(8 * (x0 - 1)), "r"(y0 - 1), "r"(z), "r"(0), "r"(bar)
        : "memory");
}

// The CTA's output work as segments: output slices o0..o1 of one xy tile.
struct TcSeg {
    int xy, o0, o1;
};

// Segment j of the CTA's contiguous range of (xy tile, z) output units;
// false past the end. Segments stop at xy boundaries.
__device__ __forceinline__ bool tc_segment(int n, int nxy, int j, TcSeg &c) {
    const int total = nxy * n;  // < 2^31: n <= 256
    const int u0 = (int)((int64_t)total * blockIdx.x / gridDim.x);
    const int u1 = (int)((int64_t)total * (blockIdx.x + 1) / gridDim.x);
    int u = u0;
    for (int i = 0;; ++i) {
        if (u >= u1) return false;
        const int xy = u / n, z = u % n;
        const int cnt = min(u1 - u, n - z);
        if (i == j) {
            c.xy = xy;
            c.o0 = z;
            c.o1 = z + cnt - 1;
            return true;
        }
        u += cnt;
    }
}

// Epilogues: EPI_GELU (z and GELU(z) in BF16), EPI_GELU_ONLY (GELU(z)),
// EPI_F32 (z in FP32), EPI_DGELU (acc * GELU'(zprev), BF16). Weights are
// stored as [9 (dy, dx)][CIN/8][3 (dz)][COUT][8].
//
// z-streaming: the CTA walks the input z-slices of each segment once (slices
// o0 - 1 .. o1 + 1, clipped to the volume). For each input slice and each of
// its 9 (dx, dy) taps it issues MMAs with N = 3 COUT, the three dz taps at
// once, into a fresh accumulator window of its own (a ring of TC_NWIN windows
// of 3 COUT columns): block b of slice zi's window holds its contribution to
// output slice zi + 1 - b. Output slice z is the sum of block 0 of slice
// z - 1, block 1 of slice z and block 2 of slice z + 1 (missing slices
// outside the volume contribute nothing), so it is finished once slice z + 1
// is (slice n - 1 also finishes output n - 1), and the epilogue adds the
// three blocks. Windows never overlap, so the MMAs of consecutive slices do
// not wait on each other's accumulators.
//
// Roles: warp 8, lane 0 issues the weight copies, the halo loads (ring of
// TC_NST slices) and the MMAs, committing each slice to ready[k % TC_RING];
// warps 0-7 read the finished output slices (warp w: accumulator lanes
// 32 (w % 4) .. + 31, column half w / 4) and arrive on wfree[w] once no
// output needs window w any more, which the producer waits for before
// reusing it.

// The pipeline's shared-memory state, kept across the layers of one launch:
// the slice counter k runs on from layer to layer, so every mbarrier phase
// and window index stays consistent without re-initialisation.
struct TcPipe {
    uint64_t full[TC_NST], empty[TC_NST], ready[TC_RING], wfree[TC_NWIN];
    uint64_t wbar[2];  // weight buffers
    uint32_t wbuf[2];  // their shared-memory addresses
    int wcount[2];     // copies issued into each buffer (producer thread only)
    uint32_t tmem_base;
    int abort_flag;
};

constexpr int tc_wbytes(int cin, int cout) { return 27 * (cin / 8) * cout * 16; }
constexpr int TC_WMAX = tc_wbytes(32, 32);  // largest layer's weights

// Output buffers and bias of one layer. out_f4 (EPI_F32, may be NULL) also
// receives channels 0-3 of each voxel as one float4, the compact copy the
// chained update reads.
struct TcOut {
    const float *bias;
    bf16 *out_z, *out_a;
    float *out_f;
    const bf16 *zprev;
    float *out_f4;
};

// What the producer does before the layer's first halo load.
enum { TC_PRO_NONE = 0, TC_PRO_PDL = 1, TC_PRO_PROXY = 2 };

// Barrier init and the TMEM allocation (all threads).
__device__ __forceinline__ uint32_t tc_pipe_open(TcPipe &pp) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        pp.abort_flag = 0;
        for (int i = 0; i < TC_NST; ++i) {
            mbar_init(smem_u32(&pp.full[i]), 1);
            mbar_init(smem_u32(&pp.empty[i]), 1);
        }
        for (int i = 0; i < TC_RING; ++i) mbar_init(smem_u32(&pp.ready[i]), 1);
        for (int i = 0; i < TC_NWIN; ++i) mbar_init(smem_u32(&pp.wfree[i]), TC_EPI_WARPS);
        mbar_init(smem_u32(&pp.wbar[0]), 1);
        mbar_init(smem_u32(&pp.wbar[1]), 1);
        pp.wcount[0] = pp.wcount[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((tid >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&pp.tmem_base)), "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return pp.tmem_base;
}

// All threads: the TMEM release at the end; before it the producer waits
// (bounded) for the last weight copy into each buffer, which an abort may
// have left in flight.
__device__ __forceinline__ void tc_pipe_close(TcPipe &pp, uint32_t taddr) {
    if (threadIdx.x == 32 * TC_EPI_WARPS)
        for (int b = 0; b < 2; ++b)
            if (pp.wcount[b] > 0) tc_wait(smem_u32(&pp.wbar[b]), (pp.wcount[b] - 1) & 1, nullptr);
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(taddr), "r"(TC_TMEM_COLS));
    }
}

// One bulk copy of a layer's weights into weight buffer b (producer thread).
__device__ __forceinline__ void tc_copy_weights(TcPipe &pp, int b, const bf16 *wt, uint32_t bytes) {
    const uint32_t bar = smem_u32(&pp.wbar[b]);
    ++pp.wcount[b];
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(pp.wbuf[b]), "l"(wt), "r"(bytes), "r"(bar) : "memory");
}

// Input slices of this CTA in one layer (the same for every layer).
__device__ __forceinline__ int tc_slices(int n, int nxy) {
    int cnt = 0;
    TcSeg c;
    for (int j = 0; tc_segment(n, nxy, j, c); ++j)
        cnt += min(c.o1 + 1, n - 1) - max(c.o0 - 1, 0) + 1;
    return cnt;
}

// One layer over the CTA's output range, called by all threads. Weight
// buffer wb holds (or receives) this layer's weights: own_wt, when not NULL,
// is copied there first by the producer. next_wt, when not NULL, is copied
// into the other buffer at the start, the prefetch of the following layer's
// weights (that buffer's previous layer has finished). k0 counts the slices
// this CTA has gone through in earlier layers of the launch. fence_out: the
// epilogue ends with a proxy fence, so that TMA reads of the output by other
// CTAs after a grid barrier see it.
template <int CIN, int COUT, int EPI>
__device__ __forceinline__ void tc_layer(TcPipe &pp, uint32_t taddr, const CUtensorMap *tm_in,
                                         const TcOut &o, int n, uint32_t hbase, int wb,
                                         const bf16 *own_wt, const bf16 *next_wt,
                                         uint32_t next_bytes, int k0, int prologue,
                                         bool fence_out, int *err) {
    static_assert(CIN % 16 == 0 && (COUT == 16 || COUT == 32), "unsupported shape");
    constexpr int KCH = CIN / 8;
    constexpr int HBYTES = KCH * TC_SLICE;
    constexpr int WBYTES = tc_wbytes(CIN, COUT);
    constexpr int CPW = COUT / (TC_EPI_WARPS / 4);  // accumulator columns per epilogue warp
    constexpr int NW = 3 * COUT;                    // MMA N: the three dz taps
    static_assert(TC_NWIN * NW <= TC_TMEM_COLS && TC_RING >= TC_NWIN + 2, "tensor memory plan");
    constexpr uint32_t IDESC = tc_idesc(NW);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const volatile int *abort_p = &pp.abort_flag;
    const int tiles_x = n / TC_TX, nxy = tiles_x * (n / TC_TY);
    if (pp.abort_flag) return;  // an earlier layer gave up

    if (warp == TC_EPI_WARPS) {
        if (lane == 0) {
            int issued = k0, consumed = k0;  // slices
            bool ok = true;
            // the slices of all segments in order, for the halo prefetch
            int pf_seg = 0, pf_z = 0;
            TcSeg pfc;
            bool pf_more = tc_segment(n, nxy, 0, pfc);
            if (pf_more) pf_z = max(pfc.o0 - 1, 0);
            auto prefetch = [&]() {
                if (!pf_more) return;
                const int s = issued % TC_NST;
                tc_load_slice<CIN>(tm_in, hbase + s * HBYTES, smem_u32(&pp.full[s]),
                                   (pfc.xy % tiles_x) * TC_TX, (pfc.xy / tiles_x) * TC_TY, pf_z);
                ++issued;
                if (pf_z < min(pfc.o1 + 1, n - 1)) {
                    ++pf_z;
                } else {
                    pf_more = tc_segment(n, nxy, ++pf_seg, pfc);
                    if (pf_more) pf_z = max(pfc.o0 - 1, 0);
                }
            };
            if (own_wt) tc_copy_weights(pp, wb, own_wt, WBYTES);
            if (next_wt) tc_copy_weights(pp, 1 - wb, next_wt, next_bytes);
            const uint32_t wbase = pp.wbuf[wb];
            if (prologue == TC_PRO_PDL) pdl_wait();
            if (prologue == TC_PRO_PROXY) asm volatile("fence.proxy.async.global;" ::: "memory");
            while (issued - k0 < TC_NST && pf_more) prefetch();
            ok = tc_wait(smem_u32(&pp.wbar[wb]), (pp.wcount[wb] - 1) & 1, abort_p);
            const uint64_t b0 = tc_desc(wbase, NW * 16, 128);
            TcSeg c;
            for (int j = 0; ok && tc_segment(n, nxy, j, c); ++j) {
                const int i0 = max(c.o0 - 1, 0), i1 = min(c.o1 + 1, n - 1);
                for (int zi = i0; zi <= i1; ++zi) {
                    const int k = consumed, s = k % TC_NST, w = k % TC_NWIN;
                    ok = tc_wait(smem_u32(&pp.full[s]), (k / TC_NST) & 1, abort_p) &&
                         tc_wait(smem_u32(&pp.wfree[w]), ((k / TC_NWIN) & 1) ^ 1, abort_p);
                    if (!ok) break;
                    ++consumed;
                    tc_fence_after();
                    const uint32_t d = taddr + (uint32_t)(w * NW);
                    const uint64_t a0 = tc_desc(hbase + s * HBYTES, TC_SLICE, TC_HX * 16);
#pragma unroll
                    for (int t = 0; t < 9; ++t) {
                        const int dx = t % 3, dy = t / 3;  // offsets + 1
#pragma unroll
                        for (int kk = 0; kk < KCH / 2; ++kk) {
                            const uint32_t a_off = (dy * TC_HX + dx) * 16 + 2 * kk * TC_SLICE;
                            const uint32_t b_off = ((t * KCH + 2 * kk) * NW) * 16;
                            const uint64_t ad = a0 + (a_off >> 4);
                            const uint64_t bd = b0 + (b_off >> 4);
                            const uint32_t acc = (t | kk) != 0;  // a fresh window per slice
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                :: "r"(d), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                                : "memory");
                        }
                    }
                    tc_commit(smem_u32(&pp.empty[s]));
                    tc_commit(smem_u32(&pp.ready[k % TC_RING]));
                    // refill the stage of slice k - TC_LAG once its MMAs are done
                    if (k - k0 >= TC_LAG && pf_more) {
                        const int k1 = k - TC_LAG;
                        ok = tc_wait(smem_u32(&pp.empty[k1 % TC_NST]), (k1 / TC_NST) & 1, abort_p);
                        if (!ok) break;
                        prefetch();
                    }
                }
            }
            if (!ok) {
                if (!pp.abort_flag) atomicOr(err, ERRBIT_TIMEOUT);
                pp.abort_flag = 1;
            }
            // drain (bounded): halo loads still in flight, the last MMA batch
            for (int k = consumed; k < issued; ++k)
                tc_wait(smem_u32(&pp.full[k % TC_NST]), (k / TC_NST) & 1, nullptr);
            if (consumed > k0)
                tc_wait(smem_u32(&pp.empty[(consumed - 1) % TC_NST]), ((consumed - 1) / TC_NST) & 1, nullptr);
        }
        __syncwarp();
    } else {
        const int q = warp & 3, hcol = warp >> 2;
        const int row = q * 32 + lane;  // accumulator lane = tile voxel (x = row & 7, y = row >> 3)
        const uint32_t tq = taddr + ((uint32_t)(q * 32) << 16) + hcol * CPW;
        const size_t nv = (size_t)n * n * n;
        int k = k0;  // slices seen in this launch
        bool ok = true;
        TcSeg c;
        for (int j = 0; ok && tc_segment(n, nxy, j, c); ++j) {
            const int i0 = max(c.o0 - 1, 0), i1 = min(c.o1 + 1, n - 1);
            const int kb = k;  // global index of slice i0
            const int x0 = (c.xy % tiles_x) * TC_TX, y0 = (c.xy / tiles_x) * TC_TY;
            for (int zi = i0; zi <= i1; ++zi, ++k) {
                int okw = 1;
                if (lane == 0) {
                    okw = tc_wait(smem_u32(&pp.ready[k % TC_RING]), (k / TC_RING) & 1, abort_p);
                    if (!okw) {
                        if (!pp.abort_flag) atomicOr(err, ERRBIT_TIMEOUT);
                        pp.abort_flag = 1;
                    }
                }
                if (!__shfl_sync(0xffffffffu, okw, 0)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // outputs finished by slice zi: zi - 1, and zi itself at the volume's end
                const int zlo = max(zi - 1, c.o0), zhi = (zi == n - 1) ? min(zi, c.o1) : min(zi - 1, c.o1);
                float r[2][CPW];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const int z = zlo + m;
                    if (z > zhi) break;
#pragma unroll
                    for (int cc = 0; cc < CPW; ++cc) r[m][cc] = 0.0f;
#pragma unroll
                    for (int b = 0; b < 3; ++b) {  // block b of slice z - 1 + b
                        const int zs = z - 1 + b;
                        if (zs < i0 || zs > i1) continue;
                        const int ks = kb + (zs - i0);
                        float part[CPW];
                        tc_ld<CPW>(tq + (uint32_t)((ks % TC_NWIN) * NW + b * COUT), part);
#pragma unroll
                        for (int cc = 0; cc < CPW; ++cc) r[m][cc] += part[cc];
                    }
                }
                tc_fence_before();
                __syncwarp();
                // windows no longer needed: slice zi - 2 (its last output, zi - 1, is
                // done), and at the segment's end the last two slices as well
                if (lane == 0) {
                    if (zi - 2 >= i0) mbar_arrive(smem_u32(&pp.wfree[(k - 2) % TC_NWIN]));
                    if (zi == i1) {
                        if (zi - 1 >= i0) mbar_arrive(smem_u32(&pp.wfree[(k - 1) % TC_NWIN]));
                        mbar_arrive(smem_u32(&pp.wfree[k % TC_NWIN]));
                    }
                }
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    if (zlo + m > zhi) break;
                    const int z = zlo + m;
                    const size_t v = ((size_t)z * n + (y0 + (row >> 3))) * n + x0 + (row & 7);
                    const int c0 = hcol * CPW;
                    auto plane = [&](int cc) { return ((size_t)((c0 + cc) >> 3) * nv + v) * 8; };
                    if (EPI == EPI_F32) {
#pragma unroll
                        for (int cc = 0; cc < CPW; cc += 4) {
                            const float4 q4 =
                                make_float4(r[m][cc] + o.bias[c0 + cc], r[m][cc + 1] + o.bias[c0 + cc + 1],
                                            r[m][cc + 2] + o.bias[c0 + cc + 2], r[m][cc + 3] + o.bias[c0 + cc + 3]);
                            *reinterpret_cast<float4 *>(o.out_f + v * COUT + c0 + cc) = q4;
                            if (cc == 0 && c0 == 0 && o.out_f4) reinterpret_cast<float4 *>(o.out_f4)[v] = q4;
                        }
                    } else if (EPI == EPI_DGELU) {
#pragma unroll
                        for (int cc = 0; cc < CPW; cc += 8) {
                            const uint4 zp = *reinterpret_cast<const uint4 *>(o.zprev + plane(cc));
                            const bf16 *zb = reinterpret_cast<const bf16 *>(&zp);
                            __align__(16) bf16 od[8];
#pragma unroll
                            for (int jj = 0; jj < 8; ++jj)
                                od[jj] = __float2bfloat16_rn(r[m][cc + jj] * gelu_grad_f(__bfloat162float(zb[jj])));
                            *reinterpret_cast<uint4 *>(o.out_z + plane(cc)) = *reinterpret_cast<const uint4 *>(od);
                        }
                    } else {
#pragma unroll
                        for (int cc = 0; cc < CPW; cc += 8) {
                            __align__(16) bf16 oz[8], oa[8];
#pragma unroll
                            for (int jj = 0; jj < 8; ++jj) {
                                const float zz = r[m][cc + jj] + o.bias[c0 + cc + jj];
                                oz[jj] = __float2bfloat16_rn(zz);
                                oa[jj] = __float2bfloat16_rn(gelu_f(zz));
                            }
                            if (EPI == EPI_GELU)
                                *reinterpret_cast<uint4 *>(o.out_z + plane(cc)) = *reinterpret_cast<const uint4 *>(oz);
                            *reinterpret_cast<uint4 *>(o.out_a + plane(cc)) = *reinterpret_cast<const uint4 *>(oa);
                        }
                    }
                }
            }
        }
        if (fence_out) asm volatile("fence.proxy.async.global;" ::: "memory");
    }
}

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(TC_THREADS, 1) k_conv3_tc(
    const __grid_constant__ CUtensorMap tm_in, const bf16 *__restrict__ wt,
    const float *__restrict__ bias, int n, bf16 *__restrict__ out_z, bf16 *__restrict__ out_a,
    float *__restrict__ out_f, const bf16 *__restrict__ zprev, float *__restrict__ out_f4,
    int *err) {
    constexpr int HBYTES = (CIN / 8) * TC_SLICE;
    extern __shared__ unsigned char smem_raw[];
    __shared__ TcPipe pp;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t hbase = smem_u32(smem);
    if (threadIdx.x == 0) pp.wbuf[0] = pp.wbuf[1] = hbase + TC_NST * HBYTES;
    const uint32_t taddr = tc_pipe_open(pp);
    // Programmatic dependent launch: the next layer may be scheduled now; this
    // grid's input (the previous layer's output) is read only after
    // griddepcontrol.wait, the weights (written before the first layer) before.
    pdl_trigger();
    const TcOut o = {bias, out_z, out_a, out_f, zprev, out_f4};
    tc_layer<CIN, COUT, EPI>(pp, taddr, &tm_in, o, n, hbase, 0, wt, nullptr, 0, 0, TC_PRO_PDL,
                             false, err);
    tc_pipe_close(pp, taddr);
}

// Grid-wide barrier of a cooperative launch for `expected` CTAs (bar[0]
// arrivals, bar[1] generation). Bounded: after about a second the CTA sets
// ERRBIT_TIMEOUT and the abort flag and leaves; every later layer of the
// launch then does nothing.
__device__ __forceinline__ void tc_grid_sync(unsigned *bar, int *err, TcPipe &pp) {
    __syncthreads();
    if (threadIdx.x == 0 && !pp.abort_flag) {
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            for (unsigned it = 0; *gen == g0; ++it) {
                if ((it & 1023u) == 0 && globaltimer_ns() - t0 > 1000000000ull) {
                    atomicOr(err, ERRBIT_TIMEOUT);
                    pp.abort_flag = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

constexpr size_t tc_forward_smem() {
    return (size_t)TC_NST * 4 * TC_SLICE + 2 * (size_t)TC_WMAX + 1024;
}

// The inference forward pass of the surrogate network in one cooperative
// launch (one CTA per SM): layers 16 -> 32 -> 32 -> 32 (GELU) -> 16 (FP32),
// a grid barrier between layers (each layer reads the previous one's output
// around its own tiles), the TMEM allocation and the mbarriers kept across
// layers, and the weights of layer l + 1 copied into the second weight
// buffer while layer l runs.
__global__ void __launch_bounds__(TC_THREADS, 1) k_surr_forward_tc(
    const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1,
    const __grid_constant__ CUtensorMap tm2, const __grid_constant__ CUtensorMap tm3,
    const bf16 *__restrict__ w0, const bf16 *__restrict__ w1, const bf16 *__restrict__ w2,
    const bf16 *__restrict__ w3, const float *__restrict__ b0, const float *__restrict__ b1,
    const float *__restrict__ b2, const float *__restrict__ b3, bf16 *__restrict__ a0,
    bf16 *__restrict__ a1, bf16 *__restrict__ a2, float *__restrict__ out, float *__restrict__ out4,
    int n, unsigned *bar, int *err) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ TcPipe pp;
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t hbase = smem_u32(smem);
    if (threadIdx.x == 0) {
        pp.wbuf[0] = hbase + TC_NST * 4 * TC_SLICE;
        pp.wbuf[1] = pp.wbuf[0] + TC_WMAX;
    }
    const uint32_t taddr = tc_pipe_open(pp);
    pdl_trigger();
    const int per = tc_slices(n, (n / TC_TX) * (n / TC_TY));
    tc_layer<16, 32, EPI_GELU_ONLY>(pp, taddr, &tm0, TcOut{b0, nullptr, a0, nullptr, nullptr, nullptr}, n,
                                    hbase, 0, w0, w1, tc_wbytes(32, 32), 0, TC_PRO_PDL, true, err);
    tc_grid_sync(bar, err, pp);
    tc_layer<32, 32, EPI_GELU_ONLY>(pp, taddr, &tm1, TcOut{b1, nullptr, a1, nullptr, nullptr, nullptr}, n,
                                    hbase, 1, nullptr, w2, tc_wbytes(32, 32), per, TC_PRO_PROXY,
                                    true, err);
    tc_grid_sync(bar, err, pp);
    tc_layer<32, 32, EPI_GELU_ONLY>(pp, taddr, &tm2, TcOut{b2, nullptr, a2, nullptr, nullptr, nullptr}, n,
                                    hbase, 0, nullptr, w3, tc_wbytes(32, 16), 2 * per,
                                    TC_PRO_PROXY, true, err);
    tc_grid_sync(bar, err, pp);
    tc_layer<32, 16, EPI_F32>(pp, taddr, &tm3, TcOut{b3, nullptr, nullptr, out, nullptr, out4}, n, hbase,
                              1, nullptr, nullptr, 0, 3 * per, TC_PRO_PROXY, false, err);
    tc_pipe_close(pp, taddr);
}

}  // namespace dw

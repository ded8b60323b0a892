/*
 * diffwind.h - C-ABI of the GB300 DiffWind hot path (libdiffwind.so).
 *
 * The library implements the data-parallel core of DiffWind (arXiv 2603.09668):
 * the differentiable MLS-MPM substep that moves object particles under a
 * spatio-temporal wind-force field (Sec. 3.3, Eq. simulation_mpm; App. A.3,
 * Eqs. P2G, G2P, deformation_update, constitutive_model, young_poisson), the
 * D3Q19 lattice Boltzmann step that supplies the wind-field physics
 * constraint (Sec. 3.1, Eqs. lbe, lbm_sum_v2; Sec. 3.4), the particle-to-voxel
 * obstacle mask (Sec. 3.4, Eq. point2voxel), and hand-written adjoints of
 * each. All compute runs in CUDA kernels built for sm_103a.
 *
 * Conventions for every call:
 *  - Pointers named as device pointers must point to device memory (cudaMalloc,
 *    or a framework's device tensor); the caller owns them. The library owns
 *    only the workspace it allocates in *_create and frees in *_destroy.
 *  - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *    dw_stream; NULL is the legacy default stream). Host-visible status only
 *    covers argument checks and launch errors; conditions found on the device
 *    (a particle outside the grid, a non-finite value, an inverted element)
 *    set a per-handle device status word read by *_device_status.
 *  - Every call returns DW_OK or an error code; dw_last_error() returns a
 *    message for the last failing call on the calling thread. No call aborts,
 *    throws or traps.
 *  - Floating point data is float32 (IEEE binary32). Particle arrays are
 *    structure of arrays: x[3][n] means x[a*n + p] for axis a of particle p;
 *    3x3 matrices are [9][n], row-major per particle: C[(3a+b)*n + p] = C_ab.
 *  - A handle may be used from one stream at a time; calls on one handle that
 *    overlap on the GPU race on its workspace.
 */
#ifndef DIFFWIND_H
#define DIFFWIND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Symbols of this header are the library's only exported names. */
#if defined(__GNUC__)
#define DW_API __attribute__((visibility("default")))
#else
#define DW_API
#endif

typedef enum {
    DW_OK = 0,
    DW_ERR_ARG = 1,       /* bad argument: null pointer, size out of range, unsupported option */
    DW_ERR_CUDA = 2,      /* a CUDA runtime call or kernel launch failed */
    DW_ERR_OOM = 3,       /* a workspace allocation failed */
    DW_ERR_NONFINITE = 4, /* device: a NaN or Inf was produced or read */
    DW_ERR_DOMAIN = 5,    /* device: a particle's 3x3x3 stencil left the grid */
    DW_ERR_TIMEOUT = 6,   /* device: a bounded wait gave up */
    DW_ERR_INVERTED = 7,  /* device: det F <= 0 where the constitutive model needs J > 0 */
    DW_ERR_IO = 8         /* host file: cannot be opened, read or written, or not the expected format */
} dw_status;

typedef void *dw_stream; /* cudaStream_t */

/* Message of the last failing call on this thread ("" if none). */
DW_API const char *dw_last_error(void);
/* Library version string. */
DW_API const char *dw_version(void);

/* FP32 throughput probe (a measurement aid; the paper has no counterpart):
 * launches `blocks` CTAs of 256 threads, each thread running `iters` x 128
 * fused multiply-adds on 16 independent chains, as scalar FFMA (paired = 0)
 * or as 64 float2 FFMA2 instructions (paired = 1). *flops receives the
 * launch's floating-point operation count (2 per multiply-add); the caller
 * times the launch on `stream` (asynchronous). out is a device float array
 * of at least `blocks` entries that is written only to keep the chains live.
 * Errors: DW_ERR_ARG for NULL pointers or counts < 1. */
DW_API dw_status dw_fp32_probe(int32_t paired, int32_t iters, int32_t blocks, float *out,
                               double *flops, dw_stream stream);

/* ===================================================================== wind
 * Wind force field a_w(x, t) (Sec. 3: the wind is a grid field whose force
 * property acts on the MPM background grid; Sec. 3.3: one field per time step).
 * Nodes are node-centred on the unit cube: node j of nf sits at j / (nf - 1).
 * Sampling is trilinear in space and linear in time between n_frames keyframes
 * at k * t_total / (n_frames - 1); positions outside [0,1]^3 and times outside
 * [0, t_total] are clamped. The value is a force per unit mass (N/kg).
 */
typedef struct {
    const float *values; /* device [n_frames][nf][nf][nf][3], x index fastest */
    int32_t nf;          /* nodes per axis, >= 2 (1 = spatially constant) */
    int32_t n_frames;    /* keyframes, >= 1 */
    float t_total;       /* time of the last keyframe; > 0 when n_frames > 1 */
} dw_wind_field;

/* out[3][n] = a_w(pos[:, p], t) for n positions pos[3][n] (device pointers).
 * Errors: DW_ERR_ARG for null pointers with n > 0, nf < 1, n_frames < 1,
 * t_total <= 0 with n_frames > 1. */
DW_API dw_status wind_field_sample(const dw_wind_field *w, const float *pos, int64_t n, float t,
                            float *out, dw_stream stream);

/* Adjoint: g_values += S^T g_out, where S is the linear map values -> out of
 * wind_field_sample at the same positions and time. g_values has the shape of
 * w->values and is accumulated into (atomically). */
DW_API dw_status wind_field_sample_adjoint(const dw_wind_field *w, const float *pos, int64_t n, float t,
                                    const float *g_out, float *g_values, dw_stream stream);

/* ====================================================================== MPM
 * One MLS-MPM substep S (Eq. simulation_mpm): (x, v, F, C)^t -> (x, v, F, C)^{t+1}.
 *   P2G (Eq. P2G) with quadratic B-spline weights on the 3x3x3 stencil, APIC
 *   affine momentum and the MLS stress term -dt V0 (4/dx^2) P F^T (x_i - x_p);
 *   grid update v_i = p_i/m_i + dt (g + a_w(x_i, t)) for nodes with m_i > 0,
 *   v_i = 0 in a sticky band of bc_band nodes at each face;
 *   G2P (Eq. G2P): v_p = sum w v_i, C_p = (4/dx^2) sum w v_i (x_i - x_p)^T,
 *   x_p += dt v_p, F_p <- (I + dt C_p) F_p (Eq. deformation_update, with the C
 *   of this G2P). Pinned particles keep v = 0, C = 0.
 *   Stress P(F): Neo-Hookean mu (F - F^-T) + lam ln(J) F^-T (the gradient of
 *   the energy of Eq. constitutive_model) or fixed-corotated
 *   2 mu (F - R) + lam (J - 1) J F^-T; mu, lam from E, nu (Eq. young_poisson).
 * The grid has n_grid^3 nodes on the unit cube, dx = 1 / n_grid, node (i,j,k)
 * at (i, j, k) dx. A particle must keep floor(x / dx - 0.5) in [0, n_grid - 3]
 * on every axis; otherwise DW_ERR_DOMAIN is raised on the device and the
 * particle is left unchanged.
 */
enum { DW_NEOHOOKEAN = 0, DW_FIXED_COROTATED = 1 };
/* P2G accumulation strategies (results agree to float rounding): global float4
 * atomics per particle and node (ATOMIC); per-warp sums of runs of particles
 * that share a cell, one atomic per node and run (WARP); a CTA-wide shared
 * tile (TILE). In mpm_rollout's fused G2P/P2G kernel, AUTO and PAIR run two
 * particles per thread on paired float2 arithmetic with the warp sums; the
 * other strategies run the one-particle-per-thread fused kernel. Outside
 * mpm_rollout PAIR and AUTO use WARP. */
enum { DW_P2G_AUTO = 0, DW_P2G_ATOMIC = 1, DW_P2G_WARP = 2, DW_P2G_TILE = 3, DW_P2G_PAIR = 4 };

typedef struct {
    int32_t n_grid;        /* nodes per axis, 8 <= n_grid <= 512 */
    float dt;              /* substep length (s) */
    float gravity[3];      /* body acceleration (m/s^2) */
    int32_t bc_band;       /* sticky wall band width in nodes, >= 0 */
    int32_t material;      /* DW_NEOHOOKEAN or DW_FIXED_COROTATED */
    float E, nu;           /* Young's modulus (Pa) and Poisson ratio, 0 <= nu < 0.5 */
    float p_mass, p_vol;   /* particle mass m_p and rest volume V_p^0 */
    int64_t max_particles; /* capacity of the per-particle workspace */
    int32_t p2g_mode;      /* DW_P2G_*: P2G accumulation strategy (results agree to rounding) */
} dw_mpm_desc;

typedef struct {
    float *x; /* device [3][n] positions */
    float *v; /* device [3][n] velocities */
    float *C; /* device [9][n] affine velocity matrices */
    float *F; /* device [9][n] deformation gradients */
    int64_t n;
} dw_mpm_state;

typedef struct dw_mpm_s *dw_mpm;

/* Allocate a handle and its workspace (grid, adjoint grid, per-particle
 * scratch for max_particles). Errors: DW_ERR_ARG, DW_ERR_OOM, DW_ERR_CUDA. */
DW_API dw_status mpm_create(const dw_mpm_desc *desc, dw_mpm *out);
DW_API dw_status mpm_destroy(dw_mpm h);

/* Change E and nu of an existing handle (takes effect for later calls). */
DW_API dw_status mpm_set_material(dw_mpm h, float E, float nu);

/* One substep at time t (the wind is sampled at t). `out` may be the same
 * arrays as `in` (in place) but must not partially overlap them. pinned is a
 * device uint8[n] (nonzero = pinned) or NULL. n <= max_particles. */
DW_API dw_status mpm_substep(dw_mpm h, const dw_mpm_state *in, const dw_mpm_state *out,
                      const uint8_t *pinned, const dw_wind_field *wind, float t,
                      dw_stream stream);

/* Reverse mode of mpm_substep at the same input state, wind and time. Given
 * g_out = dL/d(output state), writes g_in = dL/d(input state) (overwritten;
 * may be the same arrays as g_out), and accumulates dL/d(wind values) into
 * g_wind (device, shape of wind->values; NULL to skip) and dL/dE into *g_E
 * (device float; NULL to skip). The forward grid is recomputed from `in`. */
DW_API dw_status mpm_substep_adjoint(dw_mpm h, const dw_mpm_state *in, const dw_mpm_state *g_out,
                              const dw_mpm_state *g_in, const uint8_t *pinned,
                              const dw_wind_field *wind, float t, float *g_wind, float *g_E,
                              dw_stream stream);

/* Reverse mode of n_substeps substeps (a checkpointed segment) in one call:
 * recomputes the states 1 .. n_substeps - 1 from `start` (state 0, at time
 * t0) into `tape` (device float, (n_substeps - 1) * 24 * n floats, each state
 * as x, v, C, F back to back; caller-owned, tape_floats its size), then runs
 * mpm_substep_adjoint from the last substep back to the first at times
 * t0 + j dt. g holds dL/d(state after the segment) on entry and is
 * overwritten with dL/d(start); g_wind and g_E accumulate as in
 * mpm_substep_adjoint. The substeps are those of mpm_substep (no sorting).
 * The recompute also keeps each substep's grid (the active blocks' mass and
 * momentum) in a handle-owned grid tape, which the reverse substeps restore
 * instead of repeating the P2G of their input; the tape grows on the first
 * call with a longer segment (device allocation: make that call outside a
 * stream capture) and is used only while it leaves 8 GB of device memory
 * free, otherwise the grids are recomputed (results agree to the float
 * atomics' order). */
DW_API dw_status mpm_segment_adjoint(dw_mpm h, const dw_mpm_state *start, float *tape,
                                     int64_t tape_floats, const dw_mpm_state *g,
                                     const uint8_t *pinned, const dw_wind_field *wind, float t0,
                                     int32_t n_substeps, float *g_wind, float *g_E,
                                     dw_stream stream);

/* Reorder particles by grid cell (the cell of floor(x/dx - 0.5), cells
 * grouped into 4^3 blocks) so that neighbouring P2G threads share stencils.
 * Writes the permuted state into `out` (must not overlap `in`) and the
 * permuted pin flags into pinned_out (when pinned_in is not NULL). With
 * perm[k] the index in `in` of the particle now at k, ids_out[k] =
 * ids_in[perm[k]] when ids_in (device int32[n]) is given, else perm[k]; so
 * carrying ids through successive sorts tracks every particle's original
 * index. The order of particles that share a cell is unspecified. */
DW_API dw_status mpm_sort(dw_mpm h, const dw_mpm_state *in, const dw_mpm_state *out,
                          const uint8_t *pinned_in, uint8_t *pinned_out, const int32_t *ids_in,
                          int32_t *ids_out, dw_stream stream);

/* n_substeps substeps of mpm_substep at times t0, t0 + dt, ... applied in
 * place to `state` (Eq. simulation_mpm iterated), the same arithmetic as
 * calling mpm_substep n_substeps times. Every sort_every substeps (0 = never)
 * the particles are re-sorted by cell as in mpm_sort, so on return the arrays
 * hold the particles in a new order: `pinned` (device uint8[n] or NULL) is
 * permuted along, and ids (device int32[n], required when sort_every > 0) is
 * carried through the sorts (ids_out[k] = ids_in[perm[k]]), so filling it with
 * 0..n-1 beforehand yields each particle's original index. The G2P of one
 * substep and the P2G of the next run fused in one kernel, which keeps v and
 * C in registers (the arrays v and C are written only by the last substep's
 * G2P); a re-sort runs between two fused launches, after the P2G of the
 * substep that follows it. The state is complete at the end. Uses the
 * handle's second state buffer (max_particles). */
DW_API dw_status mpm_rollout(dw_mpm h, const dw_mpm_state *state, uint8_t *pinned, int32_t *ids,
                             const dw_wind_field *wind, float t0, int32_t n_substeps,
                             int32_t sort_every, dw_stream stream);

/* Waits for `stream`, returns the first device-side error recorded on this
 * handle since the last call (DW_OK if none) and clears it. */
DW_API dw_status mpm_device_status(dw_mpm h, dw_stream stream);

/* Instrumentation (no counterpart in the paper): while enabled, every kernel
 * the handle launches is bracketed by CUDA events recorded on the call's
 * stream, up to `max_records` launches (events are created here, so enable
 * before any stream capture; calls made while enabled must not be captured).
 * mpm_profile_read waits for the recorded events and returns, per kernel id
 * DW_K_*, the summed device milliseconds and the launch count since enable,
 * then clears them. Arrays have DW_K_COUNT entries. */
enum { DW_K_P2G = 0, DW_K_GRID = 1, DW_K_G2P = 2, DW_K_REV_G2P = 3, DW_K_REV_GRID = 4,
       DW_K_REV_P2G = 5, DW_K_SORT = 6, DW_K_G2P2G = 7, DW_K_COUNT = 8 };
DW_API dw_status mpm_profile_enable(dw_mpm h, int32_t max_records);
DW_API dw_status mpm_profile_read(dw_mpm h, double *total_ms, int64_t *launches);

/* Host checkpoints of an MPM state, so that a rollout or an inversion can be
 * resumed in another process from saved particles, time and substep counter
 * (the checkpoints inside a rollout's adjoint stay in device memory).
 * mpm_state_save copies `state` (device x, v, C, F of state->n particles)
 * and, when not NULL, `pinned` (device uint8[n]) and `ids` (device int32[n])
 * to the host on `stream`, waits for them, and writes the file `path`:
 * the 8-byte tag "DWMPMST1", int64 n, float64 t, int64 substep, int32 flags
 * (bit 0 pinned present, bit 1 ids present), int32 0, then the float32 rows
 * x[3][n], v[3][n], C[9][n], F[9][n], then pinned and ids when present, in
 * the host's byte order (little-endian on both supported hosts). The file is
 * written to path + ".tmp" and renamed over `path` when complete, so an
 * interrupted save keeps the previous checkpoint. mpm_state_peek reads only
 * the header (n, flags, t, substep; each output may be NULL; no GPU needed),
 * to size the buffers of a load. mpm_state_load reads the file into `state`
 * (state->n must equal the file's n: DW_ERR_ARG otherwise) and, when not
 * NULL, pinned and ids (DW_ERR_ARG if the file lacks them), and returns t and
 * substep (may be NULL); it waits for its copies on `stream`. Errors: DW_ERR_IO
 * for a file that cannot be opened, read or written, a wrong tag or header,
 * or a size that does not match the header; DW_ERR_OOM when the host buffer
 * cannot be allocated; DW_ERR_CUDA for a failed copy. */
DW_API dw_status mpm_state_save(const char *path, const dw_mpm_state *state, const uint8_t *pinned,
                                const int32_t *ids, double t, int64_t substep, dw_stream stream);
DW_API dw_status mpm_state_peek(const char *path, int64_t *n, int32_t *flags, double *t,
                                int64_t *substep);
DW_API dw_status mpm_state_load(const char *path, const dw_mpm_state *state, uint8_t *pinned,
                                int32_t *ids, double *t, int64_t *substep, dw_stream stream);

/* The same substep as mpm_substep for callers that cannot allocate device
 * memory when they need it (for example code running inside an allocator
 * callback or under its lock, a real-time loop that forbids allocation after
 * start-up, or a host whose memory pool owns the whole device and only lends
 * out buffers). The paper has no counterpart; this is a deployment variant.
 * No handle is needed: the scratch grid is a fixed device array inside the
 * library, sized for n_grid <= 64 (64^3 nodes, 8 MB, held on every GPU that
 * loads the library until the process exits); a larger n_grid is rejected
 * with DW_ERR_ARG. The call allocates nothing: no cudaMalloc, no cudaFree,
 * no allocating library routine. desc->max_particles is ignored; in, out,
 * pinned, wind and t are as in mpm_substep, and `out` may equal `in`.
 * device_status is an optional caller-owned device int32 into which
 * device-side error bits are OR-ed (DW_ERR_DOMAIN -> 2, DW_ERR_NONFINITE -> 1,
 * DW_ERR_INVERTED -> 8); with NULL those conditions are not reported.
 * The first call on a device looks up the array's device address with the
 * calling thread's current device (cudaGetSymbolAddress); make that first
 * call before any stream capture. Every call on a device shares the one
 * array and the call zeroes the part it uses before P2G, so calls that
 * overlap on the GPU (different streams, or threads without ordering) race
 * and must be serialised by the caller. */
DW_API dw_status mpm_substep_noalloc(const dw_mpm_desc *desc, const dw_mpm_state *in,
                                     const dw_mpm_state *out, const uint8_t *pinned,
                                     const dw_wind_field *wind, float t,
                                     int32_t *device_status, dw_stream stream);

/* ================================================ physics-informed wind loss
 * Sec. 3.4: the LBM velocity D_guide steers the direction of the wind force
 * D_recon through L_phys = |D_recon - (D_recon . D_guide) D_guide|^2. Read
 * per wind-grid node of one keyframe, with d = u / |u| the unit direction of
 * the LBM velocity u there: the term |F - (F.d) d|^2 is the square of the
 * force component across the flow; nodes with |u| <= eps (still or solid)
 * give no guidance and add nothing. Its gradient is 2 (F - (F.d) d).
 */

/* loss (device float, accumulated) += weight * the sum of the terms over the
 * n nodes; g_values (device [n][3], accumulated, may be NULL) += weight * their
 * gradients (weight is the loss's factor in a weighted sum of losses).
 * values [n][3] is one keyframe's slice of dw_wind_field.values, guide_u
 * [3][n] the LBM velocity at the same nodes (lbm_sample_velocity). */
DW_API dw_status wind_phys_loss(const float *values, const float *guide_u, int64_t n, float eps,
                                float weight, float *loss, float *g_values, dw_stream stream);

/* Scores of a reconstructed wind force field against a reference one
 * (App. E.2, the CosSim / NMSE evaluation): both forces at a location are
 * normalised to unit length, a^ and b^. Over the n locations where both have
 * |.| > eps, sums (device float[3], accumulated, so several keyframes add up)
 * += {sum a^.b^, sum |a^ - b^|^2, number of such locations}; CosSim =
 * sums[0] / sums[2] and NMSE = sums[1] / sums[2]. rec, gt are [n][3]. */
DW_API dw_status wind_field_scores(const float *rec, const float *gt, int64_t n, float eps,
                                   float *sums, dw_stream stream);

/* The aerodynamic drag relation of Sec. 3.4, F_w = 1/2 rho_w C_D |v|^2 v/|v|,
 * per node: values[k] = scale |u_k| u_k, with u [3][n] a wind velocity (e.g.
 * lbm_sample_velocity at the wind-grid nodes) and values [n][3] one keyframe
 * of dw_wind_field.values (overwritten). scale folds 1/2 rho_w C_D, the
 * object's mass density and the lattice-to-physical velocity unit into one
 * constant, so values is the wind acceleration the MPM grid update adds. */
DW_API dw_status wind_drag_force(const float *u, int64_t n, float scale, float *values,
                                 dw_stream stream);

/* The trajectory term of the inversion loop: loss (device float, accumulated)
 * += weight * sum_p |x_p - x_target_p|^2 over n particles, and g_x (device
 * [3][n], accumulated, may be NULL) += 2 weight (x_p - x_target_p), the
 * gradient an MPM adjoint takes as dL/dx of the final state. x and x_target
 * are device [3][n]. */
DW_API dw_status position_loss(const float *x, const float *x_target, int64_t n, float weight,
                               float *loss, float *g_x, dw_stream stream);

/* One Adam step (Kingma and Ba, with bias correction) on n parameters:
 * m, v are the moment buffers (device, zero before step 1), step >= 1. The
 * update of the wind inversion loop (per keyframe, Sec. 3.3). */
DW_API dw_status adam_step(float *param, const float *grad, float *m, float *v, int64_t n,
                           float lr, float beta1, float beta2, float eps, int32_t step,
                           dw_stream stream);

/* VectorAdam (Ling, Sharp and Jacobson, 2022) on n 3-vectors param [n][3]:
 * m [n][3] is the first moment per component, v [n] the second moment of the
 * squared norm |g|^2 of each vector's gradient (both zero before step 1);
 * param -= lr * m^ / (sqrt(v^) + eps) with Adam's bias corrections. Unlike
 * adam_step the update of a vector is a rotation of its gradient's history,
 * so a rotated problem gives the rotated answer: the wind inversion uses it
 * for the per-node force vectors. step >= 1. */
DW_API dw_status vector_adam_step(float *param, const float *grad, float *m, float *v, int64_t n,
                                  float lr, float beta1, float beta2, float eps, int32_t step,
                                  dw_stream stream);

/* ================================================ particle-bound Gaussians
 * The object's 3D Gaussians ride on MPM particles (Sec. 3.2): the covariance
 * of particle p follows its deformation gradient, Sigma_p(t) = F_p Sigma_p
 * F_p^T, and the object is drawn by alpha-blended splatting (Sec. 3.3, Eq.
 * rendering; the 3D Gaussian representation): with t = R x + T the camera-
 * space centre, mu' = (fx t_x/t_z + cx, fy t_y/t_z + cy), J the Jacobian of
 * that projection at t, Sigma' = J R Sigma R^T J^T, each pixel centre p
 * (pixel (i, j) at (i + 1/2, j + 1/2)) gets C = sum_i T_i c_i alpha_i over the
 * Gaussians in increasing t_z (ties by index), T_i = prod_{j<i} (1 -
 * alpha_j), alpha_i = o_i exp(-q/2) for q = (p - mu')^T Sigma'^-1 (p - mu') <=
 * 9 (three standard deviations) and 0 beyond; Gaussians with t_z <= near or
 * a singular Sigma' are not drawn; no background term. Layouts: x [3][n], F
 * [9][n] (row-major per particle, as dw_mpm_state), covariances [6][n] as
 * (xx, yy, zz, xy, xz, yz), colours [3][n], opacities [n], images [3][H][W].
 */
typedef struct {
    float R[9];     /* world -> camera rotation, row-major */
    float T[3];     /* world -> camera translation */
    float fx, fy;   /* focal lengths in pixels, > 0 */
    float cx, cy;   /* principal point in pixels */
    int32_t width, height;
    float near_z;   /* Gaussians with t_z <= near_z are not drawn; > 0 */
} dw_camera;

typedef struct dw_gs_s *dw_gs;

/* sigma [6][n] = F sigma0 F^T per particle (device arrays). */
DW_API dw_status gs_covariance(const float *F, const float *sigma0, int64_t n, float *sigma,
                               dw_stream stream);

/* Renderer workspace for up to max_gaussians Gaussians and width x height
 * images (about 100 bytes per Gaussian plus one image). */
DW_API dw_status gs_create(int64_t max_gaussians, int32_t width, int32_t height, dw_gs *out);
DW_API dw_status gs_destroy(dw_gs h);

/* image (device [3][H][W], overwritten) of n Gaussians at the particles x
 * with deformation gradients F and rest covariances sigma0. The handle keeps
 * the projected Gaussians, their depth order, the per-tile lists and the
 * image for gs_render_backward. cam's image size must be the handle's. The
 * call reads the tile-list length back to the host (4 bytes) to size the
 * lists, so it waits for `stream` and cannot be captured in a CUDA graph. */
DW_API dw_status gs_render(dw_gs h, const dw_camera *cam, const float *x, const float *F,
                           const float *sigma0, const float *color, const float *opacity,
                           int64_t n, float *image, dw_stream stream);

/* Reverse mode of the last gs_render, which must have drawn the same inputs:
 * given g_image = dL/d(image), accumulates dL/dx into g_x [3][n] and dL/dF
 * into g_F [9][n] (the MPM adjoint's inputs for the final state), and, when
 * not NULL, dL/d(color) into g_color [3][n] and dL/d(opacity) into g_opacity
 * [n]. The pixel rule q <= 9 makes the image piecewise smooth; the gradient
 * is that of the smooth piece. DW_ERR_ARG when n, an input pointer or the
 * camera differs from the last gs_render (the arrays' contents must not have
 * changed since; that is the caller's to keep). */
DW_API dw_status gs_render_backward(dw_gs h, const dw_camera *cam, const float *x, const float *F,
                                    const float *sigma0, const float *color,
                                    const float *opacity, int64_t n, const float *g_image,
                                    float *g_x, float *g_F, float *g_color, float *g_opacity,
                                    dw_stream stream);

/* The L1 term of the photometric loss (Sec. 3.3): loss (device float,
 * accumulated) += weight sum |image - target| over n values; g_image (device,
 * accumulated, may be NULL) += weight sign(image - target). */
DW_API dw_status image_l1_loss(const float *image, const float *target, int64_t n, float weight,
                               float *loss, float *g_image, dw_stream stream);

/* The structural term of L_render (Sec. 3.3): loss (device float,
 * accumulated) += weight (1 - mean SSIM) over the channels x height x width
 * values of image against target, SSIM = ((2 mu_x mu_y + C1)(2 s_xy + C2)) /
 * ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)) with local means and
 * (co)variances under an 11 x 11 Gaussian window (sigma 1.5, zero outside the
 * image), C1 = 0.01^2, C2 = 0.03^2; g_image (may be NULL) += its gradient
 * with respect to image. workspace: device, 10 x channels x height x width
 * floats. Images are [channels][height][width]. */
DW_API dw_status image_dssim_loss(const float *image, const float *target, int32_t channels,
                                  int32_t height, int32_t width, float weight, float *loss,
                                  float *g_image, float *workspace, dw_stream stream);

/* ============================================================ batched MPM
 * Many independent scenes, each with its own grid size, material, time step,
 * particle count and wind field, advanced by the same substep as mpm_rollout
 * (Eq. simulation_mpm per scene; no data flows between scenes). The paper
 * runs one scene at a time; batching is a throughput variant for ensembles
 * such as several objects, wind candidates or optimisation restarts.
 *
 * Particle state of the batch: ONE concatenated structure-of-arrays state of
 * n = sum n_particles particles (x[3][n], v[3][n], C[9][n], F[9][n], pinned
 * uint8[n], ids int32[n]); scene s owns the particles [off_s, off_s + n_s)
 * with off_s = n_0 + ... + n_(s-1), in the order the scenes were given. A
 * particle never changes scene: sorting permutes within each scene's range.
 *
 * Launch shape (dw_batch_config): in DW_BATCH_PERSISTENT mode every substep
 * is ONE cooperative kernel launch whose CTAs first run the grid update of the
 * active 4^3 node blocks of all scenes, meet at a grid-wide barrier, then run
 * G2P of the substep fused with the P2G of the next one over 128-particle
 * work items (one scene per item). The barrier's wait is bounded: if it gives
 * up, the device status becomes DW_ERR_TIMEOUT and later substeps of the
 * batch do nothing until mpm_batch_device_status clears it. DW_BATCH_SPLIT
 * runs the two phases as two launches (programmatic dependent launch).
 * DW_BATCH_PAIR is DW_BATCH_SPLIT with the fused phase of mpm_rollout's
 * default kernel (two particles per thread on paired FP32 instructions, 64
 * particles of one scene per warp); it is the default configuration. With
 * use_graph, the whole launch sequence of a rollout is captured once per
 * distinct (state pointers, n_substeps, sort_every, config) in a CUDA graph
 * owned by the handle and replayed; if capture is not possible the sequence
 * is launched directly (mpm_batch_get_config reports graph_active = 0).
 */
enum { DW_BATCH_PERSISTENT = 0, DW_BATCH_SPLIT = 1, DW_BATCH_PAIR = 2 };

typedef struct {
    dw_mpm_desc desc;      /* the scene's physics; desc.max_particles and desc.p2g_mode are ignored */
    int64_t n_particles;   /* particles of the scene, >= 1 */
    dw_wind_field wind;    /* the scene's wind field; its device values are read by every later
                              rollout and must stay valid and unchanged while the handle lives */
} dw_mpm_scene;

typedef struct {
    int32_t mode;          /* DW_BATCH_PERSISTENT, DW_BATCH_SPLIT or DW_BATCH_PAIR */
    int32_t threads;       /* CTA size, 128 or 256 (one or two 128-particle work items per CTA);
                              PAIR: of the grid-update launch (the paired kernel has 128) */
    int32_t ctas_per_sm;   /* PERSISTENT: resident CTAs per SM (>= 1, clamped to the occupancy
                              limit); SPLIT, PAIR: CTAs per SM of the grid-update launch */
    int32_t use_graph;     /* nonzero: replay rollouts from a CUDA graph */
    int32_t graph_active;  /* output of mpm_batch_get_config: the last rollout ran from a graph */
} dw_batch_config;

typedef struct {
    dw_batch_config config;
    float ms_per_substep;  /* measured device time of one substep with this configuration */
} dw_batch_trial;

typedef struct dw_mpm_batch_s *dw_mpm_batch;

/* Allocate a batch for n_scenes scenes (1 <= n_scenes <= 2048): per-scene
 * grids, active-block lists, the sort workspace and a second state buffer of
 * n particles. Each desc is checked as in mpm_create; every scene's n_grid
 * must be <= 400, and the sum of n_grid^3 over the scenes below 2^31. The
 * initial configuration is PERSISTENT, 128 threads, the occupancy limit of
 * CTAs per SM, graphs on. Errors: DW_ERR_ARG, DW_ERR_OOM, DW_ERR_CUDA. */
DW_API dw_status mpm_batch_create(const dw_mpm_scene *scenes, int32_t n_scenes, dw_mpm_batch *out);
DW_API dw_status mpm_batch_destroy(dw_mpm_batch h);

/* Total particle count n of the batch and the first particle of each scene:
 * offsets (host int64[n_scenes + 1] or NULL) receives off_0 .. off_n_scenes. */
DW_API dw_status mpm_batch_layout(dw_mpm_batch h, int64_t *n_total, int64_t *offsets);

/* n_substeps substeps of every scene, in place on the concatenated `state`
 * (state->n must equal the batch's n): scene s runs mpm_rollout's arithmetic
 * with its own desc and wind at times t0 + k dt_s, k = 0 .. n_substeps - 1.
 * Every sort_every substeps (0 = never) each scene's particles are re-sorted
 * by cell within the scene's range; pinned (device uint8[n] or NULL) is
 * permuted along and ids (device int32[n], required when sort_every > 0) is
 * carried through the sorts as in mpm_rollout. */
DW_API dw_status mpm_batch_rollout(dw_mpm_batch h, const dw_mpm_state *state, uint8_t *pinned,
                                   int32_t *ids, float t0, int32_t n_substeps, int32_t sort_every,
                                   dw_stream stream);

DW_API dw_status mpm_batch_set_config(dw_mpm_batch h, const dw_batch_config *config);
DW_API dw_status mpm_batch_get_config(dw_mpm_batch h, dw_batch_config *config);

/* Autotuner: times every candidate launch shape (the three modes, 128 and
 * 256 threads, each resident-CTA count up to the occupancy limit) on
 * n_trial_substeps substeps of the batch started from `state` sorted by cell
 * (as a rollout with re-sorting starts; the sorted copy goes into the
 * handle's workspace, `state` and `pinned` are not modified), keeps the
 * fastest as the handle's configuration (use_graph unchanged) and returns it
 * in *best (may be NULL). trials (host, max_trials entries, or NULL) receives
 * each candidate and its time; *n_trials (may be NULL) their number. The call
 * waits for `stream`. */
DW_API dw_status mpm_batch_tune(dw_mpm_batch h, const dw_mpm_state *state, const uint8_t *pinned,
                                int32_t n_trial_substeps, dw_batch_config *best,
                                dw_batch_trial *trials, int32_t max_trials, int32_t *n_trials,
                                dw_stream stream);

/* As mpm_device_status, for the batch (any scene). Also resets the barrier
 * state, so a batch whose barrier gave up is usable again afterwards. */
DW_API dw_status mpm_batch_device_status(dw_mpm_batch h, dw_stream stream);

/* Size of the batch's concatenated wind gradient: scene s's block (shaped like
 * its wind values, n_frames * nf^3 * 3 floats) starts at offsets[s] (host
 * int64[n_scenes + 1] or NULL); *n_floats (may be NULL) is the total. */
DW_API dw_status mpm_batch_wind_layout(dw_mpm_batch h, int64_t *n_floats, int64_t *offsets);

/* Reverse mode of n_substeps batched substeps (a checkpointed segment of
 * every scene at once; Eq. simulation_mpm differentiated as in
 * mpm_segment_adjoint, scene by scene). Recomputes the states 1 ..
 * n_substeps - 1 from `start` (state 0 of the concatenated batch, substep j
 * of scene s at t0 + j dt_s) into `tape` (device float, (n_substeps - 1) *
 * 24 * n floats, each state as x, v, C, F back to back; caller-owned,
 * tape_floats its size) with the handle's launch configuration, then runs
 * the reverse substeps from the last to the first over all scenes. The
 * recompute keeps each substep's grid in a handle-owned grid tape (every
 * block of every scene per recomputed substep: 1 KB x the batch's blocks,
 * grown on the first call with a longer segment and used only while it
 * leaves 8 GB of device memory free), from which the reverse substeps
 * restore their forward grids; without it they recompute them by a P2G of
 * their input (results agree to the float atomics' order). With use_graph the whole sequence is captured once per distinct
 * (tape, g, pinned, g_wind, g_E, n_substeps, configuration) in a CUDA graph
 * owned by the handle and replayed; `start` is first copied into the handle's
 * workspace, so successive segments with different start states share one
 * graph (the workspace is the one mpm_batch_rollout and mpm_batch_tune use;
 * calls on one handle must not overlap). g (concatenated, n particles) holds
 * dL/d(state after the segment) on entry and is overwritten with
 * dL/d(start). g_wind (device, mpm_batch_wind_layout floats, or NULL)
 * accumulates each scene's dL/d(wind values) at its offset; g_E (device
 * float[n_scenes], or NULL) accumulates each scene's dL/dE. The substeps are
 * those of mpm_batch_rollout without sorting. The first call allocates the
 * reverse-mode workspace (two float4 per grid node of all scenes, 12 floats
 * per particle) and the grid tape, kept until mpm_batch_destroy. Errors: DW_ERR_ARG (state
 * sizes, a missing or short tape), DW_ERR_OOM, DW_ERR_CUDA; device-side
 * failures go to the batch's device status. */
DW_API dw_status mpm_batch_segment_adjoint(dw_mpm_batch h, const dw_mpm_state *start,
                                           float *tape, int64_t tape_floats,
                                           const dw_mpm_state *g, const uint8_t *pinned, float t0,
                                           int32_t n_substeps, float *g_wind, float *g_E,
                                           dw_stream stream);

/* Failure-detection self-test of the persistent kernel's grid barrier: one
 * cooperative launch of one CTA per SM runs the barrier alone, told to wait
 * for missing_ctas (0..1024) more CTAs than were launched. With 0 it must
 * pass (returns DW_OK); otherwise every CTA's bounded wait runs out (about a
 * second) and the call returns DW_ERR_TIMEOUT. Waits for `stream` and clears
 * the status like mpm_batch_device_status. */
DW_API dw_status mpm_batch_barrier_selftest(dw_mpm_batch h, int32_t missing_ctas,
                                            dw_stream stream);

/* ====================================================================== LBM
 * D3Q19 lattice Boltzmann step (Eq. lbe) with the BGK collision
 * f* = f - (f - f_eq)/tau (+ Guo forcing for a uniform body force F, with
 * rho u = sum c f + F/2 as in Eq. lbm_sum_v2), f_eq = w rho (1 + 3 c.u +
 * 4.5 (c.u)^2 - 1.5 u.u), then streaming f_i(x + c_i) = f*_i(x).
 * Boundaries: halfway bounce-back on solid cells; y and z periodic; x periodic
 * (bc_x = 0) or (bc_x = 1) an equilibrium inlet at x = 0 (populations entering
 * through the x = 0 face are f_eq(1, u_inlet)) and a zero-gradient outlet at
 * x = nx - 1 (populations entering through that face equal the cell's own
 * post-collision populations of the same direction).
 * Velocity order: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (+x+y),(-x-y),
 * (+x+z),(-x-z),(+y+z),(-y-z),(+x-y),(-x+y),(+x-z),(-x+z),(+y-z),(-y+z);
 * directions 2k-1 and 2k are opposite. Weights 1/3, 1/18, 1/36.
 * Storage: f is device float [19][nz][ny][nx] (x fastest) holding the shifted
 * populations f_i - w_i (deviation from the rest equilibrium, which keeps
 * float32 resolution; a lattice at rest is all zeros). Solid cells' entries
 * are never read or written. solid is device uint8 [nz][ny][nx] (nonzero =
 * solid) or NULL (all fluid).
 */
typedef struct {
    int32_t nx, ny, nz; /* lattice size, each >= 2; 19*nx*ny*nz < 2^31 */
    float tau;          /* BGK relaxation time, > 0.5 */
    float u_inlet[3];   /* inlet velocity (lattice units), used when bc_x = 1 */
    float force[3];     /* uniform body force density (lattice units) */
    int32_t bc_x;       /* 0 periodic in x, 1 inlet/outlet in x */
    int32_t max_tape;   /* lattices of workspace for lbm_step_adjoint (>= 1) */
} dw_lbm_desc;

typedef struct dw_lbm_s *dw_lbm;

DW_API dw_status lbm_create(const dw_lbm_desc *desc, dw_lbm *out);
DW_API dw_status lbm_destroy(dw_lbm h);

/* Keep the link words of mask `solid` (per cell: which of its 18 neighbours
 * are solid, with the periodic wraps and the x boundaries folded in) in the
 * handle, so that the lattice calls given this same `solid` pointer skip
 * rebuilding them. Without it every call with a mask rebuilds them (one
 * launch over the lattice). The caller must not change the mask's contents
 * while it is registered: register it again after a change. solid = NULL
 * drops the registration; a call with another mask drops it too. Not in the
 * paper: a property of this library's lattice kernels (Eq. lbe's bounce-back
 * needs only "is the neighbour solid"). Errors: DW_ERR_ARG for a NULL handle. */
DW_API dw_status lbm_cache_mask(dw_lbm h, const uint8_t *solid, dw_stream stream);

/* Advance f in place by `steps` >= 0 lattice steps. Pairs of steps run as the
 * in-place AA pattern (one collide-only kernel, one pull-collide-push kernel);
 * an odd last step runs through the workspace. */
DW_API dw_status lbm_step(dw_lbm h, float *f, const uint8_t *solid, int32_t steps, dw_stream stream);

/* Reverse mode of lbm_step(f_in, steps): on entry g_f = dL/df(t + steps), on
 * return dL/df(t) (in place). f_in is the state the forward started from;
 * the intermediate states are recomputed into the workspace, so steps must be
 * <= max_tape. Gradients are taken with respect to the shifted populations,
 * which equal those with respect to f. */
DW_API dw_status lbm_step_adjoint(dw_lbm h, const float *f_in, float *g_f, const uint8_t *solid,
                           int32_t steps, dw_stream stream);

/* rho [nz][ny][nx] and u [3][nz][ny][nx] (Eq. lbm_sum_v2; rho u includes F/2).
 * Either output may be NULL. Solid cells get rho = 0, u = 0. */
DW_API dw_status lbm_macroscopic(dw_lbm h, const float *f, const uint8_t *solid, float *rho, float *u,
                          dw_stream stream);

/* The LBM wind velocity at points (the guide of the physics-informed loss,
 * Sec. 3.4): u_out[3][n] = the velocity of Eq. lbm_sum_v2 interpolated
 * trilinearly between cell centres (cell c of an axis with n_a cells spans
 * [c/n_a, (c+1)/n_a), its centre (c + 1/2)/n_a; points are clamped to the box
 * of centres), solid cells (solid may be NULL) counting as at rest. pos is
 * device [3][n] in unit-cube coordinates; f the shifted lattice. Errors:
 * DW_ERR_ARG for null pointers with n > 0. */
DW_API dw_status lbm_sample_velocity(dw_lbm h, const float *f, const uint8_t *solid,
                                     const float *pos, int64_t n, float *u_out, dw_stream stream);

/* Fill f with the shifted equilibrium f_eq(rho0, u0) - w at every cell. */
DW_API dw_status lbm_init_equilibrium(dw_lbm h, float *f, float rho0, const float u0[3],
                               dw_stream stream);

/* ====================================================== HOME-LBM (App. D)
 * The moment-encoded variant of the step above (after Li et al. 2023): a
 * cell stores ten moments of its post-collision populations, m = device float
 * [10][nz][ny][nx] with planes 0: rho - 1, 1-3: u' (momentum over rho after
 * the collision), 4-9: S_xx, S_yy, S_zz, S_xy, S_xz, S_yz with S = sum_i (c_i
 * c_i - I/3) f_i / rho; 40 bytes per cell instead of 76. A step rebuilds
 * every pulled population f_i(x) = f_i^post(x - c_i) from the source cell's
 * moments by the Hermite series (second order in full, plus the six
 * third-order terms H3_aab(c) = c_b (c_a^2 - 1/3) that D3Q19 carries, with
 * the coefficient A_aab = u_b S_aa + 2 u_a S_ab - 2 u_a^2 u_b closed from
 * the lower moments), with the boundaries of lbm_step (halfway bounce-back,
 * the inlet rebuilt from rho = 1, u_inlet, S = u_inlet u_inlet, the
 * zero-gradient outlet), then collides in moment space: with u = (j + F/2) /
 * rho and N = Pi - rho (I/3 + u u), the deviatoric part of N decays by
 * (1 - 1/tau), its trace is dropped (set to equilibrium), and the Guo forcing
 * moment u F + F u enters with 1 - 1/(2 tau) (deviatoric) and 1/2 (trace);
 * u' = u + F / (2 rho). It solves the same Navier-Stokes limit as lbm_step
 * with the same shear viscosity (tau - 1/2) / 3. The handle's descriptor
 * (tau, inlet, force, bc_x) applies; solid cells keep their moments. */

/* Fill m with the collided equilibrium of rho0, u0 (the HOME counterpart of
 * lbm_init_equilibrium: the state f_eq(rho0, u0) taken as pre-collision). */
DW_API dw_status lbm_home_init(dw_lbm h, float *m, float rho0, const float u0[3],
                               dw_stream stream);

/* Advance m in place by `steps` HOME-LBM steps (pull streaming between m and
 * the handle's tape in turn, so max_tape >= 1 suffices; an odd step count ends
 * with one device copy back into m). solid as in lbm_step. */
DW_API dw_status lbm_home_step(dw_lbm h, float *m, const uint8_t *solid, int32_t steps,
                               dw_stream stream);

/* rho [nz][ny][nx] and the macroscopic velocity u [3][nz][ny][nx] = u' -
 * F / (2 rho) of the moments m; solid cells report 0. Either may be NULL. */
DW_API dw_status lbm_home_macroscopic(dw_lbm h, const float *m, const uint8_t *solid, float *rho,
                                      float *u, dw_stream stream);

/* lbm_sample_velocity for HOME-LBM moments m: the macroscopic velocity of
 * lbm_home_macroscopic interpolated at points pos[3][n] the same way. */
DW_API dw_status lbm_home_sample_velocity(dw_lbm h, const float *m, const uint8_t *solid,
                                          const float *pos, int64_t n, float *u_out,
                                          dw_stream stream);

/* Solid mask of Eq. point2voxel: solid[w] = 1 iff some particle lies in
 * [x_w, x_w + dx)^3 with x_w = w dx, i.e. w = floor(x_p / dx); the mask is
 * cleared first; particles outside the lattice are ignored. pos is device
 * [3][n]. */
DW_API dw_status voxelize_particles(const float *pos, int64_t n, int32_t nx, int32_t ny, int32_t nz,
                             float dx, uint8_t *solid, dw_stream stream);

/* ================================================================ surrogate
 * Learned surrogate of the LBM wind constraint (no counterpart in the paper,
 * which runs the LBM every time step, Sec. 3.4): a 4-layer 3D convolutional
 * network on a coarse n^3 grid that maps the coarse state of a (2n)^3
 * lattice to the change du of the coarse velocity over a block of lattice
 * steps. Channels 16 -> 32 -> 32 -> 32 -> 16, kernel 3, zero padding, GELU
 * after layers 1-3; inputs (rho - 1, u - u_ref, solid fraction, u_ref,
 * 0 ...) with rho and u as 2x2x2 averages over fluid cells; outputs du in
 * channels 0..2. BF16
 * activations and weights on the tensor cores with FP32 accumulation; FP32
 * master parameters packed layer by layer as W[tap][cout][cin] then b[cout],
 * tap = (dz+1)*9 + (dy+1)*3 + (dx+1) (the input voxel is v + (dx,dy,dz)).
 * Activations are channels-last [z][y][x][c]. Calls on one handle must not
 * overlap on the GPU. */
typedef struct dw_surr_s *dw_surr;

/* n: coarse grid per axis, a multiple of 16 in [16, 256]; parameters start at 0. */
DW_API dw_status surr_create(int32_t n, dw_surr *out);
DW_API dw_status surr_destroy(dw_surr h);
/* Number of FP32 parameters (83,056 for this architecture). */
DW_API dw_status surr_num_params(dw_surr h, int64_t *count);
/* Copy parameters in from a device FP32 array (and refresh the BF16 weights),
 * or out to one; copy the accumulated gradients out; zero the gradients. */
DW_API dw_status surr_set_params(dw_surr h, const float *src, dw_stream stream);
DW_API dw_status surr_get_params(dw_surr h, float *dst, dw_stream stream);
DW_API dw_status surr_get_grads(dw_surr h, float *dst, dw_stream stream);
DW_API dw_status surr_zero_grads(dw_surr h, dw_stream stream);
/* Reference velocity of the features (host float[3], the lattice's inlet
 * velocity; zero until set): the coarse features carry the fluid velocity
 * relative to it (channels 1-3) and the reference itself (channels 5-7),
 * both multiplied by in_scale, so that BF16 resolves the flow's departures
 * from the free stream and the network knows the inlet. Not in the paper. */
DW_API dw_status surr_set_inlet(dw_surr h, const float u[3]);
/* Coarse features from a shifted (2n)^3 lattice f [19][cells] and its mask:
 * per coarse voxel the 2x2x2 fluid averages of rho - 1 and of u - u_ref
 * (0 without fluid), the solid fraction, and u_ref (surr_set_inlet), the
 * velocities multiplied by in_scale; channels 8-15 are zero. Also keeps the
 * fine rho and u for surr_apply. feats32 (device [n^3][16], may be NULL)
 * receives the features in FP32 as well. */
DW_API dw_status surr_features(dw_surr h, const float *f, const uint8_t *solid, float in_scale,
                               float *feats32, dw_stream stream);
/* Set the coarse features directly from FP32 [n^3][16] (rounded to BF16). */
DW_API dw_status surr_set_features(dw_surr h, const float *feats, dw_stream stream);
/* Copy the current BF16 features [n^3][16] out. */
DW_API dw_status surr_get_features(dw_surr h, void *feats_bf16, dw_stream stream);
/* Network forward; with keep_activations != 0 keeps what surr_backward
 * needs (training), otherwise stores only the layer outputs (inference);
 * copies the FP32 output [n^3][16] to out when out is not NULL. */
DW_API dw_status surr_forward(dw_surr h, float *out, int32_t keep_activations, dw_stream stream);
/* Waits for `stream`, returns the first device-side error of the handle's
 * kernels since the last call (DW_ERR_TIMEOUT if a bounded wait inside a
 * convolution gave up; DW_OK if none) and clears it. */
DW_API dw_status surr_device_status(dw_surr h, dw_stream stream);
/* Mean squared error of output channels 0..2 against target [n^3][16] over the
 * coarse voxels that are not fully solid; adds the loss to *loss (device
 * float, may be NULL) and sets dL/d(output) for surr_backward. */
DW_API dw_status surr_loss(dw_surr h, const float *target, float *loss, dw_stream stream);
/* Set dL/d(output) [n^3][16] directly (FP32, rounded to BF16). */
DW_API dw_status surr_set_output_grad(dw_surr h, const float *g_out, dw_stream stream);
/* Reverse pass of the last surr_forward; accumulates into the gradients. */
DW_API dw_status surr_backward(dw_surr h, dw_stream stream);

/* One layer's weight and bias gradients from given operands, the step that
 * surr_backward runs for each layer: gw[27][cout][cin] += sum over voxels v
 * of g[v][co] in[v + d(tap)][ci] (zero padding; tap = 9 (dz + 1) + 3 (dy + 1)
 * + (dx + 1)) and gb[cout] += sum_v g[v][co]. in (cin channels) and g (cout
 * channels) are device BF16 volumes of the handle's n^3 coarse voxels in the
 * planar layout [C/8][n^3][8]; gw and gb are device FP32. (cin, cout) must be
 * a layer shape of the network: (16, 32), (32, 32) or (32, 16). impl 0 runs
 * the tcgen05 kernel surr_backward uses (TMA-loaded operands, FP32 sums in
 * tensor memory), impl 1 the warp-level mma.sync kernel it replaced; the two
 * agree up to the order of the FP32 sums. Uses the handle's partial-sum
 * workspace (calls on one handle must not overlap). */
DW_API dw_status surr_weight_grad(dw_surr h, int32_t cin, int32_t cout, const void *in,
                                  const void *g, float *gw, float *gb, int32_t impl,
                                  dw_stream stream);
/* Adam step (bias-corrected, step >= 1) on the parameters; zeroes the
 * gradients and refreshes the BF16 weights. */
DW_API dw_status surr_adam(dw_surr h, float lr, float beta1, float beta2, float eps, int32_t step,
                           dw_stream stream);
/* f = f_eq(rho, u + du) on the fluid cells of the shifted (2n)^3 lattice, with
 * rho, u from the last surr_features and du = out_scale times the output
 * channels 0..2 (out [n^3][16], or the handle's last forward output when NULL)
 * upsampled trilinearly from the cell-centred coarse grid (fine cell i at
 * coarse coordinate i/2 - 1/4, clamped). Solid cells are not written. */
DW_API dw_status surr_apply(dw_surr h, const float *out, float out_scale, const uint8_t *solid,
                            float *f, dw_stream stream);
/* Chained mode: the handle's fine (rho, u) state stands in for the lattice
 * between surrogate calls. surr_features_fine takes the coarse features from
 * it; surr_advance_fine adds out_scale times the upsampled output to its u
 * and then takes the coarse features of the updated state (scaled by
 * in_scale, exactly as surr_features_fine would), so that chained calls
 * alternate surr_forward and surr_advance_fine; surr_write_lattice
 * re-initialises f = f_eq(rho, u) on the fluid cells, and
 * surr_fine_velocity_error adds sum |u_fine - u(f)|^2 and sum |u(f)|^2 over
 * the fluid cells to sums (device double[2]). */
DW_API dw_status surr_features_fine(dw_surr h, const uint8_t *solid, float in_scale,
                                    dw_stream stream);
DW_API dw_status surr_advance_fine(dw_surr h, float out_scale, const uint8_t *solid,
                                   float in_scale, dw_stream stream);
DW_API dw_status surr_write_lattice(dw_surr h, const uint8_t *solid, float *f, dw_stream stream);
DW_API dw_status surr_fine_velocity_error(dw_surr h, const float *f, const uint8_t *solid,
                                          double *sums, dw_stream stream);
/* Defect correction of the chained mode (not in the paper; the plain LBM
 * judges the surrogate, and its judgement is reused): mode 1 sets
 * corr = u(f) - u_fine on the fluid cells (0 on solid cells), where f is the
 * shifted lattice the plain LBM reached from the state the surrogate started
 * from and u_fine the handle's fine velocity after the surrogate's block;
 * mode 2 adds that difference to the current correction; mode 0 stops using
 * it. While a correction is set, every surr_advance_fine adds corr to the
 * fine velocity after the network's update, so that a slowly varying error
 * of the network per block is cancelled instead of accumulated. The
 * correction buffer (3 (2n)^3 floats) is allocated by the first call with
 * mode 1. Errors: DW_ERR_ARG for a bad mode, mode 2 without a correction, or
 * a NULL f with mode 1 or 2. */
DW_API dw_status surr_set_correction(dw_surr h, const float *f, const uint8_t *solid, int32_t mode,
                                     dw_stream stream);
/* sums[0] += sum |u_a - u_b|^2, sums[1] += sum |u_b|^2 over the fluid cells of
 * two shifted lattices with ncell cells (device double[2]). */
DW_API dw_status lbm_velocity_error(const float *fa, const float *fb, const uint8_t *solid,
                                    int64_t ncell, double *sums, dw_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* DIFFWIND_H */

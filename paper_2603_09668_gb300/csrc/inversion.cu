// Pieces of the wind inversion loop around the MPM adjoint: the
// physics-informed loss of Sec. 3.4 (the force component across the LBM flow
// direction, squared, per wind-grid node), the aerodynamic drag relation of
// Sec. 3.4 that turns an LBM velocity into a wind force, a squared-distance
// loss on particle positions (the trajectory term), and an Adam step for the
// per-keyframe optimisation of the wind force field (Sec. 3.3).
#include <math.h>

#include "common.cuh"

namespace dw {

constexpr int PHYS_THREADS = 256;

// Block sum of one float per thread into *out (one atomic per block).
__device__ __forceinline__ void block_atomic_sum(float term, float *out) {
    __shared__ float red[PHYS_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = term;
    __syncthreads();
    if (wid == 0) {
        float sum = lane < PHYS_THREADS / 32 ? red[lane] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) atomicAdd(out, sum);
    }
    __syncthreads();  // red is reused by the next call
}

// One thread per node: r = F - (F.d) d with d = u / |u| (no term where
// |u| <= eps); loss += weight |r|^2 with one atomic per block,
// g_values += 2 weight r.
__global__ void __launch_bounds__(PHYS_THREADS) k_wind_phys_loss(
    const float *__restrict__ values, const float *__restrict__ guide_u, int64_t n, float eps,
    float weight, float *__restrict__ loss, float *__restrict__ g_values) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float term = 0.0f;
    if (k < n) {
        const float u0 = guide_u[k], u1 = guide_u[n + k], u2 = guide_u[2 * n + k];
        const float norm = sqrtf(u0 * u0 + u1 * u1 + u2 * u2);
        if (norm > eps) {
            const float d0 = u0 / norm, d1 = u1 / norm, d2 = u2 / norm;
            const float F0 = values[3 * k], F1 = values[3 * k + 1], F2 = values[3 * k + 2];
            const float fd = F0 * d0 + F1 * d1 + F2 * d2;
            const float r0 = F0 - fd * d0, r1 = F1 - fd * d1, r2 = F2 - fd * d2;
            term = r0 * r0 + r1 * r1 + r2 * r2;
            if (g_values) {
                const float w2 = 2.0f * weight;
                g_values[3 * k] += w2 * r0;
                g_values[3 * k + 1] += w2 * r1;
                g_values[3 * k + 2] += w2 * r2;
            }
        }
    }
    block_atomic_sum(weight * term, loss);
}

// One thread per particle: loss += weight |x - x*|^2, g_x += 2 weight (x - x*).
__global__ void __launch_bounds__(PHYS_THREADS) k_position_loss(
    const float *__restrict__ x, const float *__restrict__ x_target, int64_t n, float weight,
    float *__restrict__ loss, float *__restrict__ g_x) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float term = 0.0f;
    if (p < n) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = x[c * n + p] - x_target[c * n + p];
            term += d * d;
            if (g_x) g_x[c * n + p] += 2.0f * weight * d;
        }
    }
    block_atomic_sum(weight * term, loss);
}

// One thread per node: values[k] = scale |u_k| u_k (u is [3][n], values [n][3]).
__global__ void k_wind_drag_force(const float *__restrict__ u, int64_t n, float scale,
                                  float *__restrict__ values) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float u0 = u[k], u1 = u[n + k], u2 = u[2 * n + k];
    const float s = scale * sqrtf(u0 * u0 + u1 * u1 + u2 * u2);
    values[3 * k] = s * u0;
    values[3 * k + 1] = s * u1;
    values[3 * k + 2] = s * u2;
}

// One thread per location: where both forces have a direction (|.| > eps),
// sums[0] += a^.b^, sums[1] += |a^ - b^|^2, sums[2] += 1.
__global__ void __launch_bounds__(PHYS_THREADS) k_wind_field_scores(
    const float *__restrict__ rec, const float *__restrict__ gt, int64_t n, float eps,
    float *__restrict__ sums) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float cs = 0.0f, sq = 0.0f, cnt = 0.0f;
    if (k < n) {
        const float a0 = rec[3 * k], a1 = rec[3 * k + 1], a2 = rec[3 * k + 2];
        const float b0 = gt[3 * k], b1 = gt[3 * k + 1], b2 = gt[3 * k + 2];
        const float na = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
        const float nb = sqrtf(b0 * b0 + b1 * b1 + b2 * b2);
        if (na > eps && nb > eps) {
            const float e0 = a0 / na - b0 / nb, e1 = a1 / na - b1 / nb, e2 = a2 / na - b2 / nb;
            cs = (a0 * b0 + a1 * b1 + a2 * b2) / (na * nb);
            sq = e0 * e0 + e1 * e1 + e2 * e2;
            cnt = 1.0f;
        }
    }
    block_atomic_sum(cs, sums);
    block_atomic_sum(sq, sums + 1);
    block_atomic_sum(cnt, sums + 2);
}

__global__ void k_adam_step(float *__restrict__ param, const float *__restrict__ grad,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                            float beta1, float beta2, float eps, float bc1, float bc2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = grad[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * g;
    const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    param[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// VectorAdam (Ling, Sharp and Jacobson, 2022): one thread per 3-vector; the
// first moment per component, the second moment on the squared norm of the
// vector's gradient, so the step keeps the gradient's direction per node.
__global__ void k_vector_adam_step(float *__restrict__ param, const float *__restrict__ grad,
                                   float *__restrict__ m, float *__restrict__ v, int64_t n,
                                   float lr, float beta1, float beta2, float eps, float bc1,
                                   float bc2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g0 = grad[3 * i], g1 = grad[3 * i + 1], g2 = grad[3 * i + 2];
    const float vi = beta2 * v[i] + (1.0f - beta2) * (g0 * g0 + g1 * g1 + g2 * g2);
    v[i] = vi;
    const float step = lr / (bc1 * (sqrtf(vi / bc2) + eps));
    const float gs[3] = {g0, g1, g2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float mi = beta1 * m[3 * i + c] + (1.0f - beta1) * gs[c];
        m[3 * i + c] = mi;
        param[3 * i + c] -= step * mi;
    }
}

}  // namespace dw

using namespace dw;

extern "C" dw_status wind_phys_loss(const float *values, const float *guide_u, int64_t n,
                                    float eps, float weight, float *loss, float *g_values,
                                    dw_stream stream) {
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(values && guide_u && loss, "values, guide_u and loss must not be NULL");
    DW_REQUIRE(eps >= 0.0f, "eps must be >= 0");
    k_wind_phys_loss<<<grid_for(n, PHYS_THREADS), PHYS_THREADS, 0, as_stream(stream)>>>(
        values, guide_u, n, eps, weight, loss, g_values);
    DW_LAUNCHED("k_wind_phys_loss");
    return DW_OK;
}

extern "C" dw_status position_loss(const float *x, const float *x_target, int64_t n,
                                   float weight, float *loss, float *g_x, dw_stream stream) {
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(x && x_target && loss, "x, x_target and loss must not be NULL");
    k_position_loss<<<grid_for(n, PHYS_THREADS), PHYS_THREADS, 0, as_stream(stream)>>>(
        x, x_target, n, weight, loss, g_x);
    DW_LAUNCHED("k_position_loss");
    return DW_OK;
}

extern "C" dw_status wind_drag_force(const float *u, int64_t n, float scale, float *values,
                                     dw_stream stream) {
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(u && values, "u and values must not be NULL");
    k_wind_drag_force<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(u, n, scale, values);
    DW_LAUNCHED("k_wind_drag_force");
    return DW_OK;
}

extern "C" dw_status wind_field_scores(const float *rec, const float *gt, int64_t n, float eps,
                                       float *sums, dw_stream stream) {
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(rec && gt && sums, "rec, gt and sums must not be NULL");
    DW_REQUIRE(eps >= 0.0f, "eps must be >= 0");
    k_wind_field_scores<<<grid_for(n, PHYS_THREADS), PHYS_THREADS, 0, as_stream(stream)>>>(
        rec, gt, n, eps, sums);
    DW_LAUNCHED("k_wind_field_scores");
    return DW_OK;
}

extern "C" dw_status adam_step(float *param, const float *grad, float *m, float *v, int64_t n,
                               float lr, float beta1, float beta2, float eps, int32_t step,
                               dw_stream stream) {
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(param && grad && m && v, "param, grad, m and v must not be NULL");
    DW_REQUIRE(step >= 1, "step must be >= 1");
    DW_REQUIRE(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f,
               "betas must be in [0, 1)");
    const float bc1 = 1.0f - (float)pow((double)beta1, (double)step);
    const float bc2 = 1.0f - (float)pow((double)beta2, (double)step);
    k_adam_step<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(param, grad, m, v, n, lr, beta1,
                                                                  beta2, eps, bc1, bc2);
    DW_LAUNCHED("k_adam_step");
    return DW_OK;
}

extern "C" dw_status vector_adam_step(float *param, const float *grad, float *m, float *v,
                                      int64_t n, float lr, float beta1, float beta2, float eps,
                                      int32_t step, dw_stream stream) {
    DW_REQUIRE(n >= 0, "n must be >= 0");
    if (n == 0) return DW_OK;
    DW_REQUIRE(param && grad && m && v, "param, grad, m and v must not be NULL");
    DW_REQUIRE(step >= 1, "step must be >= 1");
    DW_REQUIRE(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f,
               "betas must be in [0, 1)");
    const float bc1 = 1.0f - (float)pow((double)beta1, (double)step);
    const float bc2 = 1.0f - (float)pow((double)beta2, (double)step);
    k_vector_adam_step<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(param, grad, m, v, n, lr,
                                                                         beta1, beta2, eps, bc1,
                                                                         bc2);
    DW_LAUNCHED("k_vector_adam_step");
    return DW_OK;
}

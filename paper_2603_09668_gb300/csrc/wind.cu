// wind_field_sample / wind_field_sample_adjoint: standalone sampling of the
// wind force field at arbitrary positions and its transpose.
#include "wind.cuh"

namespace dw {

dw_status wind_check(const dw_wind_field *w, WindDev *out) {
    DW_REQUIRE(w != nullptr, "wind field is NULL");
    DW_REQUIRE(w->values != nullptr, "wind field values are NULL");
    DW_REQUIRE(w->nf >= 1 && w->nf <= 1024, "wind nf=%d out of range [1, 1024]", w->nf);
    DW_REQUIRE(w->n_frames >= 1, "wind n_frames=%d must be >= 1", w->n_frames);
    DW_REQUIRE(w->n_frames == 1 || w->t_total > 0.0f, "wind t_total must be > 0 with several keyframes");
    DW_REQUIRE((int64_t)w->n_frames * w->nf * w->nf * w->nf < (1ll << 31) / 3,
               "wind field too large");
    out->values = w->values;
    out->nf = w->nf;
    out->n_frames = w->n_frames;
    out->t_total = w->t_total;
    return DW_OK;
}

__global__ void wind_sample_kernel(WindDev w, const float *__restrict__ pos, int64_t n, float t,
                                   float *__restrict__ out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float3 a = wind_sample_dev(w, pos[p], pos[n + p], pos[2 * n + p], t);
    out[p] = a.x;
    out[n + p] = a.y;
    out[2 * n + p] = a.z;
}

__global__ void wind_sample_adjoint_kernel(WindDev w, const float *__restrict__ pos, int64_t n,
                                           float t, const float *__restrict__ g_out,
                                           float *__restrict__ g_values) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float3 g = make_float3(g_out[p], g_out[n + p], g_out[2 * n + p]);
    wind_sample_adjoint_dev(w, pos[p], pos[n + p], pos[2 * n + p], t, g, g_values);
}

}  // namespace dw

using namespace dw;

extern "C" dw_status wind_field_sample(const dw_wind_field *w, const float *pos, int64_t n,
                                       float t, float *out, dw_stream stream) {
    WindDev wd;
    dw_status st = wind_check(w, &wd);
    if (st != DW_OK) return st;
    DW_REQUIRE(n >= 0, "n=%lld must be >= 0", (long long)n);
    if (n == 0) return DW_OK;
    DW_REQUIRE(pos && out, "pos/out must not be NULL");
    wind_sample_kernel<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(wd, pos, n, t, out);
    DW_LAUNCHED("wind_sample_kernel");
    return DW_OK;
}

extern "C" dw_status wind_field_sample_adjoint(const dw_wind_field *w, const float *pos,
                                               int64_t n, float t, const float *g_out,
                                               float *g_values, dw_stream stream) {
    WindDev wd;
    dw_status st = wind_check(w, &wd);
    if (st != DW_OK) return st;
    DW_REQUIRE(n >= 0, "n=%lld must be >= 0", (long long)n);
    if (n == 0) return DW_OK;
    DW_REQUIRE(pos && g_out && g_values, "pos/g_out/g_values must not be NULL");
    wind_sample_adjoint_kernel<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(wd, pos, n, t,
                                                                                g_out, g_values);
    DW_LAUNCHED("wind_sample_adjoint_kernel");
    return DW_OK;
}

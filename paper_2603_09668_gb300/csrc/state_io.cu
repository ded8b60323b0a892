// Host checkpoints of an MPM state (mpm_state_save / mpm_state_peek /
// mpm_state_load): a rollout or an inversion resumed in another process
// starts from the saved particles, time and substep counter.
//
// File: the 8-byte tag "DWMPMST1", int64 n, float64 t, int64 substep, int32
// flags (bit 0: pinned present, bit 1: ids present), int32 zero, then the
// float32 rows x[3][n], v[3][n], C[9][n], F[9][n], then uint8 pinned[n] and
// int32 ids[n] when present; little-endian, as the host writes it. A save
// goes to `path` + ".tmp" first and is renamed over `path` only when it is
// complete, so an interrupted save leaves the previous checkpoint intact.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace dw {

static const char STATE_TAG[8] = {'D', 'W', 'M', 'P', 'M', 'S', 'T', '1'};

struct StateHeader {
    char tag[8];
    int64_t n;
    double t;
    int64_t substep;
    int32_t flags;
    int32_t zero;
};
static_assert(sizeof(StateHeader) == 40, "unexpected header layout");

static dw_status io_error(const char *what, const char *path) {
    set_error("%s: %s", what, path);
    return DW_ERR_IO;
}

static dw_status read_header(FILE *f, const char *path, StateHeader *hd) {
    if (fread(hd, sizeof *hd, 1, f) != 1) return io_error("not an MPM state file (short header)", path);
    if (memcmp(hd->tag, STATE_TAG, sizeof STATE_TAG) != 0)
        return io_error("not an MPM state file (tag)", path);
    if (hd->n < 0 || (hd->flags & ~3) != 0 || hd->zero != 0)
        return io_error("not an MPM state file (header fields)", path);
    return DW_OK;
}

// The 24 float rows of a state, as (device pointer, floats) in file order.
static void rows_of(const dw_mpm_state *s, float *ptr[4], int64_t cnt[4]) {
    ptr[0] = s->x;
    ptr[1] = s->v;
    ptr[2] = s->C;
    ptr[3] = s->F;
    cnt[0] = 3 * s->n;
    cnt[1] = 3 * s->n;
    cnt[2] = 9 * s->n;
    cnt[3] = 9 * s->n;
}

}  // namespace dw

using namespace dw;

extern "C" dw_status mpm_state_save(const char *path, const dw_mpm_state *state,
                                    const uint8_t *pinned, const int32_t *ids, double t,
                                    int64_t substep, dw_stream stream) {
    DW_REQUIRE(path && path[0], "path must be given");
    DW_REQUIRE(state && state->x && state->v && state->C && state->F, "state arrays must not be NULL");
    DW_REQUIRE(state->n >= 0, "state has n < 0");
    const int64_t n = state->n;
    cudaStream_t s = as_stream(stream);
    // the whole state in one host buffer, copied from the device on `stream`
    std::vector<float> buf;
    std::vector<uint8_t> pin;
    std::vector<int32_t> id;
    try {
        buf.resize((size_t)24 * (size_t)n);
        if (pinned) pin.resize((size_t)n);
        if (ids) id.resize((size_t)n);
    } catch (...) {
        set_error("out of host memory for a state of %lld particles", (long long)n);
        return DW_ERR_OOM;
    }
    float *ptr[4];
    int64_t cnt[4];
    rows_of(state, ptr, cnt);
    size_t off = 0;
    for (int r = 0; r < 4; ++r) {
        if (cnt[r] > 0)
            DW_CUDA(cudaMemcpyAsync(buf.data() + off, ptr[r], sizeof(float) * (size_t)cnt[r],
                                    cudaMemcpyDeviceToHost, s));
        off += (size_t)cnt[r];
    }
    if (pinned && n > 0)
        DW_CUDA(cudaMemcpyAsync(pin.data(), pinned, (size_t)n, cudaMemcpyDeviceToHost, s));
    if (ids && n > 0)
        DW_CUDA(cudaMemcpyAsync(id.data(), ids, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
    DW_CUDA(cudaStreamSynchronize(s));

    StateHeader hd;
    memcpy(hd.tag, STATE_TAG, sizeof STATE_TAG);
    hd.n = n;
    hd.t = t;
    hd.substep = substep;
    hd.flags = (pinned ? 1 : 0) | (ids ? 2 : 0);
    hd.zero = 0;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return io_error("cannot open for writing", tmp.c_str());
    bool ok = fwrite(&hd, sizeof hd, 1, f) == 1;
    if (ok && n > 0) ok = fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    if (ok && pinned && n > 0) ok = fwrite(pin.data(), 1, pin.size(), f) == pin.size();
    if (ok && ids && n > 0) ok = fwrite(id.data(), sizeof(int32_t), id.size(), f) == id.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        remove(tmp.c_str());
        return io_error("write failed", tmp.c_str());
    }
    if (rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return io_error("cannot rename the finished checkpoint to", path);
    }
    return DW_OK;
}

extern "C" dw_status mpm_state_peek(const char *path, int64_t *n, int32_t *flags, double *t,
                                    int64_t *substep) {
    DW_REQUIRE(path && path[0], "path must be given");
    FILE *f = fopen(path, "rb");
    if (!f) return io_error("cannot open", path);
    StateHeader hd;
    dw_status st = read_header(f, path, &hd);
    fclose(f);
    if (st != DW_OK) return st;
    if (n) *n = hd.n;
    if (flags) *flags = hd.flags;
    if (t) *t = hd.t;
    if (substep) *substep = hd.substep;
    return DW_OK;
}

extern "C" dw_status mpm_state_load(const char *path, const dw_mpm_state *state, uint8_t *pinned,
                                    int32_t *ids, double *t, int64_t *substep, dw_stream stream) {
    DW_REQUIRE(path && path[0], "path must be given");
    DW_REQUIRE(state && state->x && state->v && state->C && state->F, "state arrays must not be NULL");
    FILE *f = fopen(path, "rb");
    if (!f) return io_error("cannot open", path);
    StateHeader hd;
    dw_status st = read_header(f, path, &hd);
    if (st != DW_OK) {
        fclose(f);
        return st;
    }
    if (hd.n != state->n) {
        fclose(f);
        set_error("the checkpoint holds %lld particles, the state %lld", (long long)hd.n,
                  (long long)state->n);
        return DW_ERR_ARG;
    }
    if ((pinned && !(hd.flags & 1)) || (ids && !(hd.flags & 2))) {
        fclose(f);
        set_error("the checkpoint has no %s array", pinned && !(hd.flags & 1) ? "pinned" : "ids");
        return DW_ERR_ARG;
    }
    const int64_t n = hd.n;
    std::vector<float> buf;
    std::vector<uint8_t> pin;
    std::vector<int32_t> id;
    try {
        buf.resize((size_t)24 * (size_t)n);
        if (hd.flags & 1) pin.resize((size_t)n);
        if (hd.flags & 2) id.resize((size_t)n);
    } catch (...) {
        fclose(f);
        set_error("out of host memory for a state of %lld particles", (long long)n);
        return DW_ERR_OOM;
    }
    bool ok = n == 0 || fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    if (ok && (hd.flags & 1) && n > 0) ok = fread(pin.data(), 1, pin.size(), f) == pin.size();
    if (ok && (hd.flags & 2) && n > 0) ok = fread(id.data(), sizeof(int32_t), id.size(), f) == id.size();
    if (ok) ok = fgetc(f) == EOF;  // nothing after the last array
    fclose(f);
    if (!ok) return io_error("truncated or oversized MPM state file", path);
    cudaStream_t s = as_stream(stream);
    float *ptr[4];
    int64_t cnt[4];
    rows_of(state, ptr, cnt);
    size_t off = 0;
    for (int r = 0; r < 4; ++r) {
        if (cnt[r] > 0)
            DW_CUDA(cudaMemcpyAsync(ptr[r], buf.data() + off, sizeof(float) * (size_t)cnt[r],
                                    cudaMemcpyHostToDevice, s));
        off += (size_t)cnt[r];
    }
    if (pinned && n > 0)
        DW_CUDA(cudaMemcpyAsync(pinned, pin.data(), (size_t)n, cudaMemcpyHostToDevice, s));
    if (ids && n > 0)
        DW_CUDA(cudaMemcpyAsync(ids, id.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    DW_CUDA(cudaStreamSynchronize(s));  // the host buffers go out of scope
    if (t) *t = hd.t;
    if (substep) *substep = hd.substep;
    return DW_OK;
}

// rs_ctx.cu -- context, workspace, status reporting and launch accounting.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "rs_internal.cuh"

extern "C" void rs_params_default(rs_params *p)
{
    if (!p) return;
    p->b = 0.28;
    p->f = 0.7;
    p->min_n = 10;
    p->delta_vir = 360.0;
    p->nbar = 0.0;
    p->merge_thresh = 10.0 * std::sqrt(2.0);
    p->nn_subset = 0;
    p->nn_seed = 0;
}

namespace {

// One thread waits, at most `limit` polls, for a flag that it sets itself
// only when `set` is nonzero; running out records a timeout in the status
// word, as every bounded wait of the library does.
__global__ void k_wait_flag(int *flag, int set, int64_t limit, rs_dev_status *st)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (set) atomicExch(flag, 1);
    volatile int *f = flag;
    for (int64_t i = 0; i < limit; i++) {
        if (*f) return;
        __nanosleep(64);
    }
    dev_fail(st, DEV_TIMEOUT, 90, limit);
}

}  // namespace

extern "C" rs_status rs_selftest_wait(rs_ctx *ctx, int32_t set_flag, int64_t limit)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    if (limit < 1 || limit > ((int64_t)1 << 24))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_selftest_wait: limit must be in [1, 2^24]");
    RS_WS(ctx, int, flag, WS_SELFTEST, 4);
    RS_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    RS_LAUNCH(ctx, "selftest_wait", k_wait_flag, 1, 32, 0, flag, (int)(set_flag != 0), limit, ctx->d_status);
    return rs_sync_check(ctx, "rs_selftest_wait");
}

extern "C" double rs_linking_length(int64_t n, double box, double b)
{
    if (n <= 0) return 0.0;
    return b * std::cbrt(box * box * box / (double)n);
}

extern "C" const char *rs_status_string(rs_status s)
{
    switch (s) {
    case RS_OK: return "ok";
    case RS_ERR_INVALID_ARG: return "invalid argument";
    case RS_ERR_CUDA: return "CUDA error";
    case RS_ERR_OOM: return "out of device memory";
    case RS_ERR_TIMEOUT: return "bounded device wait ran out";
    case RS_ERR_TOO_LARGE: return "input too large";
    case RS_ERR_INTERNAL: return "internal capacity or consistency check failed";
    case RS_ERR_EXTENT: return "a group spans half the box or more";
    }
    return "unknown status";
}

rs_status rs_fail(rs_ctx *ctx, rs_status s, const std::string &msg)
{
    if (ctx) ctx->last_error = msg;
    return s;
}

rs_status rs_cuda_fail(rs_ctx *ctx, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return rs_fail(ctx, e == cudaErrorMemoryAllocation ? RS_ERR_OOM : RS_ERR_CUDA, m);
}

extern "C" void rs_tuning_default(rs_tuning *t)
{
    if (!t) return;
    t->link_blocks_per_sm = 5;
    t->nn_blocks_per_sm = 6;
    t->kd_levels = 3;
    t->bracket_min = 4096;
    t->mid_max = 256;
    t->tiny_max = 32;
    t->small_ctas_per_sm = 2;
    t->mid_ctas_per_sm = 8;
    t->tiny_ctas_per_sm = 8;
    t->fof_link_ctas_per_sm = 32;
}

extern "C" rs_status rs_set_tuning(rs_ctx *c, const rs_tuning *t)
{
    if (!c || !t) return RS_ERR_INVALID_ARG;
    auto in = [](int32_t v, int32_t lo, int32_t hi) { return v >= lo && v <= hi; };
    if (!in(t->link_blocks_per_sm, 4, 6) || !in(t->nn_blocks_per_sm, 5, 7) || !in(t->kd_levels, 0, 3) ||
        !in(t->bracket_min, 1024, 1 << 30) || !in(t->mid_max, 33, 256) || !in(t->tiny_max, 10, 32) ||
        !in(t->small_ctas_per_sm, 1, 2) || !in(t->mid_ctas_per_sm, 1, 8) || !in(t->tiny_ctas_per_sm, 1, 16) ||
        !in(t->fof_link_ctas_per_sm, 1, 64))
        return rs_fail(c, RS_ERR_INVALID_ARG, "rs_set_tuning: a field is outside its range");
    c->tune = *t;
    return RS_OK;
}

extern "C" rs_status rs_get_tuning(const rs_ctx *c, rs_tuning *t)
{
    if (!c || !t) return RS_ERR_INVALID_ARG;
    *t = c->tune;
    return RS_OK;
}

extern "C" rs_status rs_create(rs_ctx **out, void *cuda_stream)
{
    if (!out) return RS_ERR_INVALID_ARG;
    *out = nullptr;
    rs_ctx *c = new (std::nothrow) rs_ctx();
    if (!c) return RS_ERR_OOM;
    c->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(rs_dev_status));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_status, sizeof(rs_dev_status));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_scratch, 64 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(rs_dev_status), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        rs_destroy(c);
        return e == cudaErrorMemoryAllocation ? RS_ERR_OOM : RS_ERR_CUDA;
    }
    *out = c;
    return RS_OK;
}

extern "C" void rs_destroy(rs_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (int i = 0; i < WS_NUM_SLOTS; i++)
        if (c->ws_ptr[i]) cudaFree(c->ws_ptr[i]);
    if (c->d_status) cudaFree(c->d_status);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_scratch) cudaFreeHost(c->h_scratch);
    for (auto &r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->ev_free) cudaEventDestroy(e);
    for (auto e : c->ev_io)
        if (e) cudaEventDestroy(e);
    if (c->aux) {
        cudaStreamSynchronize(c->aux);
        cudaStreamDestroy(c->aux);
    }
    delete c;
}

extern "C" rs_status rs_set_stream(rs_ctx *c, void *s)
{
    if (!c) return RS_ERR_INVALID_ARG;
    c->stream = (cudaStream_t)s;
    return RS_OK;
}

extern "C" const char *rs_last_error(const rs_ctx *c)
{
    if (!c) return "null context";
    return c->last_error.c_str();
}

bool rs_fault(const char *site)
{
    const char *v = getenv("RS_FAULT");
    if (!v || !*v) return false;
    const size_t k = strlen(site);
    for (const char *p = v; *p;) {
        const char *e = strchr(p, ',');
        const size_t len = e ? (size_t)(e - p) : strlen(p);
        if (len == k && strncmp(p, site, k) == 0) return true;
        if (!e) break;
        p = e + 1;
    }
    return false;
}

// Frees the 3D FOF and group-sort slots whose call is not running (their
// contents are scratch of that call); true if anything was freed.
static bool release_idle_slots(rs_ctx *c, int keep)
{
    bool freed = false;
    for (int s = 0; s < WS_NUM_SLOTS; s++) {
        const bool fof = s >= WS_FOF_CELLKEY && s <= WS_FOF_ACC;
        const bool gs = s == WS_GS_COUNT || s == WS_GS_FLAG;
        if (s == keep || !c->ws_ptr[s] || !((fof && !c->in_fof) || (gs && !c->in_gs))) continue;
        if (!freed) {
            cudaStreamSynchronize(c->stream);
            if (c->aux) cudaStreamSynchronize(c->aux);
        }
        cudaFree(c->ws_ptr[s]);
        c->ws_ptr[s] = nullptr;
        c->ws_size[s] = 0;
        freed = true;
    }
    return freed;
}

size_t rs_ws_total(const rs_ctx *c)
{
    size_t t = 0;
    for (int s = 0; s < WS_NUM_SLOTS; s++) t += c->ws_size[s];
    return t;
}

void *rs_ws(rs_ctx *c, int slot, size_t bytes)
{
    if (c->ws_size[slot] >= bytes) return c->ws_ptr[slot];
    if (c->fixed_ws) {
        c->last_error = "fixed workspace slot " + std::to_string(slot) + " holds " +
                        std::to_string(c->ws_size[slot]) + " bytes, " + std::to_string(bytes) + " needed";
        return nullptr;
    }
    if (rs_fault("alloc")) {
        c->last_error = "workspace allocation of " + std::to_string(bytes) + " bytes failed (injected: RS_FAULT=alloc)";
        return nullptr;
    }
    if (c->ws_ptr[slot]) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->ws_ptr[slot]);
        c->ws_ptr[slot] = nullptr;
        c->ws_size[slot] = 0;
    }
    // a little headroom against regrowth (at most 64 MB)
    size_t want = bytes + std::min<size_t>(bytes / 8, (size_t)64 << 20) + 256;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaErrorMemoryAllocation && release_idle_slots(c, slot)) {
        cudaGetLastError();
        e = cudaMalloc(&p, want);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->last_error = "workspace allocation of " + std::to_string(want) + " bytes failed";
        return nullptr;
    }
    c->ws_ptr[slot] = p;
    c->ws_size[slot] = want;
    return p;
}

// ---------------------------------------------------------------------------
// launch accounting
// ---------------------------------------------------------------------------
static cudaEvent_t take_event(rs_ctx *c)
{
    if (!c->ev_free.empty()) {
        cudaEvent_t e = c->ev_free.back();
        c->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

int rs_prof_begin(rs_ctx *c, const char *name)
{
    if (!c->prof_on) return -1;
    int id = -1;
    for (size_t i = 0; i < c->prof_names.size(); i++)
        if (c->prof_names[i] == name) {
            id = (int)i;
            break;
        }
    if (id < 0) {
        id = (int)c->prof_names.size();
        c->prof_names.push_back(name);
    }
    rs_prof_rec r;
    r.name_id = id;
    r.a = take_event(c);
    r.b = take_event(c);
    if (!r.a || !r.b) return -1;
    cudaEventRecord(r.a, c->stream);
    c->prof_recs.push_back(r);
    return (int)c->prof_recs.size() - 1;
}

void rs_prof_end(rs_ctx *c, int rec)
{
    if (rec < 0) return;
    cudaEventRecord(c->prof_recs[rec].b, c->stream);
}

extern "C" rs_status rs_profile_enable(rs_ctx *c, int32_t on)
{
    if (!c) return RS_ERR_INVALID_ARG;
    c->prof_on = on ? 1 : 0;
    return RS_OK;
}

extern "C" void rs_profile_reset(rs_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (auto &r : c->prof_recs) {
        c->ev_free.push_back(r.a);
        c->ev_free.push_back(r.b);
    }
    c->prof_recs.clear();
    c->launches = 0;
}

extern "C" int32_t rs_profile_count(rs_ctx *c) { return c ? (int32_t)c->prof_names.size() : 0; }

extern "C" rs_status rs_profile_read(rs_ctx *c, int32_t i, const char **name, int64_t *launches, double *total_ms)
{
    if (!c || i < 0 || i >= (int32_t)c->prof_names.size()) return RS_ERR_INVALID_ARG;
    RS_CUDA(c, cudaStreamSynchronize(c->stream));
    int64_t n = 0;
    double ms = 0;
    for (auto &r : c->prof_recs)
        if (r.name_id == i) {
            float t = 0;
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms += t;
            n++;
        }
    if (name) *name = c->prof_names[i].c_str();
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    return RS_OK;
}

extern "C" int64_t rs_launch_count(const rs_ctx *c) { return c ? c->launches : 0; }

extern "C" int64_t rs_workspace_bytes(const rs_ctx *c) { return c ? (int64_t)rs_ws_total(c) : 0; }

rs_status rs_sync_check(rs_ctx *c, const char *where)
{
    RS_CUDA(c, cudaMemcpyAsync(c->h_status, c->d_status, sizeof(rs_dev_status), cudaMemcpyDeviceToHost, c->stream));
    RS_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->h_status->code != DEV_OK) {
        rs_dev_status s = *c->h_status;
        RS_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(rs_dev_status), c->stream));
        RS_CUDA(c, cudaStreamSynchronize(c->stream));
        char buf[256];
        snprintf(buf, sizeof buf, "%s: device check failed (code %d, site %d, detail %lld)", where, s.code, s.site,
                 (long long)s.detail);
        rs_status out = RS_ERR_INTERNAL;
        if (s.code == DEV_TIMEOUT) out = RS_ERR_TIMEOUT;
        else if (s.code == DEV_EXTENT) out = RS_ERR_EXTENT;
        else if (s.code == DEV_BADARG) out = RS_ERR_INVALID_ARG;
        return rs_fail(c, out, buf);
    }
    return RS_OK;
}

rs_status rs_read_i64(rs_ctx *c, const void *dsrc, int count, int64_t *dst, const char *where)
{
    RS_CUDA(c, cudaMemcpyAsync(c->h_scratch, dsrc, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, c->stream));
    RS_TRY(rs_sync_check(c, where));
    for (int i = 0; i < count; i++) dst[i] = c->h_scratch[i];
    return RS_OK;
}

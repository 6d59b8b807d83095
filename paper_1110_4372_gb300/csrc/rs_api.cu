// rs_api.cu -- the whole path behind one call (rs_find_halos).
#include <algorithm>

#include "rs_refine.cuh"

// Copies `bytes` (a multiple of 4) between device memory and a host buffer
// the device can address in place (mapped pinned memory): 16-byte words for
// the bulk, 4-byte words for the tail.  Used for the positions and the halo
// ids of a host-buffer call: after the refinement's kernels a copy-engine
// transfer of a large pinned buffer runs at about 15-30 GB/s for its first
// gigabytes on GB300, while this many-SM copy keeps about 200 GB/s.  The
// same holds for the velocities, which the second stream copies while the 3D
// FOF runs.
__global__ void k_mapped_copy(const float4 *__restrict__ src, float4 *__restrict__ dst, int64_t n16,
                              const unsigned *__restrict__ src_tail, unsigned *__restrict__ dst_tail, int tail4)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
    if (blockIdx.x == 0 && (int)threadIdx.x < tail4) dst_tail[threadIdx.x] = src_tail[threadIdx.x];
}

// The device address of a mapped pinned host buffer, or nullptr.
static const void *mapped_address(const void *host)
{
    cudaPointerAttributes a{};
    const bool mapped = cudaPointerGetAttributes(&a, host) == cudaSuccess && a.type == cudaMemoryTypeHost &&
                        a.devicePointer != nullptr;
    cudaGetLastError();  // an unregistered pointer may leave an error behind
    return mapped ? a.devicePointer : nullptr;
}

// Copy on `stream` between a host buffer and device memory (to_device says
// which way): the copy kernel (blocks_per_sm CTAs per SM) when the host
// buffer is mapped pinned memory and both ends are 16-byte aligned, else
// cudaMemcpyAsync.  (The launch is counted and, when profiling is on, timed
// like the library's other kernels; the events it records go on the
// context's stream, so it is timed only there.)
static rs_status copy_host(rs_ctx *ctx, void *dst, const void *src, size_t bytes, bool to_device,
                           cudaStream_t stream, int blocks_per_sm, const char *name)
{
    const void *host = to_device ? src : (const void *)dst;
    const char *hdev = (const char *)mapped_address(host);
    const char *s = to_device ? hdev : (const char *)src;
    char *d = to_device ? (char *)dst : (char *)hdev;
    if (hdev && ((uintptr_t)s & 15) == 0 && ((uintptr_t)d & 15) == 0 && bytes % 4 == 0) {
        const int64_t n16 = (int64_t)(bytes / 16);
        const int tail4 = (int)((bytes % 16) / 4);
        const int64_t grid =
            std::min<int64_t>(std::max<int64_t>(ceil_div(n16, 256), 1), (int64_t)ctx->num_sms * blocks_per_sm);
        const int pr = stream == ctx->stream ? rs_prof_begin(ctx, name) : -1;
        k_mapped_copy<<<(unsigned)grid, 256, 0, stream>>>((const float4 *)s, (float4 *)d, n16,
                                                          (const unsigned *)(s + 16 * n16),
                                                          (unsigned *)(d + 16 * n16), tail4);
        ctx->launches++;
        rs_prof_end(ctx, pr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return rs_cuda_fail(ctx, e, name);
        return RS_OK;
    }
    RS_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                                 stream));
    return RS_OK;
}

// The context's second stream and its three events, created on first use.
static rs_status rs_io_streams(rs_ctx *ctx)
{
    if (!ctx->aux) RS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
    for (auto &e : ctx->ev_io)
        if (!e) RS_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return RS_OK;
}

// On every return of a host-buffer call: nothing of it may still run on the
// second stream (its copies read caller buffers and the workspace).
static rs_status rs_io_drain(rs_ctx *ctx, rs_status s)
{
    if (ctx->aux) {
        cudaError_t e = cudaStreamSynchronize(ctx->aux);
        if (e != cudaSuccess && s == RS_OK) return rs_cuda_fail(ctx, e, "rs_find_halos: second stream");
    }
    return s;
}

static rs_status find_halos(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n, double box,
                            const rs_params *params, int32_t *fof_labels, int32_t *halo_id, rs_stats *stats,
                            int32_t host_buffers)
{
    const float *dpos = pos, *dvel = vel;
    const size_t in_bytes = sizeof(float) * (size_t)stride * (size_t)n;
    // With host buffers the copies overlap the kernels: positions go first on
    // the context's stream (the 3D FOF needs them), velocities on a second
    // stream while the 3D FOF and the group sort run, and the 3D labels (when
    // asked for) come back on it while the refinement runs.
    cudaEvent_t ev_vel = nullptr, ev_lab = nullptr, ev_lab_done = nullptr;
    if (host_buffers) {
        float *p = (float *)rs_ws(ctx, WS_IO_POS, in_bytes);
        float *v = (float *)rs_ws(ctx, WS_IO_VEL, in_bytes);
        if (!p || !v) return ctx->fixed_ws ? RS_ERR_INTERNAL : RS_ERR_OOM;
        RS_TRY(rs_io_streams(ctx));
        ev_vel = ctx->ev_io[0];
        ev_lab = ctx->ev_io[1];
        ev_lab_done = ctx->ev_io[2];
        const int pr = rs_prof_begin(ctx, "io_h2d_pos");
        RS_TRY(copy_host(ctx, p, pos, in_bytes, true, ctx->stream, 8, "io_h2d_kernel"));
        rs_prof_end(ctx, pr);
        // the second stream starts after everything already on the context's
        // stream (nothing may still read the velocity workspace)
        RS_CUDA(ctx, cudaEventRecord(ev_lab, ctx->stream));
        RS_CUDA(ctx, cudaStreamWaitEvent(ctx->aux, ev_lab, 0));
        // the velocities with a narrower copy kernel beside the 3D FOF's
        RS_TRY(copy_host(ctx, v, vel, in_bytes, true, ctx->aux, 2, "io_h2d_vel_kernel"));
        RS_CUDA(ctx, cudaEventRecord(ev_vel, ctx->aux));
        dpos = p;
        dvel = v;
    }
    RS_WS(ctx, int32_t, labels, WS_IO_LAB, n);
    RS_WS(ctx, int32_t, perm, WS_IO_PERM, n);
    const int64_t ocap = n / (params->min_n > 0 ? params->min_n : 1) + 2;
    RS_WS(ctx, int64_t, offsets, WS_IO_OFF, ocap);
    int32_t *hid = halo_id;
    if (host_buffers) {
        hid = (int32_t *)rs_ws(ctx, WS_IO_HID, sizeof(int32_t) * (size_t)n);
        if (!hid) return RS_ERR_OOM;
    }
    RS_TRY(rs_fof3d(ctx, dpos, stride, n, box, params->b, labels, nullptr, nullptr));
    const size_t ob = sizeof(int32_t) * (size_t)n;
    if (host_buffers && fof_labels) {
        RS_CUDA(ctx, cudaEventRecord(ev_lab, ctx->stream));
        RS_CUDA(ctx, cudaStreamWaitEvent(ctx->aux, ev_lab, 0));
        RS_CUDA(ctx, cudaMemcpyAsync(fof_labels, labels, ob, cudaMemcpyDeviceToHost, ctx->aux));
        RS_CUDA(ctx, cudaEventRecord(ev_lab_done, ctx->aux));
    }
    int64_t G = 0, M = 0;
    RS_TRY(rs_group_sort(ctx, labels, n, params->min_n, perm, offsets, ocap, &G, &M));
    if (G > 0 && rs_fault("offsets")) {
        // injected fault: a decreasing boundary, which the refinement's
        // argument check must turn into RS_ERR_INVALID_ARG
        static const int64_t bad = -1;
        RS_CUDA(ctx, cudaMemcpy(offsets + 1, &bad, sizeof(int64_t), cudaMemcpyHostToDevice));
    }
    if (host_buffers) {
        const int pr = rs_prof_begin(ctx, "io_wait_vel");
        RS_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ev_vel, 0));
        rs_prof_end(ctx, pr);
    }
    rs_tree *tree = nullptr;
    RS_TRY(rs_refine6d_sampled(ctx, dpos, dvel, stride, n, box, perm, offsets, G, params->f, params->min_n,
                               params->nn_subset, params->nn_seed, &tree));
    int64_t H = 0;
    rs_status s = rs_assign(ctx, tree, dpos, dvel, stride, n, box, params, hid, &H);
    if (s == RS_OK) {
        if (stats) {
            stats->n_fof_groups = G;
            stats->n_members = M;
            stats->n_nodes = tree->n_nodes;
            stats->n_levels = tree->n_levels;
            stats->n_seeds = tree->n_seeds;
            stats->n_halos = H;
            stats->n_tieband6d = tree->n_tieband;
            stats->sum_level_members = tree->sum_level_members;
            stats->sum_big_level_members = tree->sum_big_level_members;
            stats->n_fallback_levels = tree->n_fallback_levels;
        }
        if (host_buffers) {
            const int pr = rs_prof_begin(ctx, "io_d2h_halo");
            s = copy_host(ctx, halo_id, hid, ob, false, ctx->stream, 8, "io_d2h_kernel");
            rs_prof_end(ctx, pr);
            if (s == RS_OK && fof_labels) {
                const cudaError_t e = cudaStreamWaitEvent(ctx->stream, ev_lab_done, 0);
                if (e != cudaSuccess) s = rs_cuda_fail(ctx, e, "rs_find_halos: copy out");
            }
        } else if (fof_labels) {
            cudaError_t e = cudaMemcpyAsync(fof_labels, labels, ob, cudaMemcpyDeviceToDevice, ctx->stream);
            if (e != cudaSuccess) s = rs_cuda_fail(ctx, e, "rs_find_halos: copy labels");
        }
        if (s == RS_OK) s = rs_sync_check(ctx, "rs_find_halos");
    }
    rs_tree_free(tree);
    return s;
}

extern "C" rs_status rs_find_halos(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n,
                                   double box, const rs_params *params, int32_t *fof_labels, int32_t *halo_id,
                                   rs_stats *stats, int32_t host_buffers)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    if (!params || n < 0 || (stride != 3 && stride != 4) || (n > 0 && (!pos || !vel || !halo_id)))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_find_halos: bad argument");
    if (n >= ((int64_t)1 << 31)) return rs_fail(ctx, RS_ERR_TOO_LARGE, "rs_find_halos: n >= 2^31");
    if (stats) *stats = rs_stats{};
    if (n == 0) return RS_OK;
    RsRange range(host_buffers ? "rs_find_halos (host buffers)" : "rs_find_halos");
    const rs_status s = find_halos(ctx, pos, vel, stride, n, box, params, fof_labels, halo_id, stats, host_buffers);
    return host_buffers ? rs_io_drain(ctx, s) : s;
}

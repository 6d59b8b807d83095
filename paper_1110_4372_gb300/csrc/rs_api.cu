// rs_api.cu -- the whole path behind one call (rs_find_halos).
#include "rs_refine.cuh"

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
    const float *dpos = pos, *dvel = vel;
    const size_t in_bytes = sizeof(float) * (size_t)stride * (size_t)n;
    if (host_buffers) {
        float *p = (float *)rs_ws(ctx, WS_IO_POS, in_bytes);
        float *v = (float *)rs_ws(ctx, WS_IO_VEL, in_bytes);
        if (!p || !v) return RS_ERR_OOM;
        RS_CUDA(ctx, cudaMemcpyAsync(p, pos, in_bytes, cudaMemcpyHostToDevice, ctx->stream));
        RS_CUDA(ctx, cudaMemcpyAsync(v, vel, in_bytes, cudaMemcpyHostToDevice, ctx->stream));
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
    int64_t G = 0, M = 0;
    RS_TRY(rs_group_sort(ctx, labels, n, params->min_n, perm, offsets, ocap, &G, &M));
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
        const size_t ob = sizeof(int32_t) * (size_t)n;
        if (host_buffers) {
            cudaError_t e = cudaMemcpyAsync(halo_id, hid, ob, cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess && fof_labels)
                e = cudaMemcpyAsync(fof_labels, labels, ob, cudaMemcpyDeviceToHost, ctx->stream);
            if (e != cudaSuccess) s = rs_cuda_fail(ctx, e, "rs_find_halos: copy out");
        } else if (fof_labels) {
            cudaError_t e = cudaMemcpyAsync(fof_labels, labels, ob, cudaMemcpyDeviceToDevice, ctx->stream);
            if (e != cudaSuccess) s = rs_cuda_fail(ctx, e, "rs_find_halos: copy labels");
        }
        if (s == RS_OK) s = rs_sync_check(ctx, "rs_find_halos");
    }
    rs_tree_free(tree);
    return s;
}

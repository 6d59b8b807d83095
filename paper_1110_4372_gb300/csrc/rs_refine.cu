// rs_refine.cu -- the phase-space FOF hierarchy (Sec. 3.2, Eq. 1).
//
// Members of every refined group are gathered into member slots in group
// order, with positions unwrapped into one periodic image per group (x - box
// for coordinates in the upper half of the box, exact in float32, when the
// group straddles a face).  Nodes own nested slot ranges: a node's children
// occupy the front of its range.
//
// Two size classes:
//  * small nodes (<= SMALL_N members): one CTA loads the node into shared
//    memory and builds its whole subtree there (moments, nearest neighbours,
//    exact k-th select, union-find, children, recursion with an explicit
//    stack), as a persistent work queue over all small nodes;
//  * big nodes: processed level by level by tiles of 256 members spread over
//    the whole GPU, with per-node accumulators and histograms in global
//    memory; children above SMALL_N stay on the big path, smaller children
//    join the small-node queue.
//
// Exactness: means and dispersions come from exact fixed-point integer sums;
// nearest-neighbour and link tests run in float32 against a band of 2^-20
// (relative, on d^2) around the linking length, and everything inside the
// band is re-evaluated in float64.  The linking length itself is the exact
// float64 k-th smallest nearest-neighbour distance: the float32 k-th value
// brackets it, and only the members whose float32 distance lies within twice
// the band of it are re-evaluated in float64 and ranked.
#include <cmath>
#include <cstring>

#include "rs_refine.cuh"

namespace {

constexpr int SMALL_N = 1024;       // largest node handled by one CTA
constexpr int SMALL_THREADS = 256;
constexpr int STACK_CAP = 256;
constexpr int TQ = 256;             // big-node tile (members per CTA)

// ---------------------------------------------------------------------------
// setup: unwrap decision per group, gather into slots, root nodes
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load3(const float *a, int stride, int64_t i, float &x, float &y, float &z)
{
    const float *p = a + (int64_t)stride * i;
    x = p[0];
    y = p[1];
    z = p[2];
}

// Per group and axis: shift coordinates in the upper half of the box down by
// box if that makes the group's extent smaller than box/2 (bit a of
// shift[g]); minidx of the group.  One block per group.
__global__ void k_group_unwrap(int64_t G, const int64_t *off, const int32_t *perm, int64_t n, const float *pos,
                               int stride, float boxf, int *shift_bits, int *gmin, rs_dev_status *st)
{
    __shared__ float red12[32][12];
    __shared__ int redi[32];
    for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
        const int64_t a = off[g], b = off[g + 1];
        // minima of x and -x, unshifted and shifted, per axis
        float r[12];
        for (int k = 0; k < 12; k++) r[k] = INFINITY;
        int mn = 0x7fffffff;
        if (b < a) dev_fail(st, DEV_BADARG, 32, g);
        for (int64_t m = a + threadIdx.x; m < b; m += blockDim.x) {
            int i = perm[m];
            if (i < 0 || i >= n) {
                dev_fail(st, DEV_BADARG, 33, m);
                continue;
            }
            mn = min(mn, i);
            float c[3];
            load3(pos, stride, i, c[0], c[1], c[2]);
            for (int d = 0; d < 3; d++) {
                float s = c[d] >= 0.5f * boxf ? c[d] - boxf : c[d];
                r[d] = fminf(r[d], c[d]);
                r[3 + d] = fminf(r[3 + d], -c[d]);
                r[6 + d] = fminf(r[6 + d], s);
                r[9 + d] = fminf(r[9 + d], -s);
            }
        }
        for (int k = 0; k < 12; k++) r[k] = warp_min(r[k]);
        mn = warp_min(mn);
        if (lane_id() == 0) {
            for (int k = 0; k < 12; k++) red12[warp_id()][k] = r[k];
            redi[warp_id()] = mn;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int m2 = 0x7fffffff;
            for (int k = 0; k < 12; k++) r[k] = INFINITY;
            for (int w = 0; w < (int)(blockDim.x / 32); w++) {
                for (int k = 0; k < 12; k++) r[k] = fminf(r[k], red12[w][k]);
                m2 = min(m2, redi[w]);
            }
            int bits = 0;
            for (int d = 0; d < 3; d++) {
                float ext = -r[3 + d] - r[d];
                float exts = -r[9 + d] - r[6 + d];
                if (ext < 0.5f * boxf) {
                } else if (exts < 0.5f * boxf) {
                    bits |= 1 << d;
                } else {
                    dev_fail(st, DEV_EXTENT, 30, g);
                }
            }
            shift_bits[g] = bits;
            gmin[g] = m2;
        }
        __syncthreads();
    }
}

__global__ void k_gather(int64_t G, const int64_t *off, const int32_t *perm, int64_t n, const float *pos,
                         const float *vel, int stride, float boxf, const int *shift_bits, float4 *wpos, float4 *wvel, int *widx,
                         int *slot_group)
{
    // one block per group, grid-stride
    for (int64_t g = blockIdx.x; g < G; g += gridDim.x) {
        const int64_t a = off[g], b = off[g + 1], base = off[0];
        const int bits = shift_bits[g];
        for (int64_t m = a + threadIdx.x; m < b; m += blockDim.x) {
            int i = perm[m];
            if (i < 0 || i >= n) i = 0;  // recorded by k_group_unwrap
            float x, y, z, u, v, w;
            load3(pos, stride, i, x, y, z);
            load3(vel, stride, i, u, v, w);
            if ((bits & 1) && x >= 0.5f * boxf) x = x - boxf;
            if ((bits & 2) && y >= 0.5f * boxf) y = y - boxf;
            if ((bits & 4) && z >= 0.5f * boxf) z = z - boxf;
            wpos[m - base] = make_float4(x, y, z, 0.f);
            wvel[m - base] = make_float4(u, v, w, 0.f);
            widx[m - base] = i;
            slot_group[m - base] = (int)g;
        }
    }
}

__global__ void k_check_offsets(int64_t G, const int64_t *off, rs_dev_status *st)
{
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < G && off[g + 1] < off[g]) dev_fail(st, DEV_BADARG, 34, g);
}

__global__ void k_make_roots(int64_t G, const int64_t *off, const int *gmin, const int *shift_bits, int min_n,
                             NodeArrays nd,
                             int *big_list, int *big_len, int *small_list, int *small_len, rs_dev_status *st)
{
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    int64_t cnt = off[g + 1] - off[g];
    if (cnt < min_n) return;
    int id = atomicAdd(nd.counter, 1);
    if (id >= nd.cap) {
        dev_fail(st, DEV_OVERFLOW, 31, id);
        return;
    }
    nd.parent[id] = -1;
    nd.level[id] = 0;
    nd.first[id] = (int)(off[g] - off[0]);
    nd.count[id] = (int)cnt;
    nd.minidx[id] = gmin[g];
    nd.nchild[id] = 0;
    nd.tie[id] = 0;
    nd.root[id] = id;
    nd.shift[id] = shift_bits[g];
    if (cnt > SMALL_N) big_list[atomicAdd(big_len, 1)] = id;
    else small_list[atomicAdd(small_len, 1)] = id;
}

// ---------------------------------------------------------------------------
// small nodes: whole subtree in one CTA
// ---------------------------------------------------------------------------
struct SmallShared {
    float px[SMALL_N], py[SMALL_N], pz[SMALL_N], vx[SMALL_N], vy[SMALL_N], vz[SMALL_N];
    int idx[SMALL_N];
    float dnn[SMALL_N];
    int par[SMALL_N];
    int csize[SMALL_N];
    int cmin[SMALL_N];
    unsigned long long key[SMALL_N];
    float tp[6][SMALL_N];
    int tidx[SMALL_N];
    int4 stack[STACK_CAP];
    int sp;
    int job;
    MomAcc wacc[SMALL_THREADS / 32];
    Metric6 met;
    double l2;
    float lo32, hi32, tlo32, thi32;
    int nband, below, tie, nchild;
    int pick;
};

__device__ __forceinline__ float4 sp4(const SmallShared &S, int i)
{
    return make_float4(S.px[i], S.py[i], S.pz[i], 0.f);
}
__device__ __forceinline__ float4 sv4(const SmallShared &S, int i)
{
    return make_float4(S.vx[i], S.vy[i], S.vz[i], 0.f);
}

// in-place ascending bitonic sort of S.key[0 .. P), P a power of two
__device__ void bitonic_u64(unsigned long long *key, int P)
{
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
                int i = 2 * j * (t / j) + (t % j);
                int l = i + j;
                bool up = (i & k) == 0;
                unsigned long long a = key[i], b = key[l];
                if ((a > b) == up) {
                    key[i] = b;
                    key[l] = a;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(SMALL_THREADS, 2)
    k_small_subtree(const int *queue, const int *queue_len, int *queue_head, const float4 *wpos, const float4 *wvel,
                    int *widx, NodeArrays nd, double box, double f, int min_n, rs_dev_status *st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallShared &S = *reinterpret_cast<SmallShared *>(smem_raw);
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) S.job = atomicAdd(queue_head, 1);
        __syncthreads();
        const int job = S.job;
        __syncthreads();
        if (job >= *queue_len) break;
        const int node0 = queue[job];
        const int base = nd.first[node0];
        const int n0 = nd.count[node0];
        for (int i = tid; i < n0; i += SMALL_THREADS) {
            float4 p = wpos[base + i], v = wvel[base + i];
            S.px[i] = p.x;
            S.py[i] = p.y;
            S.pz[i] = p.z;
            S.vx[i] = v.x;
            S.vy[i] = v.y;
            S.vz[i] = v.z;
            S.idx[i] = widx[base + i];
        }
        if (tid == 0) {
            S.sp = 1;
            S.stack[0] = make_int4(0, n0, node0, nd.level[node0]);
        }
        __syncthreads();
        for (int guard = 0; guard < 1 << 20; guard++) {
            if (S.sp == 0) break;
            __syncthreads();
            int4 top;
            top = S.stack[S.sp - 1];
            __syncthreads();
            if (tid == 0) S.sp--;
            const int lf = top.x, cnt = top.y, node = top.z, lev = top.w;
            // ---- moments (exact) ----
            {
                MomRef ref = mom_ref(sp4(S, lf), sv4(S, lf));
                MomAcc a;
                mom_zero(a);
                for (int i = lf + tid; i < lf + cnt; i += SMALL_THREADS) mom_add(a, sp4(S, i), sv4(S, i), ref);
                mom_warp_reduce(a);
                if (lane_id() == 0) S.wacc[warp_id()] = a;
                __syncthreads();
                if (tid == 0) {
                    MomAcc t = S.wacc[0];
                    for (int w = 1; w < SMALL_THREADS / 32; w++) mom_merge(t, S.wacc[w]);
                    MomOut o = mom_finalize(t, sp4(S, lf), sv4(S, lf), cnt, box);
                    for (int d = 0; d < 3; d++) {
                        nd.xbar[3 * node + d] = o.xbar[d];
                        nd.vbar[3 * node + d] = o.vbar[d];
                    }
                    nd.sigx[node] = o.sigx;
                    nd.sigv[node] = o.sigv;
                    S.met = metric_of(o.sigx, o.sigv);
                    S.nband = 0;
                    S.below = 0;
                    S.tie = 0;
                    S.nchild = 0;
                }
                __syncthreads();
            }
            const Metric6 met = S.met;
            // ---- nearest neighbours (float32) ----
            for (int q = lf + tid; q < lf + cnt; q += SMALL_THREADS) {
                const float4 pq = sp4(S, q), vq = sv4(S, q);
                float best = INFINITY;
                for (int c = lf; c < lf + cnt; c++) {
                    if (c == q) continue;
                    float d2 = d2_32(pq, vq, sp4(S, c), sv4(S, c), met);
                    best = fminf(best, d2);
                }
                S.dnn[q] = best;
            }
            __syncthreads();
            // ---- k-th smallest, float32 ----
            int P = 1;
            while (P < cnt) P <<= 1;
            for (int i = tid; i < P; i += SMALL_THREADS)
                S.key[i] = i < cnt ? (unsigned long long)__float_as_uint(S.dnn[lf + i]) : ~0ull;
            __syncthreads();
            bitonic_u64(S.key, P);
            long long kk = (long long)ceil(f * (double)cnt);
            if (kk < 1) kk = 1;
            if (kk > cnt) kk = cnt;
            const float t32 = __uint_as_float((unsigned)S.key[kk - 1]);
            const float blo = (float)((double)t32 * (1.0 - 2.0 * RS_BAND));
            const float bhi = (float)((double)t32 * (1.0 + 2.0 * RS_BAND));
            __syncthreads();
            // ---- band members: exact float64 nearest-neighbour distances ----
            double *bval = reinterpret_cast<double *>(S.key);
            for (int q = lf + tid; q < lf + cnt; q += SMALL_THREADS) {
                const float dq = S.dnn[q];
                if (dq < blo) {
                    atomicAdd(&S.below, 1);
                } else if (dq <= bhi) {
                    const float4 pq = sp4(S, q), vq = sv4(S, q);
                    const float lim = dq * (float)(1.0 + 2.0 * RS_BAND);
                    double best = INFINITY;
                    for (int c = lf; c < lf + cnt; c++) {
                        if (c == q) continue;
                        const float4 pc = sp4(S, c), vc = sv4(S, c);
                        if (d2_32(pq, vq, pc, vc, met) <= lim) best = fmin(best, d2_64(pq, vq, pc, vc, met));
                    }
                    int slot = atomicAdd(&S.nband, 1);
                    bval[slot] = best;
                }
            }
            __syncthreads();
            // rank the band: the exact k-th value is the (k - 1 - below)-th
            {
                const int nb = S.nband, want = (int)(kk - 1) - S.below;
                if (want < 0 || want >= nb) {
                    if (tid == 0) dev_fail(st, DEV_INTERNAL, 40, node);
                }
                for (int b = tid; b < nb; b += SMALL_THREADS) {
                    int r = 0;
                    const double vb = bval[b];
                    for (int c = 0; c < nb; c++) r += (bval[c] < vb || (bval[c] == vb && c < b)) ? 1 : 0;
                    if (r == want) S.l2 = vb;
                }
                __syncthreads();
            }
            const double l2 = S.l2;
            if (tid == 0) {
                S.lo32 = (float)(l2 * (1.0 - RS_BAND));
                S.hi32 = (float)(l2 * (1.0 + RS_BAND));
                S.tlo32 = (float)(l2 * (1.0 - 3e-6));
                S.thi32 = (float)(l2 * (1.0 + 3e-6));
                nd.lnk[node] = sqrt(l2 / met.scale);
            }
            for (int i = lf + tid; i < lf + cnt; i += SMALL_THREADS) S.par[i] = i;
            __syncthreads();
            // ---- friends-of-friends at l (inclusive) ----
            {
                const float lo = S.lo32, hi = S.hi32, tlo = S.tlo32, thi = S.thi32;
                const float part = fmaxf(hi, thi);
                const double l = sqrt(l2);
                int tie = 0;
                for (int q = lf + tid; q < lf + cnt; q += SMALL_THREADS) {
                    if (S.dnn[q] > part) continue;
                    const float4 pq = sp4(S, q), vq = sv4(S, q);
                    for (int c = q + 1; c < lf + cnt; c++) {
                        if (S.dnn[c] > part) continue;
                        const float4 pc = sp4(S, c), vc = sv4(S, c);
                        const float d2 = d2_32(pq, vq, pc, vc, met);
                        if (d2 > part) continue;
                        bool link = d2 <= lo;
                        if (!link && (d2 <= hi || (d2 >= tlo && d2 <= thi))) {
                            const double e = d2_64(pq, vq, pc, vc, met);
                            link = e <= l2;
                            if (l2 > 0 && e != l2 && fabs(sqrt(e) - l) <= 1e-6 * l) tie++;
                        }
                        if (link) uf_union_s(S.par, q, c, st);
                    }
                }
                tie = warp_sum(tie);
                if (lane_id() == 0 && tie) atomicAdd(&S.tie, tie);
            }
            __syncthreads();
            // ---- components ----
            for (int i = lf + tid; i < lf + cnt; i += SMALL_THREADS) {
                S.csize[i] = 0;
                S.cmin[i] = 0x7fffffff;
            }
            __syncthreads();
            for (int i = lf + tid; i < lf + cnt; i += SMALL_THREADS) {
                int r = uf_find_s(S.par, i);
                S.par[i] = r;
                atomicAdd(&S.csize[r], 1);
                atomicMin(&S.cmin[r], S.idx[i]);
            }
            __syncthreads();
            // ---- children first (by smallest particle index), then the rest ----
            for (int i = tid; i < P; i += SMALL_THREADS) {
                unsigned long long k = ~0ull;
                if (i < cnt) {
                    int r = S.par[lf + i];
                    int sz = S.csize[r];
                    unsigned hiw = (sz >= min_n && sz < cnt) ? (unsigned)S.cmin[r] : 0xffffffffu;
                    k = ((unsigned long long)hiw << 32) | (unsigned)i;
                }
                S.key[i] = k;
            }
            __syncthreads();
            bitonic_u64(S.key, P);
            for (int p = tid; p < cnt; p += SMALL_THREADS) {
                int o = lf + (int)(S.key[p] & 0xffffffffu);
                S.tp[0][p] = S.px[o];
                S.tp[1][p] = S.py[o];
                S.tp[2][p] = S.pz[o];
                S.tp[3][p] = S.vx[o];
                S.tp[4][p] = S.vy[o];
                S.tp[5][p] = S.vz[o];
                S.tidx[p] = S.idx[o];
            }
            __syncthreads();
            for (int p = tid; p < cnt; p += SMALL_THREADS) {
                S.px[lf + p] = S.tp[0][p];
                S.py[lf + p] = S.tp[1][p];
                S.pz[lf + p] = S.tp[2][p];
                S.vx[lf + p] = S.tp[3][p];
                S.vy[lf + p] = S.tp[4][p];
                S.vz[lf + p] = S.tp[5][p];
                S.idx[lf + p] = S.tidx[p];
            }
            __syncthreads();
            for (int p = tid; p < cnt; p += SMALL_THREADS) {
                const unsigned hiw = (unsigned)(S.key[p] >> 32);
                if (hiw == 0xffffffffu) continue;
                if (p > 0 && (unsigned)(S.key[p - 1] >> 32) == hiw) continue;
                int e = p + 1;
                while (e < cnt && (unsigned)(S.key[e] >> 32) == hiw) e++;
                int id = atomicAdd(nd.counter, 1);
                if (id >= nd.cap) {
                    dev_fail(st, DEV_OVERFLOW, 41, id);
                    continue;
                }
                nd.parent[id] = node;
                nd.level[id] = lev + 1;
                nd.first[id] = base + lf + p;
                nd.count[id] = e - p;
                nd.minidx[id] = (int)hiw;
                nd.nchild[id] = 0;
                nd.tie[id] = 0;
                nd.root[id] = nd.root[node];
                nd.shift[id] = nd.shift[node];
                atomicAdd(&S.nchild, 1);
                int s = atomicAdd(&S.sp, 1);
                if (s >= STACK_CAP) {
                    dev_fail(st, DEV_OVERFLOW, 42, s);
                    atomicSub(&S.sp, 1);
                } else {
                    S.stack[s] = make_int4(lf + p, e - p, id, lev + 1);
                }
            }
            __syncthreads();
            if (tid == 0) {
                nd.nchild[node] = S.nchild;
                nd.tie[node] = S.tie;
            }
            __syncthreads();
        }
        for (int i = tid; i < n0; i += SMALL_THREADS) widx[base + i] = S.idx[i];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// big nodes: one level at a time
// ---------------------------------------------------------------------------
struct LevelBufs {
    const int *list;  // node ids, by rank
    int K;
    const int *tile_rank;
    const int *tile_q0;
    const int64_t *seg_off;  // member offset of each rank in the level's member list
    MomAcc *acc;
    Metric6 *met;
    float4 *ref;             // reference pos, vel per rank (2 entries)
    unsigned *hist;          // 2048 per rank
    unsigned *sel_prefix;    // per rank
    int *sel_krem;           // per rank
    int *below;              // per rank
    int *band_len;           // scalar
    int *band_rank;
    int *band_slot;
    double *band_val;
    double *l2;              // per rank
    int *tie;                // per rank
};

__global__ void k_lvl_prep(const int *list, int K, NodeArrays nd, int64_t *tiles, int64_t *segc)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int c = nd.count[list[k]];
    tiles[k] = ceil_div(c, TQ);
    segc[k] = c;
}

__global__ void k_lvl_tiles(int K, const int64_t *tile_off, int *tile_rank, int *tile_q0)
{
    int k = blockIdx.x;
    if (k >= K) return;
    int64_t a = tile_off[k], b = tile_off[k + 1];
    for (int64_t t = a + threadIdx.x; t < b; t += blockDim.x) {
        tile_rank[t] = k;
        tile_q0[t] = (int)((t - a) * TQ);
    }
}

__global__ void __launch_bounds__(TQ) k_lvl_moments(LevelBufs L, NodeArrays nd, const float4 *wpos,
                                                    const float4 *wvel)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const float4 pref = wpos[first], vref = wvel[first];
    MomRef ref = mom_ref(pref, vref);
    MomAcc a;
    mom_zero(a);
    int q = q0 + threadIdx.x;
    if (q < n) mom_add(a, wpos[first + q], wvel[first + q], ref);
    mom_warp_reduce(a);
    __shared__ MomAcc w[TQ / 32];
    if (lane_id() == 0) w[warp_id()] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        MomAcc t = w[0];
        for (int i = 1; i < TQ / 32; i++) mom_merge(t, w[i]);
        mom_atomic_add(&L.acc[k], t);
        if (q0 == 0) {
            L.ref[2 * k] = pref;
            L.ref[2 * k + 1] = vref;
        }
    }
}

__global__ void k_lvl_finalize(LevelBufs L, NodeArrays nd, double box)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.K) return;
    const int node = L.list[k];
    MomOut o = mom_finalize(L.acc[k], L.ref[2 * k], L.ref[2 * k + 1], nd.count[node], box);
    for (int d = 0; d < 3; d++) {
        nd.xbar[3 * node + d] = o.xbar[d];
        nd.vbar[3 * node + d] = o.vbar[d];
    }
    nd.sigx[node] = o.sigx;
    nd.sigv[node] = o.sigv;
    L.met[k] = metric_of(o.sigx, o.sigv);
}

// brute-force nearest neighbour over the node, candidates staged in smem
__global__ void __launch_bounds__(TQ) k_lvl_nn(LevelBufs L, NodeArrays nd, const float4 *wpos, const float4 *wvel,
                                               float *dnn)
{
    __shared__ float4 cp[TQ], cv[TQ];
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const Metric6 met = L.met[k];
    const int q = q0 + threadIdx.x;
    float4 pq = make_float4(0, 0, 0, 0), vq = pq;
    if (q < n) {
        pq = wpos[first + q];
        vq = wvel[first + q];
    }
    float best = INFINITY;
    for (int c0 = 0; c0 < n; c0 += TQ) {
        __syncthreads();
        if (c0 + threadIdx.x < n) {
            cp[threadIdx.x] = wpos[first + c0 + threadIdx.x];
            cv[threadIdx.x] = wvel[first + c0 + threadIdx.x];
        }
        __syncthreads();
        const int m = min(TQ, n - c0);
        for (int j = 0; j < m; j++) {
            if (c0 + j == q) continue;
            best = fminf(best, d2_32(pq, vq, cp[j], cv[j], met));
        }
    }
    if (q < n) dnn[first + q] = best;
}

// radix select: pass 0 digits bits 31..21, pass 1 bits 20..10, pass 2 bits 9..0
__device__ __forceinline__ void sel_digit(unsigned bits, int pass, unsigned &digit, unsigned &prefix_mask)
{
    if (pass == 0) {
        digit = bits >> 21;
        prefix_mask = 0;
    } else if (pass == 1) {
        digit = (bits >> 10) & 2047u;
        prefix_mask = 0xffe00000u;
    } else {
        digit = bits & 1023u;
        prefix_mask = 0xfffffc00u;
    }
}

__global__ void k_lvl_initk(LevelBufs L, NodeArrays nd, double f)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.K) return;
    const int n = nd.count[L.list[k]];
    long long kk = (long long)ceil(f * (double)n);
    if (kk < 1) kk = 1;
    if (kk > n) kk = n;
    L.sel_krem[k] = (int)kk;
    L.sel_prefix[k] = 0u;
}

__global__ void __launch_bounds__(TQ) k_lvl_hist(LevelBufs L, NodeArrays nd, const float *dnn, int pass)
{
    __shared__ unsigned h[2048];
    for (int i = threadIdx.x; i < 2048; i += TQ) h[i] = 0;
    __syncthreads();
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const int q = q0 + threadIdx.x;
    if (q < n) {
        unsigned bits = __float_as_uint(dnn[first + q]), digit, mask;
        sel_digit(bits, pass, digit, mask);
        if ((bits & mask) == (L.sel_prefix[k] & mask)) atomicAdd(&h[digit], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += TQ)
        if (h[i]) atomicAdd(&L.hist[(int64_t)k * 2048 + i], h[i]);
}

__global__ void k_lvl_pick(LevelBufs L, int pass)
{
    const int k = blockIdx.x;
    if (threadIdx.x != 0) return;
    unsigned *h = L.hist + (int64_t)k * 2048;
    int krem = L.sel_krem[k];
    const int nbins = pass == 2 ? 1024 : 2048;
    const int shift = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
    int acc = 0, d = 0;
    for (d = 0; d < nbins; d++) {
        if (acc + (int)h[d] >= krem) break;
        acc += (int)h[d];
    }
    if (d >= nbins) d = nbins - 1;
    L.sel_prefix[k] |= (unsigned)d << shift;
    L.sel_krem[k] = krem - acc;
    for (int i = 0; i < 2048; i++) h[i] = 0;
}

__global__ void __launch_bounds__(TQ) k_lvl_band(LevelBufs L, NodeArrays nd, const float *dnn)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const int q = q0 + threadIdx.x;
    if (q >= n) return;
    const float t32 = __uint_as_float(L.sel_prefix[k]);
    const float blo = (float)((double)t32 * (1.0 - 2.0 * RS_BAND));
    const float bhi = (float)((double)t32 * (1.0 + 2.0 * RS_BAND));
    const float d = dnn[first + q];
    if (d < blo) {
        atomicAdd(&L.below[k], 1);
    } else if (d <= bhi) {
        int b = atomicAdd(L.band_len, 1);
        L.band_rank[b] = k;
        L.band_slot[b] = first + q;
    }
}

__global__ void __launch_bounds__(TQ) k_lvl_band_exact(LevelBufs L, NodeArrays nd, const float4 *wpos,
                                                       const float4 *wvel, const float *dnn)
{
    const int b = blockIdx.x;
    const int k = L.band_rank[b], s = L.band_slot[b];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const Metric6 met = L.met[k];
    const float4 pq = wpos[s], vq = wvel[s];
    const float lim = dnn[s] * (float)(1.0 + 2.0 * RS_BAND);
    double best = INFINITY;
    for (int c = threadIdx.x; c < n; c += TQ) {
        if (first + c == s) continue;
        const float4 pc = wpos[first + c], vc = wvel[first + c];
        if (d2_32(pq, vq, pc, vc, met) <= lim) best = fmin(best, d2_64(pq, vq, pc, vc, met));
    }
    best = warp_min(best);
    __shared__ double w[TQ / 32];
    if (lane_id() == 0) w[warp_id()] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = w[0];
        for (int i = 1; i < TQ / 32; i++) m = fmin(m, w[i]);
        L.band_val[b] = m;
    }
}

__global__ void k_lvl_l2(LevelBufs L, NodeArrays nd, double f, rs_dev_status *st)
{
    const int k = blockIdx.x;
    const int node = L.list[k];
    const int n = nd.count[node];
    long long kk = (long long)ceil(f * (double)n);
    if (kk < 1) kk = 1;
    if (kk > n) kk = n;
    const int want = (int)(kk - 1) - L.below[k];
    const int nb = *L.band_len;
    bool found = false;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        if (L.band_rank[b] != k) continue;
        const double v = L.band_val[b];
        int r = 0;
        for (int c = 0; c < nb; c++)
            if (L.band_rank[c] == k && (L.band_val[c] < v || (L.band_val[c] == v && c < b))) r++;
        if (r == want) {
            L.l2[k] = v;
            found = true;
        }
    }
    found = __syncthreads_or(found);
    if (threadIdx.x == 0) {
        if (!found) dev_fail(st, DEV_INTERNAL, 50, node);
        nd.lnk[node] = sqrt(L.l2[k] / L.met[k].scale);
    }
}

__global__ void k_lvl_iota(LevelBufs L, NodeArrays nd, int *parent, int *csize, int *cmin)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const int q = q0 + threadIdx.x;
    if (q >= n) return;
    parent[first + q] = first + q;
    csize[first + q] = 0;
    cmin[first + q] = 0x7fffffff;
}

__global__ void __launch_bounds__(TQ) k_lvl_link(LevelBufs L, NodeArrays nd, const float4 *wpos,
                                                 const float4 *wvel, const float *dnn, int *parent,
                                                 rs_dev_status *st)
{
    __shared__ float4 cp[TQ], cv[TQ];
    __shared__ float cd[TQ];
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const Metric6 met = L.met[k];
    const double l2 = L.l2[k], l = sqrt(l2);
    const float lo = (float)(l2 * (1.0 - RS_BAND)), hi = (float)(l2 * (1.0 + RS_BAND));
    const float tlo = (float)(l2 * (1.0 - 3e-6)), thi = (float)(l2 * (1.0 + 3e-6));
    const float part = fmaxf(hi, thi);
    const int q = q0 + threadIdx.x;
    float4 pq = make_float4(0, 0, 0, 0), vq = pq;
    bool active = false;
    if (q < n) {
        pq = wpos[first + q];
        vq = wvel[first + q];
        active = dnn[first + q] <= part;
    }
    int tie = 0;
    for (int c0 = q0; c0 < n; c0 += TQ) {  // candidates c > q only
        __syncthreads();
        if (c0 + threadIdx.x < n) {
            cp[threadIdx.x] = wpos[first + c0 + threadIdx.x];
            cv[threadIdx.x] = wvel[first + c0 + threadIdx.x];
            cd[threadIdx.x] = dnn[first + c0 + threadIdx.x];
        }
        __syncthreads();
        if (!active) continue;
        const int m = min(TQ, n - c0);
        for (int j = 0; j < m; j++) {
            const int c = c0 + j;
            if (c <= q || cd[j] > part) continue;
            const float d2 = d2_32(pq, vq, cp[j], cv[j], met);
            if (d2 > part) continue;
            bool link = d2 <= lo;
            if (!link && (d2 <= hi || (d2 >= tlo && d2 <= thi))) {
                const double e = d2_64(pq, vq, cp[j], cv[j], met);
                link = e <= l2;
                if (l2 > 0 && e != l2 && fabs(sqrt(e) - l) <= 1e-6 * l) tie++;
            }
            if (link) uf_union(parent, first + q, first + c, st);
        }
    }
    tie = warp_sum(tie);
    if (lane_id() == 0 && tie) atomicAdd(&L.tie[k], tie);
}

__global__ void k_lvl_comp(LevelBufs L, NodeArrays nd, const int *widx, int *parent, int *csize, int *cmin,
                           rs_dev_status *st)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const int q = q0 + threadIdx.x;
    if (q >= n) return;
    int r = uf_find(parent, first + q, st);
    atomicAdd(&csize[r], 1);
    atomicMin(&cmin[r], widx[first + q]);
}

__global__ void k_lvl_keys(LevelBufs L, NodeArrays nd, int *parent, const int *csize, const int *cmin,
                           unsigned long long *keys, unsigned *vals, int min_n, rs_dev_status *st)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const int q = q0 + threadIdx.x;
    if (q >= n) return;
    int r = uf_find(parent, first + q, st);
    int sz = csize[r];
    unsigned comp = (sz >= min_n && sz < n) ? (unsigned)cmin[r] : 0xffffffffu;
    const int64_t p = L.seg_off[k] + q;
    keys[p] = ((unsigned long long)k << 32) | comp;
    vals[p] = (unsigned)(first + q);
}

__global__ void k_lvl_scatter(LevelBufs L, NodeArrays nd, int64_t LM, const unsigned long long *keys,
                              const unsigned *vals, const float4 *wpos, const float4 *wvel, const int *widx,
                              float4 *wpos2, float4 *wvel2, int *widx2, unsigned *dest)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= LM) return;
    const int k = (int)(keys[p] >> 32);
    const int node = L.list[k];
    const int d = nd.first[node] + (int)(p - L.seg_off[k]);
    const unsigned s = vals[p];
    wpos2[d] = wpos[s];
    wvel2[d] = wvel[s];
    widx2[d] = widx[s];
    dest[p] = (unsigned)d;
}

__global__ void k_lvl_copyback(int64_t LM, const unsigned *dest, const float4 *wpos2, const float4 *wvel2,
                               const int *widx2, float4 *wpos, float4 *wvel, int *widx)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= LM) return;
    const unsigned d = dest[p];
    wpos[d] = wpos2[d];
    wvel[d] = wvel2[d];
    widx[d] = widx2[d];
}

__global__ void k_lvl_children(LevelBufs L, NodeArrays nd, int64_t LM, const unsigned long long *keys,
                               const unsigned *vals, int *parent, const int *csize, int *next_list, int *next_len,
                               int *small_list, int *small_len, rs_dev_status *st)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= LM) return;
    const unsigned long long key = keys[p];
    const unsigned comp = (unsigned)(key & 0xffffffffu);
    if (comp == 0xffffffffu) return;
    if (p > 0 && keys[p - 1] == key) return;
    const int k = (int)(key >> 32);
    const int node = L.list[k];
    const int r = uf_find(parent, (int)vals[p], st);
    const int sz = csize[r];
    int id = atomicAdd(nd.counter, 1);
    if (id >= nd.cap) {
        dev_fail(st, DEV_OVERFLOW, 51, id);
        return;
    }
    nd.parent[id] = node;
    nd.level[id] = nd.level[node] + 1;
    nd.first[id] = nd.first[node] + (int)(p - L.seg_off[k]);
    nd.count[id] = sz;
    nd.minidx[id] = (int)comp;
    nd.nchild[id] = 0;
    nd.tie[id] = 0;
    nd.root[id] = nd.root[node];
    nd.shift[id] = nd.shift[node];
    atomicAdd(&nd.nchild[node], 1);
    if (sz > SMALL_N) next_list[atomicAdd(next_len, 1)] = id;
    else small_list[atomicAdd(small_len, 1)] = id;
}

__global__ void k_lvl_store_tie(LevelBufs L, NodeArrays nd)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.K) return;
    nd.tie[L.list[k]] = L.tie[k];
}

__global__ void k_tree_stats(NodeArrays nd, int n_nodes, unsigned long long *out)
{
    // out: [0] seeds, [1] tie sum, [2] max level, [3] sum of counts
    unsigned long long seeds = 0, tie = 0, sum = 0;
    int maxl = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += gridDim.x * blockDim.x) {
        seeds += nd.nchild[i] == 0;
        tie += (unsigned long long)nd.tie[i];
        sum += (unsigned long long)nd.count[i];
        maxl = max(maxl, nd.level[i]);
    }
    seeds = warp_sum(seeds);
    tie = warp_sum(tie);
    sum = warp_sum(sum);
    maxl = warp_max(maxl);
    if (lane_id() == 0) {
        atomicAdd(&out[0], seeds);
        atomicAdd(&out[1], tie);
        atomicMax(&out[2], (unsigned long long)maxl);
        atomicAdd(&out[3], sum);
    }
}

template <typename T>
T *carve(char *&p, int64_t count)
{
    T *r = (T *)p;
    size_t b = sizeof(T) * (size_t)(count > 0 ? count : 1);
    p += (b + 255) / 256 * 256;
    return r;
}

size_t tree_bytes(int64_t M, int64_t cap)
{
    size_t s = 0;
    auto add = [&](size_t b) { s += (b + 255) / 256 * 256; };
    for (int i = 0; i < 9; i++) add(sizeof(int) * cap);
    add(sizeof(double) * cap * 3);  // lnk, sigx, sigv
    add(sizeof(double) * cap * 3);
    add(sizeof(double) * cap * 3);
    add(sizeof(double) * cap * 3);
    add(sizeof(double) * cap * 3);
    add(sizeof(int) * 4);
    add(sizeof(int) * (M > 0 ? M : 1));
    return s + 4096;
}

}  // namespace

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static rs_status refine_impl(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n, double box,
                             const int32_t *perm, const int64_t *goff, int64_t G, double f, int32_t min_n,
                             int64_t node_cap, rs_tree **out)
{
    int64_t h[2];
    RS_TRY(rs_read_i64(ctx, goff, 1, h, "rs_refine6d"));
    RS_CUDA(ctx, cudaMemcpyAsync(ctx->h_scratch + 1, goff + G, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    RS_TRY(rs_sync_check(ctx, "rs_refine6d"));
    const int64_t M = ctx->h_scratch[1] - h[0];
    if (M < 0 || M > n || h[0] < 0) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_refine6d: inconsistent group offsets");
    RS_LAUNCH(ctx, "rf_check_offsets", k_check_offsets, ceil_div(G, 256), 256, 0, G, goff, ctx->d_status);
    RS_TRY(rs_sync_check(ctx, "rs_refine6d: group offsets must be non-decreasing"));

    rs_tree *t = new (std::nothrow) rs_tree();
    if (!t) return RS_ERR_OOM;
    t->n_total = n;
    t->n_members = M;
    t->box = box;
    const int64_t cap = node_cap;
    cudaError_t e = cudaMalloc(&t->block, tree_bytes(M, cap));
    if (e != cudaSuccess) {
        delete t;
        cudaGetLastError();
        return rs_fail(ctx, RS_ERR_OOM, "rs_refine6d: tree allocation failed");
    }
    char *p = (char *)t->block;
    NodeArrays &nd = t->nd;
    nd.parent = carve<int>(p, cap);
    nd.level = carve<int>(p, cap);
    nd.first = carve<int>(p, cap);
    nd.count = carve<int>(p, cap);
    nd.minidx = carve<int>(p, cap);
    nd.nchild = carve<int>(p, cap);
    nd.tie = carve<int>(p, cap);
    nd.root = carve<int>(p, cap);
    nd.shift = carve<int>(p, cap);
    nd.lnk = carve<double>(p, cap);
    nd.sigx = carve<double>(p, cap);
    nd.sigv = carve<double>(p, cap);
    nd.xbar = carve<double>(p, 3 * cap);
    nd.vbar = carve<double>(p, 3 * cap);
    nd.counter = carve<int>(p, 4);
    nd.cap = (int)cap;
    t->members = carve<int>(p, M);
    *out = t;

    const float boxf = (float)box;
    RS_CUDA(ctx, cudaMemsetAsync(nd.counter, 0, sizeof(int) * 4, ctx->stream));
    if (M == 0 || G == 0) return RS_OK;

    // working member arrays
    RS_WS(ctx, float4, wpos, WS_RF_POS, M);
    RS_WS(ctx, float4, wvel, WS_RF_VEL, M);
    RS_WS(ctx, float4, wpos2, WS_RF_POS2, M);
    RS_WS(ctx, float4, wvel2, WS_RF_VEL2, M);
    RS_WS(ctx, int, widx2, WS_RF_IDX2, M);
    RS_WS(ctx, float, dnn, WS_RF_DNN, M);
    RS_WS(ctx, int, uf, WS_RF_PARENT, 3 * M);
    int *csize = uf + M, *cmin = uf + 2 * M;
    int *widx = t->members;
    RS_WS(ctx, int, gmisc, WS_RF_MISC0, 2 * G + 2 * M + 8);
    int *shift_bits = gmisc, *gmin = gmisc + G, *slot_group = gmisc + 2 * G;
    // node queues: big lists (ping-pong) and the small queue; counters
    // counters first (16 ints = 64 bytes, so everything after stays 8-byte aligned)
    RS_WS(ctx, int, q, WS_RF_NODEQ, 3 * cap + 16);
    int *ctr = q, *big_a = q + 16, *big_b = q + 16 + cap, *small_q = q + 16 + 2 * cap;
    // ctr: [0] big_a len, [1] big_b len, [2] small len, [3] small head, [4] band len
    RS_CUDA(ctx, cudaMemsetAsync(ctr, 0, sizeof(int) * 16, ctx->stream));

    const int gb = (int)std::min<int64_t>(G, (int64_t)ctx->num_sms * 8);
    RS_LAUNCH(ctx, "rf_group_unwrap", k_group_unwrap, gb, 256, 0, G, goff, perm, n, pos, stride, boxf, shift_bits, gmin,
              ctx->d_status);
    RS_LAUNCH(ctx, "rf_gather", k_gather, gb, 256, 0, G, goff, perm, n, pos, vel, stride, boxf,
              (const int *)shift_bits, wpos, wvel, widx, slot_group);
    RS_LAUNCH(ctx, "rf_roots", k_make_roots, ceil_div(G, 256), 256, 0, G, goff, (const int *)gmin,
              (const int *)shift_bits, (int)min_n, nd,
              big_a, ctr + 0, small_q, ctr + 2, ctx->d_status);

    // ---- big levels ----
    int *cur = big_a, *nxt = big_b;
    int *cur_len = ctr + 0, *nxt_len = ctr + 1;
    int64_t sum_level = 0;
    for (int level = 0; level < 4096; level++) {
        int64_t K;
        RS_TRY(rs_read_i64(ctx, cur_len, 1, &K, "rs_refine6d"));
        K &= 0xffffffffll;
        if (K == 0) break;
        RS_WS(ctx, int64_t, lv64, WS_RF_MISC1, 4 * (K + 1) + 8);
        int64_t *tiles = lv64, *segc = lv64 + (K + 1), *tot = lv64 + 2 * (K + 1);
        RS_LAUNCH(ctx, "rf_lvl_prep", k_lvl_prep, ceil_div(K, 256), 256, 0, (const int *)cur, (int)K, nd, tiles,
                  segc);
        RS_CUDA(ctx, cudaMemsetAsync(tiles + K, 0, sizeof(int64_t), ctx->stream));
        RS_CUDA(ctx, cudaMemsetAsync(segc + K, 0, sizeof(int64_t), ctx->stream));
        RS_TRY(rs_scan_i64(ctx, tiles, K + 1, tot));
        RS_TRY(rs_scan_i64(ctx, segc, K + 1, tot + 1));
        int64_t TT[2];
        RS_TRY(rs_read_i64(ctx, tot, 2, TT, "rs_refine6d"));
        const int64_t T = TT[0], LM = TT[1];
        sum_level += LM;
        RS_WS(ctx, int, tl, WS_RF_MISC2, 2 * T + 8);
        LevelBufs L;
        L.list = cur;
        L.K = (int)K;
        L.tile_rank = tl;
        L.tile_q0 = tl + T;
        L.seg_off = segc;
        RS_LAUNCH(ctx, "rf_lvl_tiles", k_lvl_tiles, K, 256, 0, (int)K, (const int64_t *)tiles, tl, tl + T);
        // per-rank state
        size_t per = sizeof(MomAcc) + sizeof(Metric6) + 2 * sizeof(float4) + 2048 * sizeof(unsigned) +
                     4 * sizeof(int) + sizeof(double) + 64;
        RS_WS(ctx, char, rk, WS_RF_ACC, (int64_t)(per * K + 4096));
        char *rp = rk;
        L.acc = carve<MomAcc>(rp, K);
        L.met = carve<Metric6>(rp, K);
        L.ref = carve<float4>(rp, 2 * K);
        L.l2 = carve<double>(rp, K);
        L.hist = carve<unsigned>(rp, 2048 * K);
        L.sel_prefix = carve<unsigned>(rp, K);
        L.sel_krem = carve<int>(rp, K);
        L.below = carve<int>(rp, K);
        L.tie = carve<int>(rp, K);
        RS_CUDA(ctx, cudaMemsetAsync(rk, 0, (size_t)(rp - rk), ctx->stream));
        RS_WS(ctx, char, bandbuf, WS_RF_BAND, (int64_t)(LM * 16 + 64));
        char *bp = bandbuf;
        L.band_len = ctr + 4;
        L.band_rank = carve<int>(bp, LM);
        L.band_slot = carve<int>(bp, LM);
        L.band_val = carve<double>(bp, LM);
        RS_CUDA(ctx, cudaMemsetAsync(ctr + 4, 0, sizeof(int), ctx->stream));

        RS_LAUNCH(ctx, "rf_lvl_moments", k_lvl_moments, T, TQ, 0, L, nd, (const float4 *)wpos, (const float4 *)wvel);
        RS_LAUNCH(ctx, "rf_lvl_finalize", k_lvl_finalize, ceil_div(K, 128), 128, 0, L, nd, box);
        RS_LAUNCH(ctx, "rf_lvl_nn", k_lvl_nn, T, TQ, 0, L, nd, (const float4 *)wpos, (const float4 *)wvel, dnn);
        RS_LAUNCH(ctx, "rf_lvl_initk", k_lvl_initk, ceil_div(K, 128), 128, 0, L, nd, f);
        for (int pass = 0; pass < 3; pass++) {
            RS_LAUNCH(ctx, "rf_lvl_hist", k_lvl_hist, T, TQ, 0, L, nd, (const float *)dnn, pass);
            RS_LAUNCH(ctx, "rf_lvl_pick", k_lvl_pick, K, 32, 0, L, pass);
        }
        RS_LAUNCH(ctx, "rf_lvl_band", k_lvl_band, T, TQ, 0, L, nd, (const float *)dnn);
        int64_t NB;
        RS_TRY(rs_read_i64(ctx, ctr + 4, 1, &NB, "rs_refine6d"));
        NB &= 0xffffffffll;
        RS_LAUNCH(ctx, "rf_lvl_band_exact", k_lvl_band_exact, NB, TQ, 0, L, nd, (const float4 *)wpos,
                  (const float4 *)wvel, (const float *)dnn);
        RS_LAUNCH(ctx, "rf_lvl_l2", k_lvl_l2, K, 128, 0, L, nd, f, ctx->d_status);
        RS_LAUNCH(ctx, "rf_lvl_iota", k_lvl_iota, T, TQ, 0, L, nd, uf, csize, cmin);
        RS_LAUNCH(ctx, "rf_lvl_link", k_lvl_link, T, TQ, 0, L, nd, (const float4 *)wpos, (const float4 *)wvel,
                  (const float *)dnn, uf, ctx->d_status);
        RS_LAUNCH(ctx, "rf_lvl_comp", k_lvl_comp, T, TQ, 0, L, nd, (const int *)widx, uf, csize, cmin,
                  ctx->d_status);
        // reorder: children first, by smallest particle index, then the rest
        RS_WS(ctx, uint64_t, k0, WS_SORT_K0, LM);
        RS_WS(ctx, uint64_t, k1, WS_SORT_K1, LM);
        RS_WS(ctx, uint32_t, v0, WS_SORT_V0, LM);
        RS_WS(ctx, uint32_t, v1, WS_SORT_V1, LM);
        RS_LAUNCH(ctx, "rf_lvl_keys", k_lvl_keys, T, TQ, 0, L, nd, uf, (const int *)csize, (const int *)cmin,
                  (unsigned long long *)k0, v0, (int)min_n, ctx->d_status);
        int kbits = 32;
        while (kbits < 64 && ((uint64_t)(K - 1) >> (kbits - 32)) != 0) kbits++;
        bool alt = false;
        RS_TRY(rs_radix_sort_u64(ctx, k0, k1, v0, v1, LM, kbits, &alt));
        const unsigned long long *sk = (const unsigned long long *)(alt ? k1 : k0);
        const unsigned *sv = alt ? v1 : v0;
        unsigned *dest = (unsigned *)(alt ? v0 : v1);
        RS_LAUNCH(ctx, "rf_lvl_children", k_lvl_children, ceil_div(LM, 256), 256, 0, L, nd, LM, sk, sv, uf,
                  (const int *)csize, nxt, nxt_len, small_q, ctr + 2, ctx->d_status);
        RS_LAUNCH(ctx, "rf_lvl_scatter", k_lvl_scatter, ceil_div(LM, 256), 256, 0, L, nd, LM, sk, sv,
                  (const float4 *)wpos, (const float4 *)wvel, (const int *)widx, wpos2, wvel2, widx2, dest);
        RS_LAUNCH(ctx, "rf_lvl_copyback", k_lvl_copyback, ceil_div(LM, 256), 256, 0, LM, (const unsigned *)dest,
                  (const float4 *)wpos2, (const float4 *)wvel2, (const int *)widx2, wpos, wvel, widx);
        RS_LAUNCH(ctx, "rf_lvl_tie", k_lvl_store_tie, ceil_div(K, 128), 128, 0, L, nd);
        // next level
        RS_CUDA(ctx, cudaMemsetAsync(cur_len, 0, sizeof(int), ctx->stream));
        int *tq = cur;
        cur = nxt;
        nxt = tq;
        int *tl2 = cur_len;
        cur_len = nxt_len;
        nxt_len = tl2;
    }

    // ---- small nodes: whole subtrees ----
    const size_t smem = sizeof(SmallShared);
    RS_CUDA(ctx, cudaFuncSetAttribute(k_small_subtree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RS_LAUNCH(ctx, "rf_small_subtree", k_small_subtree, (int64_t)ctx->num_sms * 2, SMALL_THREADS, smem,
              (const int *)small_q, (const int *)(ctr + 2), ctr + 3, (const float4 *)wpos, (const float4 *)wvel, widx,
              nd, box, f, (int)min_n, ctx->d_status);

    // ---- summary ----
    RS_WS(ctx, unsigned long long, so, WS_RF_MISC3, 4);
    RS_CUDA(ctx, cudaMemsetAsync(so, 0, 4 * sizeof(unsigned long long), ctx->stream));
    int64_t nn;
    RS_TRY(rs_read_i64(ctx, nd.counter, 1, &nn, "rs_refine6d"));
    nn &= 0xffffffffll;
    if (nn > cap) return rs_fail(ctx, RS_ERR_INTERNAL, "rs_refine6d: node capacity exceeded");
    RS_LAUNCH(ctx, "rf_tree_stats", k_tree_stats, std::min<int64_t>(ceil_div(nn, 256), ctx->num_sms * 4), 256, 0, nd,
              (int)nn, so);
    int64_t s4[4];
    RS_TRY(rs_read_i64(ctx, so, 4, s4, "rs_refine6d"));
    t->n_nodes = nn;
    t->n_seeds = s4[0];
    t->n_tieband = s4[1];
    t->n_levels = nn > 0 ? (int32_t)s4[2] + 1 : 0;
    t->sum_level_members = s4[3];
    (void)sum_level;
    return RS_OK;
}

// ---------------------------------------------------------------------------
// public tree API
// ---------------------------------------------------------------------------
namespace {

__global__ void k_tree_export(NodeArrays nd, int nn, int32_t *parent, int32_t *level, int64_t *first,
                              int64_t *count, int32_t *minidx, int32_t *nchild, double *lnk, double *xbar,
                              double *vbar, double *sigx, double *sigv, int64_t *tie)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
        if (parent) parent[i] = nd.parent[i];
        if (level) level[i] = nd.level[i];
        if (first) first[i] = nd.first[i];
        if (count) count[i] = nd.count[i];
        if (minidx) minidx[i] = nd.minidx[i];
        if (nchild) nchild[i] = nd.nchild[i];
        if (lnk) lnk[i] = nd.lnk[i];
        if (sigx) sigx[i] = nd.sigx[i];
        if (sigv) sigv[i] = nd.sigv[i];
        if (tie) tie[i] = nd.tie[i];
        for (int d = 0; d < 3; d++) {
            if (xbar) xbar[3 * i + d] = nd.xbar[3 * i + d];
            if (vbar) vbar[3 * i + d] = nd.vbar[3 * i + d];
        }
    }
}

__global__ void k_level_labels(NodeArrays nd, int nn, int level, const int *members, int32_t *labels)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = w; i < nn; i += nw) {
        if (nd.level[i] != level) continue;
        const int a = nd.first[i], c = nd.count[i], id = nd.minidx[i];
        for (int m = lane_id(); m < c; m += 32) labels[members[a + m]] = id;
    }
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

}  // namespace

extern "C" void rs_tree_free(rs_tree *t)
{
    if (!t) return;
    if (t->block) cudaFree(t->block);
    delete t;
}

extern "C" rs_status rs_refine6d(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n,
                                 double box, const int32_t *perm, const int64_t *group_offsets, int64_t n_groups,
                                 double f, int32_t min_n, rs_tree **out)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    if (!out) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_refine6d: out is NULL");
    *out = nullptr;
    if (n < 0 || n_groups < 0 || (stride != 3 && stride != 4) || !(box > 0) || !(f > 0 && f < 1) || min_n < 2 ||
        !group_offsets || (n > 0 && (!pos || !vel)) || (n_groups > 0 && !perm))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_refine6d: bad argument");
    if (n >= ((int64_t)1 << 31)) return rs_fail(ctx, RS_ERR_TOO_LARGE, "rs_refine6d: n >= 2^31");
    if ((double)(float)box != box) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_refine6d: box must be a float32 value");
    int64_t cap = 0;
    {
        int64_t h[2];
        RS_TRY(rs_read_i64(ctx, group_offsets, 1, h, "rs_refine6d"));
        RS_CUDA(ctx, cudaMemcpyAsync(ctx->h_scratch + 1, group_offsets + n_groups, sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, ctx->stream));
        RS_TRY(rs_sync_check(ctx, "rs_refine6d"));
        int64_t M = ctx->h_scratch[1] - h[0];
        cap = M / 4 + 4096;
    }
    for (int attempt = 0; attempt < 4; attempt++) {
        rs_tree *t = nullptr;
        rs_status s = refine_impl(ctx, pos, vel, stride, n, box, perm, group_offsets, n_groups, f, min_n, cap, &t);
        if (s == RS_OK) {
            *out = t;
            return RS_OK;
        }
        bool overflow = false;
        if (t) {
            int cnt = 0;
            cudaStreamSynchronize(ctx->stream);
            if (cudaMemcpy(&cnt, t->nd.counter, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
                overflow = (int64_t)cnt > cap;
            rs_tree_free(t);
        }
        if (!overflow || cap > ((int64_t)1 << 30)) return s;
        cap *= 4;
    }
    return rs_fail(ctx, RS_ERR_INTERNAL, "rs_refine6d: node capacity");
}

extern "C" rs_status rs_tree_info(const rs_tree *t, int64_t *n_nodes, int32_t *n_levels, int64_t *n_seeds,
                                  int64_t *n_tieband, int64_t *n_members)
{
    if (!t) return RS_ERR_INVALID_ARG;
    if (n_nodes) *n_nodes = t->n_nodes;
    if (n_levels) *n_levels = t->n_levels;
    if (n_seeds) *n_seeds = t->n_seeds;
    if (n_tieband) *n_tieband = t->n_tieband;
    if (n_members) *n_members = t->n_members;
    return RS_OK;
}

extern "C" rs_status rs_tree_nodes(rs_ctx *ctx, const rs_tree *t, int32_t *parent, int32_t *level, int64_t *first,
                                   int64_t *count, int32_t *minidx, int32_t *nchild, double *lnk, double *xbar,
                                   double *vbar, double *sigx, double *sigv, int64_t *tie)
{
    if (!ctx || !t) return RS_ERR_INVALID_ARG;
    const int nn = (int)t->n_nodes;
    RS_LAUNCH(ctx, "tree_export", k_tree_export, std::min<int64_t>(ceil_div(nn, 256), 4096), 256, 0, t->nd, nn,
              parent, level, first, count, minidx, nchild, lnk, xbar, vbar, sigx, sigv, tie);
    return RS_OK;
}

extern "C" rs_status rs_tree_members(rs_ctx *ctx, const rs_tree *t, int32_t *members)
{
    if (!ctx || !t || (t->n_members > 0 && !members)) return RS_ERR_INVALID_ARG;
    if (t->n_members > 0)
        RS_CUDA(ctx, cudaMemcpyAsync(members, t->members, sizeof(int32_t) * t->n_members, cudaMemcpyDeviceToDevice,
                                     ctx->stream));
    return RS_OK;
}

extern "C" rs_status rs_tree_level_labels(rs_ctx *ctx, const rs_tree *t, int32_t level, int64_t n, int32_t *labels)
{
    if (!ctx || !t || n < 0 || (n > 0 && !labels)) return RS_ERR_INVALID_ARG;
    if (n != t->n_total) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_tree_level_labels: n differs from the tree's");
    if (n == 0) return RS_OK;
    RS_LAUNCH(ctx, "tree_fill", k_fill_i32, std::min<int64_t>(ceil_div(n, 256), 4096), 256, 0, labels, n, -1);
    const int nn = (int)t->n_nodes;
    RS_LAUNCH(ctx, "tree_level_labels", k_level_labels, std::min<int64_t>(ceil_div((int64_t)nn * 32, 256), 8192),
              256, 0, t->nd, nn, level, (const int *)t->members, labels);
    return RS_OK;
}

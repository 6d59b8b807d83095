// rs_refine.cu -- the phase-space FOF hierarchy (Sec. 3.2, Eq. 1).
//
// Members of every refined group are gathered into member slots in group
// order, with positions unwrapped into one periodic image per group (x - box
// for coordinates in the upper half of the box, exact in float32, when the
// group straddles a face).  Nodes own nested slot ranges: a node's children
// occupy the front of its range.
//
// Size classes:
//  * big nodes (> SMALL_N members): processed level by level by tiles of 256
//    members spread over the whole GPU, with per-node accumulators and
//    histograms in global memory.  At levels 0 and 1 their members are put in
//    k-d order (splits at leaf-aligned medians); each node then has a 32-ary
//    box hierarchy over 32-member leaves, searched one query per warp for
//    nearest neighbours and friends.  Children above SMALL_N stay on the big
//    path, smaller children join the small-node queue;
//  * small nodes (<= SMALL_N members): one CTA loads the node into shared
//    memory and builds its whole subtree there (moments, nearest neighbours,
//    exact k-th select, union-find, children, recursion with an explicit
//    stack), as a persistent work queue; a second instance with 128 threads
//    and MID_N-member shared arrays takes the subtrees of at most MID_N
//    members, which the first forwards to it;
//  * tiny nodes (<= TINY_N = 32 members): one warp holds the node in
//    registers, a member per lane, and builds its whole subtree with warp
//    shuffles and votes, eight subtrees per CTA at a time; the middle
//    instance forwards them here.
//
// Exactness: means and dispersions come from exact fixed-point integer sums;
// nearest-neighbour and link tests run in float32 against a band of 2^-20
// (relative, on d^2) around the linking length, and everything inside the
// band is re-evaluated in float64.  The linking length itself is the exact
// float64 k-th smallest nearest-neighbour distance: the float32 k-th value
// brackets it, and only the members whose float32 distance lies within twice
// the band of it are re-evaluated in float64 and ranked.
//
// Optionally (subset size s > 0) a big node of more than s members takes its
// linking length from the nearest-neighbour distances of a random s-member
// subset only (Sec. 3.2, the paper's s = 10,000): the subset is found by a
// radix select on per-particle SplitMix64 keys and searched one warp per
// member; the other members skip the nearest-neighbour search.
#include <cmath>
#include <cstring>

#include "rs_refine.cuh"

namespace {

constexpr int SMALL_N = 1024;       // largest node handled by one CTA
constexpr int SMALL_THREADS = 256;
constexpr int STACK_CAP = 256;
constexpr int MID_N = 256;          // largest node of the middle CTA size
constexpr int MID_THREADS = 128;
constexpr int TINY_N = 32;          // largest node handled by one warp
constexpr int TINY_WARPS = 8;       // warps per block of the tiny-node kernel
constexpr int TINY_STACK = 32;      // pending nodes per warp
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
// float <-> int with the same order (finite values and infinities)
__device__ __forceinline__ int ord_i(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__device__ __forceinline__ float ord_f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_fill_s32(int32_t *p, int64_t n, int32_t v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// group of member slot m (off[g] <= base + m < off[g + 1])
__device__ __forceinline__ int64_t group_of(const int64_t *off, int64_t G, int64_t at)
{
    int64_t lo = 0, hi = G;  // off[lo] <= at < off[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= at) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Unwrap decision inputs, one member per thread over all groups: per group
// and axis the minima of x and -x, unshifted and with the upper half of the
// box shifted down by the box, and the smallest particle index.  Lanes of
// one group (groups are contiguous runs of slots) combine before their
// atomics, kept on order-preserving integer images of the floats.
__global__ void k_unwrap_tiles(int64_t G, const int64_t *off, const int32_t *perm, int64_t n, int64_t M,
                               const float *pos, int stride, float boxf, int *slot_group, int *gred, int *gmin,
                               rs_dev_status *st)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = m < M;
    int g = -1, i = 0x7fffffff;
    float r[12];
    for (int k = 0; k < 12; k++) r[k] = INFINITY;
    if (ok) {
        g = (int)group_of(off, G, off[0] + m);
        slot_group[m] = g;
        i = perm[off[0] + m];
        if (i < 0 || i >= n) {
            dev_fail(st, DEV_BADARG, 33, m);
            i = 0x7fffffff;
        } else {
            float c[3];
            load3(pos, stride, i, c[0], c[1], c[2]);
            for (int d = 0; d < 3; d++) {
                const float sft = c[d] >= 0.5f * boxf ? c[d] - boxf : c[d];
                r[d] = c[d];
                r[3 + d] = -c[d];
                r[6 + d] = sft;
                r[9 + d] = -sft;
            }
        }
    }
    const unsigned grp = __match_any_sync(0xffffffffu, g);
    const int lead = __ffs(grp) - 1;
    int v[12];
    for (int k = 0; k < 12; k++) v[k] = __reduce_min_sync(grp, ord_i(r[k]));
    const int mi = (int)__reduce_min_sync(grp, (unsigned)i);
    if (ok && lane_id() == lead) {
        for (int k = 0; k < 12; k++) atomicMin(&gred[12 * (int64_t)g + k], v[k]);
        atomicMin(&gmin[g], mi);
    }
}

// per group: which axes wrap (the group spans less than half the box once
// the upper half is shifted down), or an extent error
__global__ void k_unwrap_bits(int64_t G, const int *gred, float boxf, int *shift_bits, rs_dev_status *st)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int *r = gred + 12 * g;
    int bits = 0;
    for (int d = 0; d < 3; d++) {
        const float ext = -ord_f(r[3 + d]) - ord_f(r[d]);
        const float exts = -ord_f(r[9 + d]) - ord_f(r[6 + d]);
        if (ext < 0.5f * boxf) {
        } else if (exts < 0.5f * boxf) {
            bits |= 1 << d;
        } else {
            dev_fail(st, DEV_EXTENT, 30, g);
        }
    }
    shift_bits[g] = bits;
}

__global__ void k_gather(int64_t M, const int64_t *off, const int32_t *perm, int64_t n, const float *pos,
                         const float *vel, int stride, float boxf, const int *slot_group, const int *shift_bits,
                         float4 *wpos, float4 *wvel, int *widx)
{
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int bits = shift_bits[slot_group[m]];
    int i = perm[off[0] + m];
    if (i < 0 || i >= n) i = 0;  // recorded by k_unwrap_tiles
    float x, y, z, u, v, w;
    load3(pos, stride, i, x, y, z);
    load3(vel, stride, i, u, v, w);
    if ((bits & 1) && x >= 0.5f * boxf) x = x - boxf;
    if ((bits & 2) && y >= 0.5f * boxf) y = y - boxf;
    if ((bits & 4) && z >= 0.5f * boxf) z = z - boxf;
    wpos[m] = make_float4(x, y, z, 0.f);
    wvel[m] = make_float4(u, v, w, 0.f);
    widx[m] = i;
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
    if (cnt > ((int64_t)8 << 23)) {  // the per-node hierarchy has at most 24 levels
        dev_fail(st, DEV_OVERFLOW, 35, g);
        return;
    }
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
template <int NMAX, int NT>
struct SmallShared {
    float px[NMAX], py[NMAX], pz[NMAX], vx[NMAX], vy[NMAX], vz[NMAX];
    int idx[NMAX];
    float dnn[NMAX];
    int par[NMAX];
    int csize[NMAX];
    int cmin[NMAX];
    unsigned long long key[NMAX];
    float tp[6][NMAX];
    int tidx[NMAX];
    int4 stack[STACK_CAP];
    int sp;
    int job;
    MomAcc wacc[NT / 32];
    Metric6 met;
    double l2;
    float lo32, hi32, tlo32, thi32;
    int nband, below, tie, nchild;
    int pick;
};

template <class SS>
__device__ __forceinline__ float4 sp4(const SS &S, int i)
{
    return make_float4(S.px[i], S.py[i], S.pz[i], 0.f);
}
template <class SS>
__device__ __forceinline__ float4 sv4(const SS &S, int i)
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

// One CTA of NT threads per subtree of at most NMAX members; nodes of at most
// `fwd_limit` members (roots or children) go to the next queue, whose kernel
// runs after this one (members are written back in their final order).
template <int NMAX, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_small_subtree(const int *queue, const int *queue_len, int *queue_head, float4 *wpos, float4 *wvel, int *widx,
                    int fwd_limit, int *fwd_q, int *fwd_len, NodeArrays nd, double box, double f, int min_n,
                    rs_dev_status *st)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallShared<NMAX, NT> &S = *reinterpret_cast<SmallShared<NMAX, NT> *>(smem_raw);
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
        if (n0 <= fwd_limit) {  // a subtree for the next, smaller kernel
            if (tid == 0) fwd_q[atomicAdd(fwd_len, 1)] = node0;
            continue;
        }
        for (int i = tid; i < n0; i += NT) {
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
                for (int i = lf + tid; i < lf + cnt; i += NT) mom_add(a, sp4(S, i), sv4(S, i), ref);
                mom_warp_reduce(a);
                if (lane_id() == 0) S.wacc[warp_id()] = a;
                __syncthreads();
                if (tid == 0) {
                    MomAcc t = S.wacc[0];
                    for (int w = 1; w < NT / 32; w++) mom_merge(t, S.wacc[w]);
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
            for (int q = lf + tid; q < lf + cnt; q += NT) {
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
            for (int i = tid; i < P; i += NT)
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
            // (one warp per band member, lanes over the candidates)
            double *bval = reinterpret_cast<double *>(S.key);
            int *blist = S.tidx;
            for (int q = lf + tid; q < lf + cnt; q += NT) {
                const float dq = S.dnn[q];
                if (dq < blo)
                    atomicAdd(&S.below, 1);
                else if (dq <= bhi)
                    blist[atomicAdd(&S.nband, 1)] = q;
            }
            __syncthreads();
            for (int b = warp_id(); b < S.nband; b += NT / 32) {
                const int q = blist[b];
                const float4 pq = sp4(S, q), vq = sv4(S, q);
                const float lim = S.dnn[q] * (float)(1.0 + 2.0 * RS_BAND);
                double best = INFINITY;
                for (int c = lf + lane_id(); c < lf + cnt; c += 32) {
                    if (c == q) continue;
                    const float4 pc = sp4(S, c), vc = sv4(S, c);
                    if (d2_32(pq, vq, pc, vc, met) <= lim) best = fmin(best, d2_64(pq, vq, pc, vc, met));
                }
                for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
                if (lane_id() == 0) bval[b] = best;
            }
            __syncthreads();
            // rank the band: the exact k-th value is the (k - 1 - below)-th
            {
                const int nb = S.nband, want = (int)(kk - 1) - S.below;
                if (want < 0 || want >= nb) {
                    if (tid == 0) dev_fail(st, DEV_INTERNAL, 40, node);
                }
                for (int b = tid; b < nb; b += NT) {
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
            for (int i = lf + tid; i < lf + cnt; i += NT) S.par[i] = i;
            __syncthreads();
            // ---- friends-of-friends at l (inclusive) ----
            {
                const float lo = S.lo32, hi = S.hi32, tlo = S.tlo32, thi = S.thi32;
                const float part = fmaxf(hi, thi);
                const double l = sqrt(l2);
                int tie = 0;
                // warp-uniform candidate loop from the warp's first query: the
                // candidate test and its loads are the same for every lane
                for (int qb = lf + 32 * warp_id(); qb < lf + cnt; qb += NT) {
                    const int q = qb + lane_id();
                    const bool act = q < lf + cnt && S.dnn[q] <= part;
                    if (!__any_sync(0xffffffffu, act)) continue;
                    const float4 pq = act ? sp4(S, q) : make_float4(0, 0, 0, 0);
                    const float4 vq = act ? sv4(S, q) : make_float4(0, 0, 0, 0);
                    for (int c = qb + 1; c < lf + cnt; c++) {
                        if (S.dnn[c] > part) continue;
                        const float4 pc = sp4(S, c), vc = sv4(S, c);
                        if (!act || c <= q) continue;
                        const float d2 = d2_32(pq, vq, pc, vc, met);
                        if (d2 > part) continue;
                        // below both bands: a friend, and not a tie-band pair
                        bool link = d2 < fminf(lo, tlo);
                        if (!link) {
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
            for (int i = lf + tid; i < lf + cnt; i += NT) {
                S.csize[i] = 0;
                S.cmin[i] = 0x7fffffff;
            }
            __syncthreads();
            for (int i = lf + tid; i < lf + cnt; i += NT) {
                int r = uf_find_s(S.par, i);
                S.par[i] = r;
                atomicAdd(&S.csize[r], 1);
                atomicMin(&S.cmin[r], S.idx[i]);
            }
            __syncthreads();
            // ---- children first (by smallest particle index), then the rest ----
            for (int i = tid; i < P; i += NT) {
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
            for (int p = tid; p < cnt; p += NT) {
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
            for (int p = tid; p < cnt; p += NT) {
                S.px[lf + p] = S.tp[0][p];
                S.py[lf + p] = S.tp[1][p];
                S.pz[lf + p] = S.tp[2][p];
                S.vx[lf + p] = S.tp[3][p];
                S.vy[lf + p] = S.tp[4][p];
                S.vz[lf + p] = S.tp[5][p];
                S.idx[lf + p] = S.tidx[p];
            }
            __syncthreads();
            for (int p = tid; p < cnt; p += NT) {
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
                if (e - p <= fwd_limit) {  // its subtree goes to the next, smaller kernel
                    fwd_q[atomicAdd(fwd_len, 1)] = id;
                    continue;
                }
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
        // members in their final order (the tiny-node kernel reads its nodes here)
        for (int i = tid; i < n0; i += NT) {
            widx[base + i] = S.idx[i];
            wpos[base + i] = make_float4(S.px[i], S.py[i], S.pz[i], 0.f);
            wvel[base + i] = make_float4(S.vx[i], S.vy[i], S.vz[i], 0.f);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// tiny nodes: whole subtree in one warp
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 shfl_xyz(float4 a, int src)
{
    return make_float4(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src),
                       __shfl_sync(0xffffffffu, a.z, src), 0.f);
}

// ascending bitonic sort of one 64-bit key per lane across the warp
__device__ __forceinline__ unsigned long long warp_sort_u64(unsigned long long key)
{
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            key = keep_min ? (o < key ? o : key) : (o > key ? o : key);
        }
    return key;
}

// One warp per tiny subtree: lane i holds member i of the subtree root's slot
// range, and a node is a contiguous range of lanes.  The steps and their
// arithmetic are those of the one-CTA path: exact moments, float32 nearest
// neighbours, the float32 k-th value and the float64 band around it, the
// float64 k-th value, friends-of-friends with the float64 recheck in the band,
// then children first by smallest particle index and the rest after them.
__global__ void __launch_bounds__(TINY_WARPS * 32)
    k_tiny_subtree(const int *queue, const int *queue_len, int *queue_head, const float4 *wpos, const float4 *wvel,
                   int *widx, NodeArrays nd, double box, double f, int min_n, rs_dev_status *st)
{
    __shared__ int par_s[TINY_WARPS][32];
    __shared__ int csz_s[TINY_WARPS][32];
    __shared__ int cmin_s[TINY_WARPS][32];
    __shared__ int4 stk_s[TINY_WARPS][TINY_STACK];
    const unsigned FULL = 0xffffffffu;
    const int w = warp_id(), lane = lane_id();
    int *par = par_s[w], *csz = csz_s[w], *cmn = cmin_s[w];
    int4 *stk = stk_s[w];
    const int qlen = *queue_len;
    for (int guard = 0; guard < (1 << 30); guard++) {
        int job = 0;
        if (lane == 0) job = atomicAdd(queue_head, 1);
        job = __shfl_sync(FULL, job, 0);
        if (job >= qlen) break;
        const int node0 = queue[job];
        const int base = nd.first[node0], n0 = nd.count[node0];
        if (n0 > TINY_N) {
            if (lane == 0) dev_fail(st, DEV_INTERNAL, 44, node0);
            continue;
        }
        float4 p = make_float4(0, 0, 0, 0), v = p;
        int idx = 0x7fffffff;
        if (lane < n0) {
            p = wpos[base + lane];
            v = wvel[base + lane];
            idx = widx[base + lane];
        }
        if (lane == 0) stk[0] = make_int4(0, n0, node0, nd.level[node0]);
        int sp = 1;
        __syncwarp();
        for (int it = 0; sp > 0 && it < 4096; it++) {
            const int4 top = stk[--sp];
            __syncwarp();
            const int off = top.x, cnt = top.y, node = top.z, lev = top.w;
            const bool mine = lane >= off && lane < off + cnt;
            // ---- moments (exact), the node's first member as reference ----
            const float4 pr = shfl_xyz(p, off), vr = shfl_xyz(v, off);
            MomAcc a;
            mom_zero(a);
            if (mine) mom_add(a, p, v, mom_ref(pr, vr));
            mom_warp_reduce(a);
            Metric6 met;
            {
                double ax64 = 0, av64 = 0, scale = 0;
                if (lane == 0) {
                    const MomOut o = mom_finalize(a, pr, vr, cnt, box);
                    for (int d = 0; d < 3; d++) {
                        nd.xbar[3 * node + d] = o.xbar[d];
                        nd.vbar[3 * node + d] = o.vbar[d];
                    }
                    nd.sigx[node] = o.sigx;
                    nd.sigv[node] = o.sigv;
                    const Metric6 m = metric_of(o.sigx, o.sigv);
                    ax64 = m.ax64;
                    av64 = m.av64;
                    scale = m.scale;
                }
                met.ax64 = __shfl_sync(FULL, ax64, 0);
                met.av64 = __shfl_sync(FULL, av64, 0);
                met.scale = __shfl_sync(FULL, scale, 0);
                met.ax = (float)met.ax64;
                met.av = (float)met.av64;
            }
            // ---- nearest neighbours (float32) ----
            float dnn = INFINITY;
            for (int c = off; c < off + cnt; c++) {
                const float4 pc = shfl_xyz(p, c), vc = shfl_xyz(v, c);
                if (mine && c != lane) dnn = fminf(dnn, d2_32(p, v, pc, vc, met));
            }
            // ---- k-th smallest, float32: the member of rank k - 1 by (value, lane) ----
            long long kk = (long long)ceil(f * (double)cnt);
            if (kk < 1) kk = 1;
            if (kk > cnt) kk = cnt;
            int rank = 0;
            for (int c = off; c < off + cnt; c++) {
                const float dc = __shfl_sync(FULL, dnn, c);
                if (mine && (dc < dnn || (dc == dnn && c < lane))) rank++;
            }
            const unsigned pick = __ballot_sync(FULL, mine && rank == kk - 1);
            const float t32 = __shfl_sync(FULL, dnn, pick ? __ffs(pick) - 1 : off);
            const float blo = (float)((double)t32 * (1.0 - 2.0 * RS_BAND));
            const float bhi = (float)((double)t32 * (1.0 + 2.0 * RS_BAND));
            // ---- band members: exact float64 nearest-neighbour distances ----
            const bool inband = mine && dnn >= blo && dnn <= bhi;
            const int below = __popc(__ballot_sync(FULL, mine && dnn < blo));
            double ex = INFINITY;
            if (__any_sync(FULL, inband)) {
                const float lim = dnn * (float)(1.0 + 2.0 * RS_BAND);
                for (int c = off; c < off + cnt; c++) {
                    const float4 pc = shfl_xyz(p, c), vc = shfl_xyz(v, c);
                    if (inband && c != lane && d2_32(p, v, pc, vc, met) <= lim) ex = fmin(ex, d2_64(p, v, pc, vc, met));
                }
            }
            // the exact k-th value is the (k - 1 - below)-th smallest band value
            const int want = (int)(kk - 1) - below;
            const unsigned bmask = __ballot_sync(FULL, inband);
            int brank = 0;
            for (int c = off; c < off + cnt; c++) {
                const double ec = __shfl_sync(FULL, ex, c);
                if (inband && ((bmask >> c) & 1u) && (ec < ex || (ec == ex && c < lane))) brank++;
            }
            const unsigned bp = __ballot_sync(FULL, inband && brank == want);
            if (!bp && lane == 0) dev_fail(st, DEV_INTERNAL, 45, node);
            const double l2 = bp ? __shfl_sync(FULL, ex, __ffs(bp) - 1) : 0.0;
            if (lane == 0) nd.lnk[node] = sqrt(l2 / met.scale);
            // ---- friends-of-friends at l (inclusive) ----
            const float lo = (float)(l2 * (1.0 - RS_BAND)), hi = (float)(l2 * (1.0 + RS_BAND));
            const float tlo = (float)(l2 * (1.0 - 3e-6)), thi = (float)(l2 * (1.0 + 3e-6));
            const float part = fmaxf(hi, thi);
            const double l = sqrt(l2);
            par[lane] = lane;
            __syncwarp();
            int tie = 0;
            const bool act = mine && dnn <= part;
            for (int c = off; c < off + cnt; c++) {
                const float dc = __shfl_sync(FULL, dnn, c);
                const float4 pc = shfl_xyz(p, c), vc = shfl_xyz(v, c);
                if (!act || c <= lane || dc > part) continue;
                const float d2 = d2_32(p, v, pc, vc, met);
                if (d2 > part) continue;
                // below both bands: a friend, and not a tie-band pair
                bool link = d2 < fminf(lo, tlo);
                if (!link) {
                    const double e = d2_64(p, v, pc, vc, met);
                    link = e <= l2;
                    if (l2 > 0 && e != l2 && fabs(sqrt(e) - l) <= 1e-6 * l) tie++;
                }
                if (link) uf_union_s(par, lane, c, st);
            }
            tie = warp_sum(tie);
            __syncwarp();
            // ---- components ----
            csz[lane] = 0;
            cmn[lane] = 0x7fffffff;
            __syncwarp();
            int r = lane;
            if (mine) {
                r = uf_find_s(par, lane);
                atomicAdd(&csz[r], 1);
                atomicMin(&cmn[r], idx);
            }
            __syncwarp();
            // ---- children first (by smallest particle index), then the rest ----
            unsigned hiw = 0xffffffffu;
            if (mine) {
                const int sz = csz[r];
                if (sz >= min_n && sz < cnt) hiw = (unsigned)cmn[r];
            }
            const unsigned long long key =
                warp_sort_u64(mine ? (((unsigned long long)hiw << 32) | (unsigned)(lane - off)) : ~0ull);
            // the lane at position q of the node takes the member whose key sorted to q
            const unsigned long long kq = __shfl_sync(FULL, key, mine ? lane - off : lane);
            const int from = mine ? off + (int)(kq & 0xffffffffu) : lane;
            p = shfl_xyz(p, from);
            v = shfl_xyz(v, from);
            idx = __shfl_sync(FULL, idx, from);
            const unsigned khi = mine ? (unsigned)(kq >> 32) : 0xfffffffeu;
            // ---- emit the children ----
            const unsigned same = __match_any_sync(FULL, khi);
            const bool start = mine && khi != 0xffffffffu && (__ffs(same) - 1) == lane;
            const unsigned starts = __ballot_sync(FULL, start);
            const int nch = __popc(starts);
            if (sp + nch > TINY_STACK) {
                if (lane == 0) dev_fail(st, DEV_OVERFLOW, 46, node);
                break;
            }
            int id = -1;
            if (start) {
                id = atomicAdd(nd.counter, 1);
                if (id >= nd.cap) {  // the host retries with a larger capacity
                    dev_fail(st, DEV_OVERFLOW, 47, id);
                    id = -1;
                } else {
                    nd.parent[id] = node;
                    nd.level[id] = lev + 1;
                    nd.first[id] = base + lane;
                    nd.count[id] = __popc(same);
                    nd.minidx[id] = (int)khi;
                    nd.nchild[id] = 0;
                    nd.tie[id] = 0;
                    nd.root[id] = nd.root[node];
                    nd.shift[id] = nd.shift[node];
                }
            }
            const unsigned pushed = __ballot_sync(FULL, id >= 0);
            if (id >= 0) stk[sp + __popc(pushed & ((1u << lane) - 1u))] = make_int4(lane, __popc(same), id, lev + 1);
            sp += __popc(pushed);
            if (lane == 0) {
                nd.nchild[node] = __popc(pushed);
                nd.tie[node] = tie;
            }
            __syncwarp();
        }
        if (lane < n0) widx[base + lane] = idx;
        __syncwarp();
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
    unsigned *sub_t;         // per rank: subset key threshold, high and low words (2 entries)
    int *sub_cnt;            // per rank: members drawn into the subset
};

__global__ void k_lvl_prep(const int *list, int K, NodeArrays nd, int64_t *tiles, int64_t *segc,
                           unsigned long long *max_count)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    int c = nd.count[list[k]];
    tiles[k] = ceil_div(c, TQ);
    segc[k] = c;
    atomicMax(max_count, (unsigned long long)c);
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

// ---- raw-coordinate boxes ----
// A box is (lo, hi) over the six raw float32 coordinates of its members (the
// unwrapped positions and the velocities).  The gap between two boxes along
// an axis is one float32 subtraction of exact input values, so the box
// distance below is within 8 float32 ulps (relative) of the exact minimum
// squared distance between the boxes under the node's metric; a box is
// skipped only when that bound exceeds the current radius by 2^-18 relative,
// which can never skip a member whose float32 distance would change the
// result.
#define RS_PRUNE_SLACK 1.000003814697265625f  // 1 + 2^-18

struct Box6 {
    float4 plo, phi, vlo, vhi;
};

// Boxes of one level's hierarchies as three float4 streams (the lows and
// highs of the six coordinates, 48 bytes a box) and one flag byte, so a warp
// reading 32 consecutive boxes uses every byte of every sector it touches.
struct BoxStore {
    float4 *a;         // plo.x, plo.y, plo.z, vlo.x
    float4 *b;         // vlo.y, vlo.z, phi.x, phi.y
    float4 *c;         // phi.z, vhi.x, vhi.y, vhi.z
    unsigned char *cl; // clique flag
};

__device__ __forceinline__ Box6 box_get(const BoxStore &S, int64_t i)
{
    const float4 x = S.a[i], y = S.b[i], z = S.c[i];
    Box6 r;
    r.plo = make_float4(x.x, x.y, x.z, 0.f);
    r.vlo = make_float4(x.w, y.x, y.y, 0.f);
    r.phi = make_float4(y.z, y.w, z.x, 0.f);
    r.vhi = make_float4(z.y, z.z, z.w, 0.f);
    return r;
}

__device__ __forceinline__ void box_put(const BoxStore &S, int64_t i, const Box6 &r)
{
    S.a[i] = make_float4(r.plo.x, r.plo.y, r.plo.z, r.vlo.x);
    S.b[i] = make_float4(r.vlo.y, r.vlo.z, r.phi.x, r.phi.y);
    S.c[i] = make_float4(r.phi.z, r.vhi.x, r.vhi.y, r.vhi.z);
}

__device__ __forceinline__ BoxStore box_shift(const BoxStore &S, int64_t base)
{
    BoxStore r;
    r.a = S.a + base;
    r.b = S.b + base;
    r.c = S.c + base;
    r.cl = S.cl + base;
    return r;
}

// The searched members of one level, packed to the six coordinates (24
// bytes a member, by slot): written while the hierarchy is built.
struct MemberStore {
    float4 *a;  // px, py, pz, vx
    float2 *b;  // vy, vz
};

__device__ __forceinline__ void mem_get(const MemberStore &M, int64_t i, float4 &p, float4 &v)
{
    const float4 x = M.a[i];
    const float2 y = M.b[i];
    p = make_float4(x.x, x.y, x.z, 0.f);
    v = make_float4(x.w, y.x, y.y, 0.f);
}

__device__ __forceinline__ MemberStore mem_shift(const MemberStore &M, int64_t base)
{
    MemberStore r;
    r.a = M.a + base;
    r.b = M.b + base;
    return r;
}

// ---- per-node 32-ary bounding-volume hierarchy over the member range ----
// Leaves hold BVH_LEAF = 32 consecutive members (the range is in k-d order at
// level 0, inherited below); box (h, i) of level h is the union of boxes
// (h-1, 32i .. 32i+31), so it spans members [i 32^(h+1), (i+1) 32^(h+1)).  The fan-out equals the
// warp width: a search gives each lane one child box of the box it opens, or
// one member of the leaf it scans.  Boxes of a node are stored level by
// level from its base offset.
constexpr int BVH_LEAF = 32;
constexpr int BVH_LOG = 5;  // log2 of the leaf size and of the fan-out
constexpr int BVH_MAXH = 8;

__device__ __forceinline__ int bvh_levels(int nl)
{
    int h = 1;
    while (nl > 1) {
        nl = (nl + 31) >> BVH_LOG;
        h++;
    }
    return h;
}

__device__ __forceinline__ int64_t bvh_total(int nl)
{
    int64_t t = nl;
    while (nl > 1) {
        nl = (nl + 31) >> BVH_LOG;
        t += nl;
    }
    return t;
}

// first member of box (h, i) and the end of its member range
__device__ __forceinline__ int64_t bvh_m0(int h, int i) { return (int64_t)i << (BVH_LOG * (h + 1)); }

__global__ void k_bvh_prep(const int *list, int K, NodeArrays nd, int64_t *nbox)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int n = nd.count[list[k]];
    nbox[k] = bvh_total((int)ceil_div(n, BVH_LEAF));
}

__device__ __forceinline__ Box6 box_empty()
{
    Box6 b;
    b.plo = b.vlo = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    b.phi = b.vhi = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
    return b;
}

__device__ __forceinline__ void box_add(Box6 &b, float4 p, float4 v)
{
    b.plo.x = fminf(b.plo.x, p.x); b.plo.y = fminf(b.plo.y, p.y); b.plo.z = fminf(b.plo.z, p.z);
    b.phi.x = fmaxf(b.phi.x, p.x); b.phi.y = fmaxf(b.phi.y, p.y); b.phi.z = fmaxf(b.phi.z, p.z);
    b.vlo.x = fminf(b.vlo.x, v.x); b.vlo.y = fminf(b.vlo.y, v.y); b.vlo.z = fminf(b.vlo.z, v.z);
    b.vhi.x = fmaxf(b.vhi.x, v.x); b.vhi.y = fmaxf(b.vhi.y, v.y); b.vhi.z = fmaxf(b.vhi.z, v.z);
}

__device__ __forceinline__ void box_merge(Box6 &b, const Box6 &c)
{
    b.plo.x = fminf(b.plo.x, c.plo.x); b.plo.y = fminf(b.plo.y, c.plo.y); b.plo.z = fminf(b.plo.z, c.plo.z);
    b.phi.x = fmaxf(b.phi.x, c.phi.x); b.phi.y = fmaxf(b.phi.y, c.phi.y); b.phi.z = fmaxf(b.phi.z, c.phi.z);
    b.vlo.x = fminf(b.vlo.x, c.vlo.x); b.vlo.y = fminf(b.vlo.y, c.vlo.y); b.vlo.z = fminf(b.vlo.z, c.vlo.z);
    b.vhi.x = fmaxf(b.vhi.x, c.vhi.x); b.vhi.y = fmaxf(b.vhi.y, c.vhi.y); b.vhi.z = fmaxf(b.vhi.z, c.vhi.z);
}

// warp min/max votes on order-preserving integer images
__device__ __forceinline__ float wmin_f(float x) { return ord_f(__reduce_min_sync(0xffffffffu, ord_i(x))); }
__device__ __forceinline__ float wmax_f(float x) { return ord_f(__reduce_max_sync(0xffffffffu, ord_i(x))); }

// Leaf boxes and the packed member copy, one warp per leaf over the whole
// level (tiles of 256 members, eight leaves each).
__global__ void __launch_bounds__(TQ) k_bvh_leaves(LevelBufs L, NodeArrays nd, const int64_t *box_base, BoxStore B,
                                                   MemberStore MS, const float4 *wpos, const float4 *wvel)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x] + 32 * warp_id();
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    if (q0 >= n) return;
    const int m = q0 + lane_id();
    const bool ok = m < n;
    float4 p = make_float4(0, 0, 0, 0), v = p;
    if (ok) {
        p = wpos[first + m];
        v = wvel[first + m];
        MS.a[first + m] = make_float4(p.x, p.y, p.z, v.x);
        MS.b[first + m] = make_float2(v.y, v.z);
    }
    Box6 b;
    b.plo = make_float4(wmin_f(ok ? p.x : INFINITY), wmin_f(ok ? p.y : INFINITY), wmin_f(ok ? p.z : INFINITY), 0.f);
    b.phi = make_float4(wmax_f(ok ? p.x : -INFINITY), wmax_f(ok ? p.y : -INFINITY), wmax_f(ok ? p.z : -INFINITY), 0.f);
    b.vlo = make_float4(wmin_f(ok ? v.x : INFINITY), wmin_f(ok ? v.y : INFINITY), wmin_f(ok ? v.z : INFINITY), 0.f);
    b.vhi = make_float4(wmax_f(ok ? v.x : -INFINITY), wmax_f(ok ? v.y : -INFINITY), wmax_f(ok ? v.z : -INFINITY), 0.f);
    if (lane_id() == 0) box_put(box_shift(B, box_base[k]), q0 / BVH_LEAF, b);
}

// one block per node: the levels above the leaves
__global__ void __launch_bounds__(256) k_bvh_build(LevelBufs L, NodeArrays nd, const int64_t *box_base, BoxStore B)
{
    const int k = blockIdx.x;
    if (k >= L.K) return;
    const int node = L.list[k], n = nd.count[node];
    const int nl = (int)ceil_div(n, BVH_LEAF);
    const BoxStore bx = box_shift(B, box_base[k]);
    const int H = bvh_levels(nl);
    int64_t off_prev = 0, off = nl;
    int cprev = nl;
    for (int h = 1; h < H; h++) {
        const int cnt = (cprev + 31) >> BVH_LOG;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            Box6 b = box_get(bx, off_prev + 32 * i);
            const int e = min(cprev, 32 * i + 32);
            for (int c = 32 * i + 1; c < e; c++) box_merge(b, box_get(bx, off_prev + c));
            box_put(bx, off + i, b);
        }
        __syncthreads();
        off_prev = off;
        off += cnt;
        cprev = cnt;
    }
}

__device__ __forceinline__ float point_box_d2(float4 p, float4 v, const Box6 &b, const Metric6 &m)
{
    float gx = fmaxf(0.f, fmaxf(b.plo.x - p.x, p.x - b.phi.x)), gy = fmaxf(0.f, fmaxf(b.plo.y - p.y, p.y - b.phi.y)),
          gz = fmaxf(0.f, fmaxf(b.plo.z - p.z, p.z - b.phi.z));
    float gu = fmaxf(0.f, fmaxf(b.vlo.x - v.x, v.x - b.vhi.x)), gv = fmaxf(0.f, fmaxf(b.vlo.y - v.y, v.y - b.vhi.y)),
          gw = fmaxf(0.f, fmaxf(b.vlo.z - v.z, v.z - b.vhi.z));
    return (gx * gx + gy * gy + gz * gz) * m.ax + (gu * gu + gv * gv + gw * gw) * m.av;
}

// A node's hierarchy: its boxes and, per level, the first box (off) and the
// box count (cnt).  The two small per-level tables live in shared memory
// the caller provides (2 BVH_MAXH ints): the searches index them by a
// run-time level, which from registers would put them in local memory.
struct BvhView {
    BoxStore S;
    int nl, H;
    const int *off;
    const int *cnt;
};

__device__ __forceinline__ void bvh_fill(int *lv, int nl)
{
    int o = 0, c = nl;
    for (int h = 0; h < BVH_MAXH; h++) {
        lv[h] = o;
        lv[BVH_MAXH + h] = c;
        o += c;
        c = (c + 31) >> BVH_LOG;
    }
}

__device__ __forceinline__ void bvh_set(BvhView &V, const BoxStore &B, int64_t base, int n, const int *lv)
{
    V.S = box_shift(B, base);
    V.nl = (int)ceil_div(n, BVH_LEAF);
    V.H = min(bvh_levels(V.nl), BVH_MAXH);  // n <= 2^26 members per node (checked on the host): H <= 6
    V.off = lv;
    V.cnt = lv + BVH_MAXH;
}

// the view for a whole warp; lv is the warp's own shared table
__device__ __forceinline__ void bvh_view(BvhView &V, const BoxStore &B, int64_t base, int n, int *lv)
{
    if (lane_id() == 0) bvh_fill(lv, (int)ceil_div(n, BVH_LEAF));
    __syncwarp();
    bvh_set(V, B, base, n, lv);
}

// ---- dense boxes at the linking length ----
// A box whose float32 diameter under the node's metric is at most
// l^2 (1 - 2^-17) holds only mutual friends (the float32 diameter is within
// 8 ulps of the exact one), so all its members are joined once and a query
// that reaches the whole box within the same margin joins it with a single
// union.  These pairs lie strictly inside the linking length, never in the
// tie band.  The flag is kept in the box store's flag byte.
#define RS_CLIQUE_MARGIN 0.99999237060546875  // 1 - 2^-17

// linking limits of one node: float32 band edges around l^2 (decided in
// float64 inside them), the reporting band for ties, and the pruning radius
struct LinkLim {
    float lo, hi, tlo, thi, part, lim, cl_lim;
    double l2, l;
};

__device__ __forceinline__ LinkLim link_lim(double l2)
{
    LinkLim r;
    r.l2 = l2;
    r.l = sqrt(l2);
    r.lo = (float)(l2 * (1.0 - RS_BAND));
    r.hi = (float)(l2 * (1.0 + RS_BAND));
    r.tlo = (float)(l2 * (1.0 - 3e-6));
    r.thi = (float)(l2 * (1.0 + 3e-6));
    r.part = fmaxf(r.hi, r.thi);
    r.lim = r.part * RS_PRUNE_SLACK;
    r.cl_lim = (float)(l2 * RS_CLIQUE_MARGIN);
    return r;
}

__device__ __forceinline__ float box_diam2(const Box6 &b, const Metric6 &m)
{
    float ex = b.phi.x - b.plo.x, ey = b.phi.y - b.plo.y, ez = b.phi.z - b.plo.z;
    float eu = b.vhi.x - b.vlo.x, ev = b.vhi.y - b.vlo.y, ew = b.vhi.z - b.vlo.z;
    return (ex * ex + ey * ey + ez * ez) * m.ax + (eu * eu + ev * ev + ew * ew) * m.av;
}

__device__ __forceinline__ float point_box_far2(float4 p, float4 v, const Box6 &b, const Metric6 &m)
{
    float fx = fmaxf(p.x - b.plo.x, b.phi.x - p.x), fy = fmaxf(p.y - b.plo.y, b.phi.y - p.y),
          fz = fmaxf(p.z - b.plo.z, b.phi.z - p.z);
    float fu = fmaxf(v.x - b.vlo.x, b.vhi.x - v.x), fv = fmaxf(v.y - b.vlo.y, b.vhi.y - v.y),
          fw = fmaxf(v.z - b.vlo.z, b.vhi.z - v.z);
    return (fx * fx + fy * fy + fz * fz) * m.ax + (fu * fu + fv * fv + fw * fw) * m.av;
}

// One block per node, once the linking length is known.  The boxes are
// rebuilt over the members that can have a friend (nearest-neighbour value
// within reach; the link search skips the others as candidates and as
// queries), which drops the phase-space outliers that stretch them.  A box
// whose members all can have a friend and whose diameter is within the
// clique margin is flagged, and the members of every maximal flagged box (a
// flagged box whose parent is not flagged) are joined.
__global__ void __launch_bounds__(256) k_bvh_linkbox(LevelBufs L, NodeArrays nd, const int64_t *box_base, BoxStore B,
                                                     const float4 *wpos, const float4 *wvel, const float *dnn,
                                                     int *parent, rs_dev_status *st)
{
    const int k = blockIdx.x;
    if (k >= L.K) return;
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const Metric6 met = L.met[k];
    const LinkLim lm = link_lim(L.l2[k]);
    const float lim = (float)(L.l2[k] * RS_CLIQUE_MARGIN);
    __shared__ int lv_s[2 * BVH_MAXH];
    if (threadIdx.x == 0) bvh_fill(lv_s, (int)ceil_div(n, BVH_LEAF));
    __syncthreads();
    BvhView V;
    bvh_set(V, B, box_base[k], n, lv_s);
    // leaves; the flag holds "every member can have a friend" until the end
    for (int i = threadIdx.x; i < V.nl; i += blockDim.x) {
        Box6 b = box_empty();
        bool all = true;
        const int e = min(n, (i + 1) * BVH_LEAF);
        for (int m = i * BVH_LEAF; m < e; m++) {
            if (dnn[first + m] <= lm.part)
                box_add(b, wpos[first + m], wvel[first + m]);
            else
                all = false;
        }
        box_put(V.S, i, b);
        V.S.cl[i] = all ? 1 : 0;
    }
    __syncthreads();
    for (int h = 1; h < V.H; h++) {
        const int cprev = V.cnt[h - 1];
        for (int i = threadIdx.x; i < V.cnt[h]; i += blockDim.x) {
            Box6 b = box_get(V.S, V.off[h - 1] + 32 * i);
            bool all = V.S.cl[V.off[h - 1] + 32 * i] != 0;
            const int e = min(cprev, 32 * i + 32);
            for (int c = 32 * i + 1; c < e; c++) {
                box_merge(b, box_get(V.S, V.off[h - 1] + c));
                all = all && V.S.cl[V.off[h - 1] + c] != 0;
            }
            box_put(V.S, V.off[h] + i, b);
            V.S.cl[V.off[h] + i] = all ? 1 : 0;
        }
        __syncthreads();
    }
    const int total = V.off[V.H - 1] + 1;
    for (int b = threadIdx.x; b < total; b += blockDim.x)
        if (V.S.cl[b] && !(box_diam2(box_get(V.S, b), met) <= lim)) V.S.cl[b] = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        if (!V.S.cl[b]) continue;
        int h = 0;
        while (h + 1 < V.H && V.off[h + 1] <= b) h++;
        const int i = b - V.off[h];
        if (h + 1 < V.H && V.S.cl[V.off[h + 1] + (i >> BVH_LOG)]) continue;  // not maximal
        const int m0 = (int)bvh_m0(h, i), m1 = (int)min((int64_t)n, bvh_m0(h, i + 1));
        for (int m = m0 + 1; m < m1; m++) uf_union(parent, first + m0, first + m, st);
    }
}

// ---- warp-per-query search over the 32-ary hierarchy ----
// One query at a time per warp.  Opening a box, lane c bounds the query's
// distance to child box c (a float32 point-to-box gap, within 8 ulps of the
// exact one; a box is skipped only when the bound exceeds the radius by
// 2^-18, so no member that could change a float32 result is skipped).
// Scanning a leaf, lane c evaluates member c and the warp minimum (redux on
// the bit patterns, which order like the non-negative floats) updates the
// radius.  The leaves under an opened box are scanned nearest first and
// re-tested as the radius shrinks; needed inner boxes are pushed on a
// shared-memory stack all at once, each with its bound, the nearest on top.
constexpr int W_WARPS = 8;    // warps per block of the search kernels
constexpr int W_STACK = 192;  // stack entries per warp: at most 31 pending per level
constexpr unsigned FULLW = 0xffffffffu;

__device__ __forceinline__ unsigned ford(float x) { return __float_as_uint(x); }

__device__ __forceinline__ float wmin(float x) { return __uint_as_float(__reduce_min_sync(FULLW, ford(x))); }

__device__ __forceinline__ float4 shfl4(float4 a, int src)
{
    return make_float4(__shfl_sync(FULLW, a.x, src), __shfl_sync(FULLW, a.y, src), __shfl_sync(FULLW, a.z, src), 0.f);
}

struct WarpJobs {
    const int *rank;  // per warp job: node rank
    const int *q0;    // first member of the job's 32 queries (a multiple of 32)
    const int *out;   // where the first query's result goes (query j writes out + j)
    int64_t count;
};

// Nearest-neighbour distance of member q (coordinates pq, vq) among the
// node's members P, Q (n of them), starting from the radius `best` (the own
// leaf `own` already scanned).  Returns as soon as the radius drops below
// `stop`.  `best` is warp-uniform throughout.
__device__ __forceinline__ float w32_nn(const BvhView &V, const MemberStore &M, int n, int q, float4 pq, float4 vq,
                        const Metric6 &met, float best, float stop, int own, int *si, float *sd, rs_dev_status *st,
                        int node)
{
    const int lane = lane_id();
    if (V.H < 2 || best < stop) return best;
    if (lane == 0) {
        si[0] = (V.H - 1) << 24;
        sd[0] = 0.f;
    }
    int sp = 1;
    __syncwarp();
    for (int it = 0; sp > 0 && it < (1 << 24); it++) {
        sp--;
        const int ent = si[sp];
        const float elb = sd[sp];
        __syncwarp();
        if (elb > best * RS_PRUNE_SLACK) continue;
        const int ch = (ent >> 24) - 1, i = ent & 0xffffff;
        const int c = 32 * i + lane;
        const bool ok = c < V.cnt[ch] && !(ch == 0 && c == own);
        const float lb = ok ? point_box_d2(pq, vq, box_get(V.S, V.off[ch] + c), met) : INFINITY;
        unsigned mask = __ballot_sync(FULLW, ok && lb <= best * RS_PRUNE_SLACK);
        if (ch == 0) {
            // the two nearest needed leaves at a time (their loads overlap)
            while (mask) {
                bool mine = (mask >> lane) & 1u;
                unsigned key = mine ? ford(lb) : 0xffffffffu;
                unsigned mn = __reduce_min_sync(FULLW, key);
                const int s0 = __ffs(__ballot_sync(FULLW, mine && key == mn)) - 1;
                mask &= ~(1u << s0);
                int s1 = -1;
                if (mask) {
                    mine = (mask >> lane) & 1u;
                    key = mine ? ford(lb) : 0xffffffffu;
                    mn = __reduce_min_sync(FULLW, key);
                    s1 = __ffs(__ballot_sync(FULLW, mine && key == mn)) - 1;
                    mask &= ~(1u << s1);
                }
                const int m0 = (32 * i + s0) * BVH_LEAF + lane, m1 = (32 * i + s1) * BVH_LEAF + lane;
                const bool v0 = m0 < n && m0 != q, v1 = s1 >= 0 && m1 < n && m1 != q;
                float4 p0 = make_float4(0, 0, 0, 0), u0 = p0, p1 = p0, u1 = p0;
                if (v0) mem_get(M, m0, p0, u0);
                if (v1) mem_get(M, m1, p1, u1);
                float d = v0 ? d2_32(pq, vq, p0, u0, met) : INFINITY;
                if (v1) d = fminf(d, d2_32(pq, vq, p1, u1, met));
                best = fminf(best, wmin(d));
                if (best < stop) return best;
                mask &= __ballot_sync(FULLW, lb <= best * RS_PRUNE_SLACK);
            }
            continue;
        }
        if (sp + __popc(mask) > W_STACK) {
            if (lane == 0) dev_fail(st, DEV_OVERFLOW, 54, node);
            return best;
        }
        if (mask) {
            const bool mine = (mask >> lane) & 1u;
            const int cntm = __popc(mask);
            if (mine) {
                const int slot = sp + __popc(mask & ((1u << lane) - 1u));
                si[slot] = (ch << 24) | c;
                sd[slot] = lb;
            }
            const unsigned key = mine ? ford(lb) : 0xffffffffu;
            const unsigned mn = __reduce_min_sync(FULLW, key);
            const int src = __ffs(__ballot_sync(FULLW, mine && key == mn)) - 1;
            const int top = sp + cntm - 1, from = sp + __popc(mask & ((1u << src) - 1u));
            __syncwarp();
            if (lane == 0 && from != top) {
                const int e0 = si[from];
                const float d0 = sd[from];
                si[from] = si[top];
                sd[from] = sd[top];
                si[top] = e0;
                sd[top] = d0;
            }
            sp += cntm;
        }
        __syncwarp();
    }
    return best;
}

// nearest-neighbour distances, one warp per job of 32 consecutive members
// (one leaf): the leaf is held in registers, one member per lane, and its 32
// queries are searched one after another.  Blocks are of NN_WARPS warps, so a
// slot frees as soon as its few warps end.
constexpr int NN_WARPS = 4;
template <int MINB>
__global__ void __launch_bounds__(NN_WARPS * 32, MINB * W_WARPS / NN_WARPS)
    k_bvh_nn(LevelBufs L, WarpJobs J, NodeArrays nd, const int64_t *box_base, BoxStore B, MemberStore MS,
             const float *R2, const float *STOP, int redo_failed, float *out, rs_dev_status *st)
{
    __shared__ int si_s[NN_WARPS][W_STACK];
    __shared__ float sd_s[NN_WARPS][W_STACK];
    __shared__ int lv_s[NN_WARPS][2 * BVH_MAXH];
    const int w = warp_id(), lane = lane_id();
    const int64_t gw = (int64_t)blockIdx.x * NN_WARPS + w;
    if (gw >= J.count) return;
    const int k = J.rank[gw], q0 = J.q0[gw];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    if (q0 >= n) return;
    const Metric6 met = L.met[k];
    BvhView V;
    bvh_view(V, B, box_base[k], n, lv_s[w]);
    const MemberStore M = mem_shift(MS, first);
    // start from the node's radius when one is given (just above it, so a
    // result at or above the start means "nothing within the radius"); a
    // query whose radius falls below the stop value is done: its member is
    // certainly below the linking length and its exact value is not needed.
    // With redo_failed, only the nodes whose bracket failed (R2 = -1) are
    // searched again, unbounded.
    float start = INFINITY, stop = 0.f;
    if (redo_failed) {
        if (!(R2[k] < 0.f)) return;
    } else {
        start = R2 ? R2[k] * 1.00000095367431640625f : INFINITY;
        stop = STOP ? STOP[k] : 0.f;
    }
    const int own = q0 / BVH_LEAF;
    const int mo = q0 + lane;
    const bool have = mo < n;
    float4 po = make_float4(0, 0, 0, 0), vo = po;
    if (have) mem_get(M, mo, po, vo);
    const int nq = min(32, n - q0);
    float res = INFINITY;
    for (int j = 0; j < nq; j++) {
        const float4 pq = shfl4(po, j), vq = shfl4(vo, j);
        const float d = (have && lane != j) ? d2_32(pq, vq, po, vo, met) : INFINITY;
        float best = fminf(start, wmin(d));
        best = w32_nn(V, M, n, q0 + j, pq, vq, met, best, stop, own, si_s[w], sd_s[w], st, node);
        if (lane == j) res = best;
    }
    if (have) out[J.out[gw] + lane] = res >= start ? INFINITY : res;
}

// nearest-neighbour distance of single sampled members, one warp each
__global__ void __launch_bounds__(W_WARPS * 32) k_bvh_nn_sample(LevelBufs L, NodeArrays nd, const int64_t *box_base,
                                                                BoxStore B, MemberStore MS, const int64_t *soff,
                                                                float *out, rs_dev_status *st)
{
    __shared__ int si_s[W_WARPS][W_STACK];
    __shared__ float sd_s[W_WARPS][W_STACK];
    __shared__ int lv_s[W_WARPS][2 * BVH_MAXH];
    const int w = warp_id(), lane = lane_id();
    const int k = blockIdx.y;
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const int S = (int)(soff[k + 1] - soff[k]);
    const int s = blockIdx.x * W_WARPS + w;
    if (s >= S) return;
    const int q = (int)(((int64_t)s * n) / S);
    const Metric6 met = L.met[k];
    BvhView V;
    bvh_view(V, B, box_base[k], n, lv_s[w]);
    const MemberStore M = mem_shift(MS, first);
    float4 pq, vq, pm = make_float4(0, 0, 0, 0), vm = pm;
    mem_get(M, q, pq, vq);
    const int own = q / BVH_LEAF, m = own * BVH_LEAF + lane;
    if (m < n) mem_get(M, m, pm, vm);
    const float d = (m < n && m != q) ? d2_32(pq, vq, pm, vm, met) : INFINITY;
    const float best = w32_nn(V, M, n, q, pq, vq, met, wmin(d), 0.f, own, si_s[w], sd_s[w], st, node);
    if (lane == 0) out[soff[k] + s] = best;
}

// nearest-neighbour distance of listed members (rank, member), one warp
// each, unbounded; the result goes to the member's own slot
__global__ void __launch_bounds__(W_WARPS * 32) k_bvh_nn_list(LevelBufs L, NodeArrays nd, const int64_t *box_base,
                                                              BoxStore B, MemberStore MS, const int2 *qlist,
                                                              const int *qlen, int cap, float *dnn,
                                                              rs_dev_status *st)
{
    __shared__ int si_s[W_WARPS][W_STACK];
    __shared__ float sd_s[W_WARPS][W_STACK];
    __shared__ int lv_s[W_WARPS][2 * BVH_MAXH];
    const int w = warp_id(), lane = lane_id();
    const int64_t s = (int64_t)blockIdx.x * W_WARPS + w;
    if (s >= min(*qlen, cap)) return;
    const int2 e = qlist[s];
    const int k = e.x, q = e.y;
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const Metric6 met = L.met[k];
    BvhView V;
    bvh_view(V, B, box_base[k], n, lv_s[w]);
    const MemberStore M = mem_shift(MS, first);
    float4 pq, vq, pm = make_float4(0, 0, 0, 0), vm = pm;
    mem_get(M, q, pq, vq);
    const int own = q / BVH_LEAF, m = own * BVH_LEAF + lane;
    if (m < n) mem_get(M, m, pm, vm);
    const float d = (m < n && m != q) ? d2_32(pq, vq, pm, vm, met) : INFINITY;
    const float best = w32_nn(V, M, n, q, pq, vq, met, wmin(d), 0.f, own, si_s[w], sd_s[w], st, node);
    if (lane == 0) dnn[first + q] = best;
}

// one candidate pair: bit 0 set when it is within l (decided in float64
// inside the band), bit 1 set for a pair within 1e-6 (relative) of l but not
// at it
// (The float64 metric and l^2 are read from memory on the rare band path
// only, which keeps them out of the search kernel's registers.)
__device__ __forceinline__ int pair_test(const LinkLim &lm, const Metric6 &met, const Metric6 *met64,
                                         const double *l2p, float4 pa, float4 va, float4 pb, float4 vb)
{
    const float d2 = d2_32(pa, va, pb, vb, met);
    if (d2 > lm.part) return 0;
    // below both bands (the linking band and the wider tie band): a friend,
    // and not a tie-band pair
    if (d2 < fminf(lm.lo, lm.tlo)) return 1;
    const Metric6 m = *met64;
    const double l2 = *l2p, l = sqrt(l2);
    const double e64 = d2_64(pa, va, pb, vb, m);
    const int tie = (l2 > 0 && e64 != l2 && fabs(sqrt(e64) - l) <= 1e-6 * l) ? 2 : 0;
    return (e64 <= l2 ? 1 : 0) | tie;
}

// Join a and b; returns the smaller of the two roots it joined (a member of
// the merged set).
__device__ __forceinline__ int uf_union_root(int *parent, int a, int b, rs_dev_status *st)
{
    for (int it = 0; it < RS_SPIN_LIMIT; it++) {
        a = uf_find(parent, a, st);
        b = uf_find(parent, b, st);
        if (a == b) return a;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(&parent[b], b, a);
        if (old == b) return a;
        b = old;
    }
    dev_fail(st, DEV_TIMEOUT, 2, a);
    return a;
}

// Join the query's set with friend b.  `rq` is a member known to be in the
// query's set (sets only grow, so it stays one): when b's parent is rq the
// two are joined already and the union is skipped.  Dense regions give each
// query many friends whose parent is the set's root, so most unions end at
// this one load.  Returns a member of the merged set, or INT_MAX when skipped.
__device__ __forceinline__ int join_friend(int *parent, int a, int b, int rq, rs_dev_status *st)
{
    if (__ldcg(&parent[b]) == rq) return 0x7fffffff;
    return uf_union_root(parent, a, b, st);
}

// Child c = 32 i + lane of stack entry `ent` for a friends-of-friends search
// of member q: true when the child can hold a friend after q (its member
// range extends past q + 1 and its box is within reach).  A clique box wholly
// within reach is joined with one union and not searched.
__device__ __forceinline__ bool link_child(const BvhView &V, int ent, int lane, int q, int own, float4 pq, float4 vq,
                                           const Metric6 &met, const LinkLim &lm, int *parent, int first, int rq,
                                           rs_dev_status *st)
{
    if (ent < 0) return false;
    const int ch = (ent >> 24) - 1, c = 32 * (ent & 0xffffff) + lane;
    if (!(c < V.cnt[ch] && !(ch == 0 && c == own) && bvh_m0(ch, c + 1) > (int64_t)q + 1)) return false;
    const int64_t bi = V.off[ch] + c;
    const Box6 bx = box_get(V.S, bi);
    // the clique flag is loaded with the box, not after the reach test, so
    // its latency overlaps the box loads instead of following them
    const unsigned char clique = V.S.cl[bi];
    if (!(point_box_d2(pq, vq, bx, met) <= lm.lim)) return false;
    if (clique && point_box_far2(pq, vq, bx, met) <= lm.cl_lim) {
        join_friend(parent, first + q, first + (int)bvh_m0(ch, c), rq, st);
        return false;
    }
    return true;
}

constexpr int LK_STACK = 256;  // link stack entries per warp
constexpr int LK_LEAVES = 128; // pending leaves per warp
constexpr int LK_BATCH = 2;    // leaves scanned together

// Friends-of-friends pairs of member q with the members after it (outside
// its own leaf) by a whole warp; returns this lane's tie count.  The search
// pops two boxes at a time and collects the leaves within reach in a list,
// which it scans LK_BATCH leaves at a time (one member per lane and leaf), so
// several independent loads are in flight per warp.
__device__ __forceinline__ int w32_link(const BvhView &V, const MemberStore &M, const float *D, int n,
                                        int q, float4 pq, float4 vq, const Metric6 &met, const Metric6 *met64,
                                        const double *l2p, const LinkLim &lm, int own,
                                        int *parent, int first, int *si, int *lf, int &rq, rs_dev_status *st,
                                        int node)
{
    const int lane = lane_id();
    int tie = 0;
    if (V.H < 2) return 0;
    if (lane == 0) si[0] = (V.H - 1) << 24;
    int sp = 1, nl = 0;
    __syncwarp();
    const unsigned below = (1u << lane) - 1u;
    for (int it = 0; (sp > 0 || nl > 0) && it < (1 << 24); it++) {
        if (sp > 0 && nl <= LK_LEAVES - 64) {
            const int ea = si[sp - 1];
            const int eb = sp >= 2 ? si[sp - 2] : -1;
            __syncwarp();
            sp -= eb >= 0 ? 2 : 1;
            const bool na = link_child(V, ea, lane, q, own, pq, vq, met, lm, parent, first, rq, st);
            const bool nb = link_child(V, eb, lane, q, own, pq, vq, met, lm, parent, first, rq, st);
            const unsigned ma = __ballot_sync(FULLW, na), mb = __ballot_sync(FULLW, nb);
            if (sp + __popc(ma) + __popc(mb) > LK_STACK) {
                if (lane == 0) dev_fail(st, DEV_OVERFLOW, 55, node);
                return tie;
            }
            const int ents[2] = {ea, eb};
            const unsigned ms[2] = {ma, mb};
            const bool nd2[2] = {na, nb};
            for (int u = 0; u < 2; u++) {
                if (!ms[u]) continue;
                const int ch = (ents[u] >> 24) - 1, c = 32 * (ents[u] & 0xffffff) + lane;
                const int slot = __popc(ms[u] & below);
                if (ch == 0) {
                    if (nd2[u]) lf[nl + slot] = c;
                    nl += __popc(ms[u]);
                } else {
                    if (nd2[u]) si[sp + slot] = (ch << 24) | c;
                    sp += __popc(ms[u]);
                }
            }
            __syncwarp();
            continue;
        }
        // scan the collected leaves
        while (nl > 0) {
            const int kk = min(nl, LK_BATCH);
            nl -= kk;
            int mm[LK_BATCH];
#pragma unroll
            for (int u = 0; u < LK_BATCH; u++) mm[u] = u < kk ? lf[nl + u] * BVH_LEAF + lane : -1;
            __syncwarp();
            float dd[LK_BATCH];
            float4 pp[LK_BATCH], vv[LK_BATCH];
#pragma unroll
            for (int u = 0; u < LK_BATCH; u++) {
                dd[u] = INFINITY;
                if (mm[u] > q && mm[u] < n) {
                    dd[u] = D[mm[u]];
                    mem_get(M, mm[u], pp[u], vv[u]);
                }
            }
            int nr = 0x7fffffff;
#pragma unroll
            for (int u = 0; u < LK_BATCH; u++) {
                if (dd[u] <= lm.part) {
                    const int r = pair_test(lm, met, met64, l2p, pq, vq, pp[u], vv[u]);
                    tie += r >> 1;
                    if (r & 1) nr = min(nr, join_friend(parent, first + q, first + mm[u], rq, st));
                }
            }
            rq = min(rq, (int)__reduce_min_sync(FULLW, (unsigned)nr));
        }
    }
    return tie;
}

// friends-of-friends at l, one warp per leaf of 32 consecutive members, pairs
// with the candidate after the query in the node's member order; only
// members with a neighbour within reach take part.  A tile's eight warps are
// spread over blocks of LK_WARPS warps: the cost of a leaf varies widely, and
// a small block frees its slot as soon as its own few warps end instead of
// waiting for the slowest of eight.
constexpr int LK_WARPS = 2;
template <int MINB>
__global__ void __launch_bounds__(LK_WARPS * 32, MINB * (TQ / 32) / LK_WARPS)
    k_bvh_link(LevelBufs L, NodeArrays nd, const int64_t *box_base, BoxStore B, MemberStore MS, const float *dnn,
               int *parent, rs_dev_status *st)
{
    static_assert((TQ / 32) % LK_WARPS == 0, "a tile's warps fill whole blocks");
    __shared__ int si_s[LK_WARPS][LK_STACK];
    __shared__ int lf_s[LK_WARPS][LK_LEAVES];
    __shared__ int lv_s[LK_WARPS][2 * BVH_MAXH];
    const int w = warp_id(), lane = lane_id();
    // the grid holds exactly the tiles' warps: block b takes warps
    // (b % bpt) * LK_WARPS + w of tile b / bpt
    constexpr int bpt = (TQ / 32) / LK_WARPS;
    const int tile = blockIdx.x / bpt, jw = (blockIdx.x % bpt) * LK_WARPS + w;
    const int k = L.tile_rank[tile], q0 = L.tile_q0[tile] + 32 * jw;
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    if (q0 >= n) return;
    Metric6 met;  // float32 factors only; the float64 ones are read where needed
    met.ax = L.met[k].ax;
    met.av = L.met[k].av;
    const Metric6 *met64 = L.met + k;
    const double *l2p = L.l2 + k;
    const LinkLim lm = link_lim(L.l2[k]);
    const MemberStore M = mem_shift(MS, first);
    const float *D = dnn + first;
    const int mo = q0 + lane;
    const bool have = mo < n;
    const bool act = have && D[mo] <= lm.part;
    unsigned rem = __ballot_sync(FULLW, act);
    if (!rem) return;
    float4 po = make_float4(0, 0, 0, 0), vo = po;
    if (have) mem_get(M, mo, po, vo);
    BvhView V;
    bvh_view(V, B, box_base[k], n, lv_s[w]);
    const int own = q0 / BVH_LEAF;
    int tie = 0;
    while (rem) {
        const int j = __ffs(rem) - 1;
        rem &= rem - 1;
        const int q = q0 + j;
        const float4 pq = shfl4(po, j), vq = shfl4(vo, j);
        // a member of the query's set (its parent), refined as unions report roots
        int rq = __ldcg(&parent[first + q]);
        // pairs inside the own leaf, lane > j
        int nr = 0x7fffffff;
        if (lane > j && act) {
            const int r = pair_test(lm, met, met64, l2p, pq, vq, po, vo);
            tie += r >> 1;
            if (r & 1) nr = join_friend(parent, first + q, first + mo, rq, st);
        }
        rq = min(rq, (int)__reduce_min_sync(FULLW, (unsigned)nr));
        tie += w32_link(V, M, D, n, q, pq, vq, met, met64, l2p, lm, own, parent, first, si_s[w], lf_s[w], rq, st,
                        node);
    }
    tie = warp_sum(tie);
    if (lane == 0 && tie) atomicAdd(&L.tie[k], tie);
}

// ---- sampled bracket for the nearest-neighbour search ----
// The exact nearest-neighbour distances of an evenly spread sample of a
// node's members give a radius t_hi that lies above the node's f-quantile
// with overwhelming probability (five binomial standard deviations).  The
// search for every member then starts from t_hi instead of infinity: members
// with a neighbour within t_hi get their exact float32 distance, the others
// stop early with "none within t_hi".  Only values up to the k-th are needed
// for the linking length; if the k-th value is not within t_hi the level
// falls back to the unbounded search, so the result is always exact.
constexpr int SMP_MAX = 1024;       // sample size per node
// (nodes of at most rs_tuning::bracket_min members, 4096 by default, are
// searched without a bracket)

// (nodes that draw a member subset for the linking length search only the
// subset, without a bracket)
__global__ void k_smp_prep(const int *list, int K, NodeArrays nd, int64_t *ns, int sub_n, int min_node)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int n = nd.count[list[k]];
    ns[k] = (n > min_node && !(sub_n > 0 && n > sub_n)) ? SMP_MAX : 0;
}

// full-search warp jobs: every 32 consecutive members of every node
__global__ void k_full_jobs(const int *list, int K, NodeArrays nd, const int64_t *woff, int *jrank, int *jq0,
                            int *jout)
{
    const int k = blockIdx.x;
    if (k >= K) return;
    const int node = list[k], first = nd.first[node];
    const int64_t a = woff[k], c = woff[k + 1] - woff[k];
    for (int64_t j = threadIdx.x; j < c; j += blockDim.x) {
        jrank[a + j] = k;
        jq0[a + j] = (int)(32 * j);
        jout[a + j] = first + (int)(32 * j);
    }
}

// warp jobs of 32 members per node; none for a node above the subset size
// (sub_n > 0), whose subset members are searched one by one instead
__global__ void k_full_prep(const int *list, int K, NodeArrays nd, int64_t *nw, int sub_n)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int n = nd.count[list[k]];
    nw[k] = (sub_n > 0 && n > sub_n) ? 0 : ceil_div(n, 32);
}

// bracket of the search from the sample: the radius R2 is the sample's
// quantile at f + 5 sigma widened by 16 band widths; the stop value is the
// quantile at f - 5 sigma narrowed by 16 band widths (a member with a
// neighbour closer than it is certainly below the linking length)
__global__ void k_smp_thresh(LevelBufs L, NodeArrays nd, const int64_t *soff, const float *sdnn, double f,
                             float *R2, float *STOP)
{
    __shared__ float v[SMP_MAX];
    const int k = blockIdx.x;
    if (k >= L.K) return;
    const int64_t a = soff[k];
    const int S = (int)(soff[k + 1] - a);
    for (int i = threadIdx.x; i < SMP_MAX; i += blockDim.x) v[i] = i < S ? sdnn[a + i] : INFINITY;
    __syncthreads();
    for (int kk = 2; kk <= SMP_MAX; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < SMP_MAX / 2; t += blockDim.x) {
                int i = 2 * j * (t / j) + (t % j), l = i + j;
                bool up = (i & kk) == 0;
                float x = v[i], y = v[l];
                if ((x > y) == up) {
                    v[i] = y;
                    v[l] = x;
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        if (S == 0) {  // not sampled: unbounded search, no early stop
            R2[k] = INFINITY;
            STOP[k] = 0.f;
        } else {
            const double sd = 5.0 * sqrt(f * (1.0 - f) / (double)S);
            long long hi = (long long)ceil(fmin(1.0, f + sd) * (double)S) - 1;
            long long lo = (long long)ceil(fmax(0.0, f - sd) * (double)S) - 2;
            hi = hi < 0 ? 0 : (hi >= S ? S - 1 : hi);
            const float th = v[hi];
            R2[k] = isinf(th) ? INFINITY : (float)((double)th * (1.0 + 16.0 * RS_BAND));
            STOP[k] = lo < 0 ? 0.f : (float)((double)v[lo] * (1.0 - 16.0 * RS_BAND));
        }
    }
}

// the level falls back to the full search when the float32 band around a
// node's k-th value is not inside (stop, radius)
// A node whose bracket did not hold gets R2 = -1: the fallback search
// redoes that node only (force_odd, from the injected fault
// RS_FAULT=bracket, fails every node of odd rank that has a bracket).
__global__ void k_bracket_check(LevelBufs L, float *R2, const float *STOP, int *fallback, int force_odd)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.K) return;
    // the whole float32 band around the k-th value must lie inside the radius,
    // so no member that belongs in the band was cut off by it
    const float t32 = __uint_as_float(L.sel_prefix[k]);
    bool fail = !((double)t32 * (1.0 + 4.0 * RS_BAND) <= (double)R2[k]) ||
                !((double)t32 * (1.0 - 4.0 * RS_BAND) >= (double)STOP[k]);
    if (force_odd && (k & 1) && !isinf(R2[k])) fail = true;
    if (fail) {
        R2[k] = -1.f;
        atomicExch(fallback, 1);
    }
}

// ---- big-node member order: k-d splits at leaf-aligned medians ----
// A node's member range is split recursively: a range of m > 32 members
// splits at h = m/2 rounded up to a multiple of 32, the h members with the
// smallest coordinate on the round's axis going left, the axes cycling
// through x, vx, y, vy, z, vz.  Every split lands on a leaf boundary, so each
// leaf of 32 consecutive members is one cell of the k-d tree: compact in
// phase space, which is what the leaf boxes of the searches need.  The split
// positions depend only on the node's size, so each round is one stable sort
// of all members by (segment, 16-bit coordinate), the coordinate relative to
// the node's reference member in units of its dispersion.
__host__ __device__ __forceinline__ int kd_split(int m)
{
    int h = ((m / 2 + 31) / 32) * 32;
    h = h < 32 ? 32 : h;
    return h > m - 1 ? m - 1 : h;
}

// splits until a range of m members is at most `limit`
__host__ __device__ __forceinline__ int kd_rounds(int64_t m, int limit)
{
    int r = 0;
    while (m > limit) {
        m = kd_split((int)m);
        r++;
    }
    return r;
}

constexpr int KD_CTA = 1024;  // ranges of at most this many members finish in one CTA

// 16-bit coordinate of a member on an axis (x, vx, y, vy, z, vz), relative to
// the node's reference member in units of its dispersion
__device__ __forceinline__ unsigned kd_coord(const float4 *wpos, const float4 *wvel, unsigned slot, int axis,
                                             float4 pref, float4 vref, float ix, float iv)
{
    const int d = axis >> 1;
    float c, r, inv;
    if ((axis & 1) == 0) {
        const float4 a = wpos[slot];
        c = d == 0 ? a.x : (d == 1 ? a.y : a.z);
        r = d == 0 ? pref.x : (d == 1 ? pref.y : pref.z);
        inv = ix;
    } else {
        const float4 a = wvel[slot];
        c = d == 0 ? a.x : (d == 1 ? a.y : a.z);
        r = d == 0 ? vref.x : (d == 1 ? vref.y : vref.z);
        inv = iv;
    }
    const float u = ((c - r) * inv + 12.f) * (65536.f / 24.f);
    return (unsigned)fminf(fmaxf(u, 0.f), 65535.f);
}

// One global round over the nodes still being split (act_off: their members'
// offsets in the round's compact arrays; equal neighbours mark a node that is
// done): ranges of more than KD_CTA members at this depth are sorted by the
// round's axis; smaller ranges keep their order (value 0).  vcur holds every
// member's slot in the current order.
__global__ void k_kd_keys(LevelBufs L, NodeArrays nd, const int64_t *seg_base, const int64_t *act_off,
                          const float4 *wpos, const float4 *wvel, const unsigned *vcur, unsigned long long *kout,
                          unsigned *vout, int round, int key32)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], n = nd.count[node];
    const int p = q0 + threadIdx.x;
    if (p >= n || act_off[k + 1] == act_off[k]) return;
    const int64_t A = act_off[k] + p;
    const unsigned slot = vcur[L.seg_off[k] + p];
    int start = 0, size = n;
    for (int i = 0; i < round && size > KD_CTA; i++) {
        const int h = kd_split(size);
        if (p - start < h) {
            size = h;
        } else {
            start += h;
            size -= h;
        }
    }
    unsigned qv = 0;
    if (size > KD_CTA) {
        const float ix = nd.sigx[node] > 0 ? (float)(1.0 / nd.sigx[node]) : 0.f;
        const float iv = nd.sigv[node] > 0 ? (float)(1.0 / nd.sigv[node]) : 0.f;
        qv = kd_coord(wpos, wvel, slot, round % 6, L.ref[2 * k], L.ref[2 * k + 1], ix, iv);
    }
    // Key: (block of KD_CTA members holding the range's start, coordinate).
    // A range still being split has more than KD_CTA members, so it is the
    // only such range whose start lies in its block, and a later range starts
    // in a later block; ranges already final (coordinate 0) that share the
    // block lie before it and keep their places under the stable sort.  So
    // the block number separates what must stay apart, with 5 fewer bits
    // than a leaf number.
    const unsigned long long key = ((unsigned long long)(seg_base[k] + start / KD_CTA) << 16) | qv;
    if (key32)
        ((unsigned *)kout)[A] = (unsigned)key;
    else
        kout[A] = key;
    vout[A] = slot;
}

// the round's sorted slots back to their nodes' places in the current order
__global__ void k_kd_back(LevelBufs L, NodeArrays nd, const int64_t *act_off, const unsigned *vs, unsigned *vcur)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int n = nd.count[L.list[k]];
    const int p = q0 + threadIdx.x;
    if (p >= n || act_off[k + 1] == act_off[k]) return;
    vcur[L.seg_off[k] + p] = vs[act_off[k] + p];
}

// the current order before the rounds: every member in its own place
__global__ void k_kd_init(LevelBufs L, NodeArrays nd, unsigned *vcur)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], n = nd.count[node];
    const int p = q0 + threadIdx.x;
    if (p < n) vcur[L.seg_off[k] + p] = (unsigned)(nd.first[node] + p);
}

// Nodes still being split in round r (their largest range at depth r, the
// first, has more than KD_CTA members): blocks of KD_CTA members (the range
// keys) and members; 0 for the others, which sit the round out.
__global__ void k_kd_active(const int *list, int K, NodeArrays nd, int round, int64_t *nb, int64_t *na)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int n = nd.count[list[k]];
    const bool act = kd_rounds(n, KD_CTA) > round;
    nb[k] = act ? ceil_div(n, KD_CTA) : 0;
    na[k] = act ? n : 0;
}

// Ranges of at most KD_CTA members left by the global rounds, one entry per
// range: (rank, start in the node, size, depth).  One thread per node.
__global__ void k_kd_ranges(LevelBufs L, NodeArrays nd, int4 *ranges, int *count, int cap, rs_dev_status *st)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.K) return;
    const int n = nd.count[L.list[k]];
    int stk_s[32], stk_m[32], stk_d[32];
    int sp = 0;
    stk_s[0] = 0;
    stk_m[0] = n;
    stk_d[0] = 0;
    sp = 1;
    for (int it = 0; sp > 0 && it < (1 << 26); it++) {
        sp--;
        const int s0 = stk_s[sp], m = stk_m[sp], d = stk_d[sp];
        if (m <= KD_CTA) {
            if (m > 32) {
                const int slot = atomicAdd(count, 1);
                if (slot < cap) ranges[slot] = make_int4(k, s0, m, d);
                else dev_fail(st, DEV_OVERFLOW, 58, slot);
            }
            continue;
        }
        if (sp + 2 > 32) {
            dev_fail(st, DEV_OVERFLOW, 59, k);
            return;
        }
        const int h = kd_split(m);
        stk_s[sp] = s0 + h;
        stk_m[sp] = m - h;
        stk_d[sp++] = d + 1;
        stk_s[sp] = s0;
        stk_m[sp] = h;
        stk_d[sp++] = d + 1;
    }
}

// Finish one range in shared memory: the remaining splits.  Round r orders
// every sub-range of more than 32 members (at depth r) along the round's axis,
// which puts its leaf-aligned median split in place, as the global rounds do.
// The members' ranks along each axis the range uses come first, from a
// stable two-pass radix sort of their 16-bit coordinates (ties keep the
// order the range came in); a round then moves member e of sub-range s to s's
// start plus the number of s's members of smaller rank, counted from a
// bitmap of the ranks per sub-range and its prefix popcounts.
constexpr int KDF_ROUNDS = 5;   // kd_rounds(KD_CTA, 32)
constexpr int KDF_SUB = 16;     // sub-ranges ordered in the last round
static_assert(KD_CTA == 8 * 128, "eight warps of 128 positions rank a range");

// stable radix ranking of key[0..m) (16-bit): rk[e] = position of element e
// in the sorted order (8 warps, positions 128 w .. 128 w + 127 per warp)
__device__ __forceinline__ void kdf_rank(int m, const unsigned short *key, unsigned short *rk,
                                         unsigned short (*ord)[KD_CTA], unsigned short (*wcnt)[256],
                                         unsigned *dstart, unsigned *wsum)
{
    const int tid = threadIdx.x, lane = lane_id(), w = warp_id();
    const unsigned lt = (1u << lane) - 1u;
    for (int i = tid; i < m; i += blockDim.x) ord[0][i] = (unsigned short)i;
    int cur = 0;
    for (int sh = 0; sh < 16; sh += 8) {
        for (int i = tid; i < 8 * 256; i += blockDim.x) wcnt[i >> 8][i & 255] = 0;
        __syncthreads();
        unsigned dd[4], rr[4], ee[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int pos = 128 * w + 32 * j + lane;
            const bool ok = pos < m;
            const unsigned e = ok ? ord[cur][pos] : 0u;
            const unsigned d = ok ? ((unsigned)key[e] >> sh) & 255u : 256u;
            const unsigned peers = __match_any_sync(FULLW, d);
            const unsigned before = ok ? wcnt[w][d] : 0u;
            __syncwarp();
            if (ok && (peers & lt) == 0) wcnt[w][d] = (unsigned short)(before + __popc(peers));
            __syncwarp();
            dd[j] = d;
            rr[j] = before + __popc(peers & lt);
            ee[j] = e;
        }
        __syncthreads();
        {
            // thread d: offsets of the warps within digit d, then digit d's start
            const int d = tid;
            unsigned tot = 0;
#pragma unroll
            for (int ww = 0; ww < 8; ww++) {
                const unsigned t = wcnt[ww][d];
                wcnt[ww][d] = (unsigned short)tot;
                tot += t;
            }
            unsigned x = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(FULLW, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[w] = x;
            __syncthreads();
            unsigned pre = 0;
            for (int ww = 0; ww < w; ww++) pre += wsum[ww];
            dstart[d] = pre + x - tot;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (dd[j] < 256u) ord[cur ^ 1][dstart[dd[j]] + wcnt[w][dd[j]] + rr[j]] = (unsigned short)ee[j];
        __syncthreads();
        cur ^= 1;
    }
    for (int i = tid; i < m; i += blockDim.x) rk[ord[cur][i]] = (unsigned short)i;
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_kd_finish(LevelBufs L, NodeArrays nd, const int4 *ranges, const int *count,
                                                     const float4 *wpos, const float4 *wvel, unsigned *vals)
{
    __shared__ unsigned slot[KD_CTA];
    __shared__ unsigned short rk[KDF_ROUNDS][KD_CTA];
    __shared__ unsigned short key[KD_CTA];
    __shared__ unsigned short pm[2][KD_CTA];  // ranking order, then position -> element
    __shared__ unsigned short wcnt[8][256];
    __shared__ unsigned dstart[256];
    __shared__ unsigned wsum[8];
    __shared__ unsigned bm[KDF_SUB][32];
    __shared__ unsigned short pre[KDF_SUB][32];
    const int tid = threadIdx.x, lane = lane_id(), w = warp_id();
    const int nr = *count;
    for (int ri = blockIdx.x; ri < nr; ri += gridDim.x) {
        const int4 rg = ranges[ri];
        const int k = rg.x, s0 = rg.y, m = rg.z, d0 = rg.w;
        const int node = L.list[k];
        const int64_t P0 = L.seg_off[k] + s0;
        const float ix = nd.sigx[node] > 0 ? (float)(1.0 / nd.sigx[node]) : 0.f;
        const float iv = nd.sigv[node] > 0 ? (float)(1.0 / nd.sigv[node]) : 0.f;
        const float4 pref = L.ref[2 * k], vref = L.ref[2 * k + 1];
        const int R = kd_rounds(m, 32);
        for (int i = tid; i < m; i += blockDim.x) slot[i] = vals[P0 + i];
        __syncthreads();
        for (int r = 0; r < R; r++) {
            const int axis = (d0 + r) % 6;
            for (int i = tid; i < m; i += blockDim.x)
                key[i] = (unsigned short)kd_coord(wpos, wvel, slot[i], axis, pref, vref, ix, iv);
            __syncthreads();
            kdf_rank(m, key, rk[r], pm, wcnt, dstart, wsum);
        }
        int cur = 0;
        for (int i = tid; i < m; i += blockDim.x) pm[0][i] = (unsigned short)i;
        for (int r = 0; r < R; r++) {
            for (int i = tid; i < KDF_SUB * 32; i += blockDim.x) bm[i >> 5][i & 31] = 0u;
            __syncthreads();
            for (int j = tid; j < m; j += blockDim.x) {
                int start = 0, size = m, sub = 0;
                for (int i = 0; i < r && size > 32; i++) {
                    const int h = kd_split(size);
                    const int hi = j - start >= h ? 1 : 0;
                    start = hi ? start + h : start;
                    size = hi ? size - h : h;
                    sub = 2 * sub + hi;
                }
                if (size > 32) {
                    const unsigned q = rk[r][pm[cur][j]];
                    atomicOr(&bm[sub][q >> 5], 1u << (q & 31));
                }
            }
            __syncthreads();
            for (int sb = w; sb < (1 << r); sb += 8) {
                const unsigned c = __popc(bm[sb][lane]);
                unsigned x = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(FULLW, x, o);
                    if (lane >= o) x += y;
                }
                pre[sb][lane] = (unsigned short)(x - c);
            }
            __syncthreads();
            for (int j = tid; j < m; j += blockDim.x) {
                int start = 0, size = m, sub = 0;
                for (int i = 0; i < r && size > 32; i++) {
                    const int h = kd_split(size);
                    const int hi = j - start >= h ? 1 : 0;
                    start = hi ? start + h : start;
                    size = hi ? size - h : h;
                    sub = 2 * sub + hi;
                }
                const unsigned short e = pm[cur][j];
                int np = j;
                if (size > 32) {
                    const unsigned q = rk[r][e];
                    np = start + pre[sub][q >> 5] + __popc(bm[sub][q >> 5] & ((1u << (q & 31)) - 1u));
                }
                pm[cur ^ 1][np] = e;
            }
            __syncthreads();
            cur ^= 1;
        }
        for (int j = tid; j < m; j += blockDim.x) vals[P0 + j] = slot[pm[cur][j]];
        __syncthreads();
    }
}

// members into the sorted order of their node's range
__global__ void k_kd_place(LevelBufs L, NodeArrays nd, const unsigned *vals, const float4 *wpos, const float4 *wvel,
                           const int *widx, float4 *wpos2, float4 *wvel2, int *widx2, unsigned *dest)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const int p = q0 + threadIdx.x;
    if (p >= n) return;
    const int64_t P = L.seg_off[k] + p;
    const unsigned s = vals[P];
    const int dd = first + p;
    wpos2[dd] = wpos[s];
    wvel2[dd] = wvel[s];
    widx2[dd] = widx[s];
    dest[P] = (unsigned)dd;
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

// ---- random member subsets for the linking length (Sec. 3.2) ----
// Above sub_n members a node takes its linking length from the nearest-
// neighbour distances of sub_n randomly drawn members (their neighbours are
// still searched among all members).  Each particle carries a 64-bit key from
// the SplitMix64 generator (Steele, Lea & Flood 2014) used counter-based:
// particle i gets the finaliser of seed + (i+1)*gamma.  The finaliser is a
// bijection, so keys are distinct and the subset -- the sub_n members with
// the smallest keys -- is well defined; it is found by a radix select on the
// key's high word, then on its low word among the members that tie on the
// high word.  Members outside the subset get a nearest-neighbour value of -1,
// which the select skips and the link treats as "may have a friend".
__device__ __forceinline__ unsigned long long subset_key(unsigned long long seed, int i)
{
    unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_sub_init(LevelBufs L, NodeArrays nd, int sub_n)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.K) return;
    const int n = nd.count[L.list[k]];
    L.sel_krem[k] = n > sub_n ? sub_n : 1;
    L.sel_prefix[k] = 0u;
    L.sub_cnt[k] = 0;
}

// one radix-select pass over the keys of the members of nodes above sub_n:
// stage 0 selects on the high word, stage 1 on the low word of the members
// whose high word equals the stage-0 result
__global__ void __launch_bounds__(TQ) k_sub_hist(LevelBufs L, NodeArrays nd, const int *widx,
                                                 unsigned long long seed, int sub_n, int stage, int pass)
{
    __shared__ unsigned h[2048];
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    if (n <= sub_n) return;  // the whole tile belongs to one node
    for (int i = threadIdx.x; i < 2048; i += TQ) h[i] = 0;
    __syncthreads();
    const int q = q0 + threadIdx.x;
    if (q < n) {
        const unsigned long long key = subset_key(seed, widx[first + q]);
        const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
        if (stage == 0 || hi == L.sub_t[2 * k]) {
            const unsigned bits = stage == 0 ? hi : lo;
            unsigned digit, mask;
            sel_digit(bits, pass, digit, mask);
            if ((bits & mask) == (L.sel_prefix[k] & mask)) atomicAdd(&h[digit], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += TQ)
        if (h[i]) atomicAdd(&L.hist[(int64_t)k * 2048 + i], h[i]);
}

// stores a stage's selected word; the rank still to select carries over
__global__ void k_sub_stage(LevelBufs L, int stage)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.K) return;
    L.sub_t[2 * k + stage] = L.sel_prefix[k];
    L.sel_prefix[k] = 0u;
}

// members of the subset go to the query list (rank, member); the others get
// the "outside the subset" value
__global__ void __launch_bounds__(TQ) k_sub_mark(LevelBufs L, NodeArrays nd, const int *widx,
                                                 unsigned long long seed, int sub_n, float *dnn, int2 *qlist,
                                                 int *qlen, int cap, rs_dev_status *st)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    if (n <= sub_n) return;
    const int q = q0 + threadIdx.x;
    bool in = false;
    if (q < n) {
        const unsigned long long key = subset_key(seed, widx[first + q]);
        const unsigned long long t = ((unsigned long long)L.sub_t[2 * k] << 32) | L.sub_t[2 * k + 1];
        in = key <= t;
        if (!in) dnn[first + q] = -1.0f;
    }
    const unsigned m = __ballot_sync(FULLW, in);
    if (!m) return;
    const int lane = lane_id();
    int base = 0;
    if (lane == __ffs(m) - 1) {
        base = atomicAdd(qlen, __popc(m));
        atomicAdd(&L.sub_cnt[k], __popc(m));
    }
    base = __shfl_sync(FULLW, base, __ffs(m) - 1);
    if (in) {
        const int pos = base + __popc(m & ((1u << lane) - 1u));
        if (pos < cap)
            qlist[pos] = make_int2(k, q);
        else
            dev_fail(st, DEV_OVERFLOW, 58, node);
    }
}

// every node above sub_n drew exactly sub_n members (keys are distinct)
__global__ void k_sub_check(LevelBufs L, NodeArrays nd, int sub_n, rs_dev_status *st)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.K) return;
    const int node = L.list[k], n = nd.count[node];
    if (n > sub_n && L.sub_cnt[k] != sub_n) dev_fail(st, DEV_INTERNAL, 59, node);
}

// number of members whose nearest-neighbour distance sets a node's linking
// length: all of them, or the subset's size above it
__device__ __forceinline__ int n_select(int n, int sub_n) { return (sub_n > 0 && n > sub_n) ? sub_n : n; }

__global__ void k_lvl_initk(LevelBufs L, NodeArrays nd, double f, int sub_n)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= L.K) return;
    const int n = n_select(nd.count[L.list[k]], sub_n);
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
        // a negative value marks a member outside the node's subset
        unsigned bits = __float_as_uint(dnn[first + q]), digit, mask;
        sel_digit(bits, pass, digit, mask);
        if (!(bits >> 31) && (bits & mask) == (L.sel_prefix[k] & mask)) atomicAdd(&h[digit], 1u);
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
    if (__float_as_uint(d) >> 31) return;  // outside the subset
    if (d < blo) {
        atomicAdd(&L.below[k], 1);
    } else if (d <= bhi) {
        int b = atomicAdd(L.band_len, 1);
        L.band_rank[b] = k;
        L.band_slot[b] = first + q;
    }
}

// Exact float64 nearest-neighbour distance of a band member: the minimum
// float64 distance over the members whose float32 distance is within `lim`
// (a bound above the member's float32 value), one warp per band member over
// the node's hierarchy.  A box is skipped only when its float32 bound exceeds
// lim by the pruning slack, so every member that passes the float32 test is
// evaluated.
__global__ void __launch_bounds__(W_WARPS * 32) k_lvl_band_exact(LevelBufs L, NodeArrays nd, const int64_t *box_base,
                                                                 BoxStore B, MemberStore MS, const float *dnn,
                                                                 rs_dev_status *st)
{
    __shared__ int si_s[W_WARPS][W_STACK];
    __shared__ int lv_s[W_WARPS][2 * BVH_MAXH];
    const int w = warp_id(), lane = lane_id();
    const int b = blockIdx.x * W_WARPS + w;
    if (b >= *L.band_len) return;
    const int k = L.band_rank[b], s = L.band_slot[b];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const Metric6 met = L.met[k];
    const MemberStore M = mem_shift(MS, first);
    const int q = s - first;
    float4 pq, vq;
    mem_get(M, q, pq, vq);
    const float lim = dnn[s] * (float)(1.0 + 2.0 * RS_BAND);
    BvhView V;
    bvh_view(V, B, box_base[k], n, lv_s[w]);
    const int own = q / BVH_LEAF;
    double best = INFINITY;
    {
        const int m = own * BVH_LEAF + lane;
        if (m < n && m != q) {
            float4 pc, vc;
            mem_get(M, m, pc, vc);
            if (d2_32(pq, vq, pc, vc, met) <= lim) best = fmin(best, d2_64(pq, vq, pc, vc, met));
        }
    }
    int *si = si_s[w];
    if (V.H >= 2) {
        if (lane == 0) si[0] = (V.H - 1) << 24;
        int sp = 1;
        __syncwarp();
        for (int it = 0; sp > 0 && it < (1 << 24); it++) {
            sp--;
            const int ent = si[sp];
            __syncwarp();
            const int ch = (ent >> 24) - 1, c = 32 * (ent & 0xffffff) + lane;
            const bool ok = c < V.cnt[ch] && !(ch == 0 && c == own) &&
                            point_box_d2(pq, vq, box_get(V.S, V.off[ch] + c), met) <= lim * RS_PRUNE_SLACK;
            unsigned mask = __ballot_sync(FULLW, ok);
            if (ch == 0) {
                while (mask) {
                    const int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int m = (32 * (ent & 0xffffff) + src) * BVH_LEAF + lane;
                    if (m < n && m != q) {
                        float4 pc, vc;
                        mem_get(M, m, pc, vc);
                        if (d2_32(pq, vq, pc, vc, met) <= lim) best = fmin(best, d2_64(pq, vq, pc, vc, met));
                    }
                }
                continue;
            }
            if (sp + __popc(mask) > W_STACK) {
                if (lane == 0) dev_fail(st, DEV_OVERFLOW, 57, node);
                break;
            }
            if (ok) si[sp + __popc(mask & ((1u << lane) - 1u))] = (ch << 24) | c;
            sp += __popc(mask);
            __syncwarp();
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(FULLW, best, o));
    if (lane == 0) L.band_val[b] = best;
}

__global__ void k_lvl_l2(LevelBufs L, NodeArrays nd, double f, int sub_n, rs_dev_status *st)
{
    const int k = blockIdx.x;
    const int node = L.list[k];
    const int n = n_select(nd.count[node], sub_n);
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

__global__ void k_lvl_comp(LevelBufs L, NodeArrays nd, const int *widx, int *parent, int *csize, int *cmin,
                           rs_dev_status *st)
{
    const int k = L.tile_rank[blockIdx.x], q0 = L.tile_q0[blockIdx.x];
    const int node = L.list[k], first = nd.first[node], n = nd.count[node];
    const int q = q0 + threadIdx.x;
    const bool ok = q < n;
    const int r = ok ? uf_find(parent, first + q, st) : -1;
    const int mi = ok ? widx[first + q] : 0x7fffffff;
    // lanes of one component add once (consecutive members mostly share a root)
    const unsigned grp = __match_any_sync(0xffffffffu, r);
    const int lead = __ffs(grp) - 1;
    const int gm = (int)__reduce_min_sync(grp, (unsigned)mi);
    if (ok && lane_id() == lead) {
        atomicAdd(&csize[r], __popc(grp));
        atomicMin(&cmin[r], gm);
    }
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
                              float4 *wpos2, float4 *wvel2, int *widx2, unsigned *dest, int rank_shift)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= LM) return;
    const int k = (int)(keys[p] >> rank_shift);
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

// the big-node nearest-neighbour search, compiled for 40, 48 or 56 resident
// warps per SM (rs_tuning::nn_blocks_per_sm = 5, 6 or 7, in units of eight)
static rs_status launch_nn(rs_ctx *ctx, const char *name, int64_t W, const LevelBufs &L, const WarpJobs &JF,
                           const NodeArrays &nd, const int64_t *bo, const BoxStore &boxes, const MemberStore &ms,
                           const float *R2, const float *STOP, int redo_failed, float *dnn)
{
    const int64_t g = ceil_div(W, NN_WARPS);
    switch (ctx->tune.nn_blocks_per_sm) {
    case 5:
        RS_LAUNCH(ctx, name, k_bvh_nn<5>, g, NN_WARPS * 32, 0, L, JF, nd, bo, boxes, ms, R2, STOP, redo_failed, dnn,
                  ctx->d_status);
        break;
    case 7:
        RS_LAUNCH(ctx, name, k_bvh_nn<7>, g, NN_WARPS * 32, 0, L, JF, nd, bo, boxes, ms, R2, STOP, redo_failed, dnn,
                  ctx->d_status);
        break;
    default:
        RS_LAUNCH(ctx, name, k_bvh_nn<6>, g, NN_WARPS * 32, 0, L, JF, nd, bo, boxes, ms, R2, STOP, redo_failed, dnn,
                  ctx->d_status);
    }
    return RS_OK;
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static rs_status refine_impl(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n, double box,
                             const int32_t *perm, const int64_t *goff, int64_t G, double f, int32_t min_n,
                             int64_t sub_n, uint64_t sub_seed, int64_t node_cap, rs_tree **out)
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
    RS_WS(ctx, int, gmisc, WS_RF_MISC0, 14 * G + 2 * M + 8);
    int *shift_bits = gmisc, *gmin = gmisc + G, *slot_group = gmisc + 2 * G, *gred = gmisc + 2 * G + M;
    // node queues: big lists (ping-pong) and the small queue; counters
    // counters first (16 ints = 64 bytes, so everything after stays 8-byte aligned)
    RS_WS(ctx, int, q, WS_RF_NODEQ, 5 * cap + 16);
    int *ctr = q, *big_a = q + 16, *big_b = q + 16 + cap, *small_q = q + 16 + 2 * cap, *tiny_q = q + 16 + 3 * cap,
        *mid_q = q + 16 + 4 * cap;
    // ctr: [0] big_a len, [1] big_b len, [2] small len, [3] small head, [4] band len,
    // [6..7] bracket fallback flag, [8] tiny len, [9] tiny head, [10] k-d ranges,
    // [11] middle len, [12] middle head, [13] subset query list length
    RS_CUDA(ctx, cudaMemsetAsync(ctr, 0, sizeof(int) * 16, ctx->stream));

    const int gb = (int)std::min<int64_t>(G, (int64_t)ctx->num_sms * 8);
    RS_LAUNCH(ctx, "rf_unwrap_init", k_fill_s32, ceil_div(12 * G, 256), 256, 0, (int32_t *)gred, 12 * G,
              (int32_t)0x7f800000);
    RS_LAUNCH(ctx, "rf_unwrap_init", k_fill_s32, ceil_div(G, 256), 256, 0, (int32_t *)gmin, G, (int32_t)0x7fffffff);
    RS_LAUNCH(ctx, "rf_group_unwrap", k_unwrap_tiles, ceil_div(M, 256), 256, 0, G, goff, perm, n, M, pos, stride,
              boxf, slot_group, gred, gmin, ctx->d_status);
    RS_LAUNCH(ctx, "rf_unwrap_bits", k_unwrap_bits, ceil_div(G, 256), 256, 0, G, (const int *)gred, boxf, shift_bits,
              ctx->d_status);
    RS_LAUNCH(ctx, "rf_gather", k_gather, ceil_div(M, 256), 256, 0, M, goff, perm, n, pos, vel, stride, boxf,
              (const int *)slot_group, (const int *)shift_bits, wpos, wvel, widx);
    RS_LAUNCH(ctx, "rf_roots", k_make_roots, ceil_div(G, 256), 256, 0, G, goff, (const int *)gmin,
              (const int *)shift_bits, (int)min_n, nd,
              big_a, ctr + 0, small_q, ctr + 2, ctx->d_status);

    // ---- big levels ----
    int *cur = big_a, *nxt = big_b;
    int *cur_len = ctr + 0, *nxt_len = ctr + 1;
    int64_t sum_level = 0;
    int n_fallback_levels = 0;
    for (int level = 0; level < 4096; level++) {
        int64_t K;
        RS_TRY(rs_read_i64(ctx, cur_len, 1, &K, "rs_refine6d"));
        K &= 0xffffffffll;
        if (K == 0) break;
        RS_WS(ctx, int64_t, lv64, WS_RF_MISC1, 4 * (K + 1) + 8);
        int64_t *tiles = lv64, *segc = lv64 + (K + 1), *tot = lv64 + 2 * (K + 1);
        RS_CUDA(ctx, cudaMemsetAsync(tot + 3, 0, sizeof(int64_t), ctx->stream));
        RS_LAUNCH(ctx, "rf_lvl_prep", k_lvl_prep, ceil_div(K, 256), 256, 0, (const int *)cur, (int)K, nd, tiles,
                  segc, (unsigned long long *)(tot + 3));
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
                     7 * sizeof(int) + sizeof(double) + 64;
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
        L.sub_t = carve<unsigned>(rp, 2 * K);
        L.sub_cnt = carve<int>(rp, K);
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
        RS_WS(ctx, uint64_t, k0, WS_SORT_K0, LM);
        RS_WS(ctx, uint64_t, k1, WS_SORT_K1, LM);
        RS_WS(ctx, uint32_t, v0, WS_SORT_V0, LM);
        RS_WS(ctx, uint32_t, v1, WS_SORT_V1, LM);
        int rbits = 0;
        while (rbits < 32 && ((uint64_t)(K - 1) >> rbits) != 0) rbits++;
        if (level < ctx->tune.kd_levels) {
            // order each big node's members by k-d splits at leaf-aligned
            // medians (levels 0-2 by default, where most of the search work
            // is); deeper levels keep this order through the stable child
            // partition below
            int64_t maxn = 0;
            RS_TRY(rs_read_i64(ctx, tot + 3, 1, &maxn, "rs_refine6d"));
            RS_WS(ctx, int64_t, kw, WS_RF_MISC5, 2 * (K + 1) + 8);
            int64_t *kseg = kw, *aoff = kw + (K + 1), *ktot = kw + 2 * (K + 1);
            RS_WS(ctx, unsigned, vcur, WS_RF_KDV, LM);
            RS_LAUNCH(ctx, "rf_kd_init", k_kd_init, T, TQ, 0, L, nd, vcur);
            // each round sorts only the members of the nodes still being
            // split, so a node costs the rounds its own size needs, not the
            // largest node's; the range keys shrink with the active blocks
            const int R = kd_rounds(maxn, KD_CTA);
            for (int r = 0; r < R; r++) {
                RS_LAUNCH(ctx, "rf_kd_active", k_kd_active, ceil_div(K, 256), 256, 0, (const int *)cur, (int)K, nd,
                          r, kseg, aoff);
                RS_CUDA(ctx, cudaMemsetAsync(kseg + K, 0, sizeof(int64_t), ctx->stream));
                RS_CUDA(ctx, cudaMemsetAsync(aoff + K, 0, sizeof(int64_t), ctx->stream));
                RS_TRY(rs_scan_i64(ctx, kseg, K + 1, ktot));
                RS_TRY(rs_scan_i64(ctx, aoff, K + 1, ktot + 1));
                int64_t tots[2];
                RS_TRY(rs_read_i64(ctx, ktot, 2, tots, "rs_refine6d"));
                const int64_t NS = tots[0], NA = tots[1];
                if (NA <= 0) break;
                int sbits = 0;
                while (sbits < 40 && (NS >> sbits) != 0) sbits++;
                // 32-bit keys (half the bytes, fewer passes) while the blocks fit in 16 bits
                const int key32 = 16 + sbits <= 32 ? 1 : 0;
                RS_LAUNCH(ctx, "rf_kd_keys", k_kd_keys, T, TQ, 0, L, nd, (const int64_t *)kseg, (const int64_t *)aoff,
                          (const float4 *)wpos, (const float4 *)wvel, (const unsigned *)vcur,
                          (unsigned long long *)k0, v0, r, key32);
                bool kalt = false;
                if (key32)
                    RS_TRY(rs_radix_sort_u32(ctx, (uint32_t *)k0, (uint32_t *)k1, v0, v1, NA, 16 + sbits, &kalt,
                                             "sort_kd"));
                else
                    RS_TRY(rs_radix_sort_u64(ctx, k0, k1, v0, v1, NA, 16 + sbits, &kalt, "sort_kd"));
                RS_LAUNCH(ctx, "rf_kd_back", k_kd_back, T, TQ, 0, L, nd, (const int64_t *)aoff,
                          (const unsigned *)(kalt ? v1 : v0), vcur);
            }
            // ranges of at most KD_CTA members finish in one CTA each
            const int64_t rcap = ceil_div(LM, 32) + K;
            RS_WS(ctx, int4, kranges, WS_RF_JOBS, rcap + 1);
            int *kcount = ctr + 10;
            RS_CUDA(ctx, cudaMemsetAsync(kcount, 0, sizeof(int), ctx->stream));
            RS_LAUNCH(ctx, "rf_kd_ranges", k_kd_ranges, ceil_div(K, 128), 128, 0, L, nd, kranges, kcount, (int)rcap,
                      ctx->d_status);
            RS_LAUNCH(ctx, "rf_kd_finish", k_kd_finish, (int64_t)ctx->num_sms * 8, 256, 0, L, nd,
                      (const int4 *)kranges, (const int *)kcount, (const float4 *)wpos, (const float4 *)wvel, vcur);
            const unsigned *vsorted = vcur;
            {
                unsigned *kdest = v0;
                RS_LAUNCH(ctx, "rf_kd_place", k_kd_place, T, TQ, 0, L, nd, vsorted, (const float4 *)wpos,
                          (const float4 *)wvel, (const int *)widx, wpos2, wvel2, widx2, kdest);
                RS_LAUNCH(ctx, "rf_lvl_copyback", k_lvl_copyback, ceil_div(LM, 256), 256, 0, LM,
                          (const unsigned *)kdest, (const float4 *)wpos2, (const float4 *)wvel2, (const int *)widx2,
                          wpos, wvel, widx);
            }
        }
        // bounding-volume hierarchy of every big node
        RS_WS(ctx, int64_t, bo, WS_RF_MISC3, (K + 1) + 8);
        RS_LAUNCH(ctx, "rf_bvh_prep", k_bvh_prep, ceil_div(K, 256), 256, 0, (const int *)cur, (int)K, nd, bo);
        RS_CUDA(ctx, cudaMemsetAsync(bo + K, 0, sizeof(int64_t), ctx->stream));
        RS_TRY(rs_scan_i64(ctx, bo, K + 1, tot + 2));
        int64_t NBX;
        RS_TRY(rs_read_i64(ctx, tot + 2, 1, &NBX, "rs_refine6d"));
        RS_WS(ctx, char, boxmem, WS_RF_HIST, NBX * 49 + 1024);
        BoxStore boxes;
        {
            char *bp2 = boxmem;
            boxes.a = carve<float4>(bp2, NBX);
            boxes.b = carve<float4>(bp2, NBX);
            boxes.c = carve<float4>(bp2, NBX);
            boxes.cl = carve<unsigned char>(bp2, NBX);
        }
        RS_WS(ctx, char, srch, WS_RF_SRCH, M * 24 + 512);
        MemberStore ms;
        {
            char *sp2 = srch;
            ms.a = carve<float4>(sp2, M);
            ms.b = carve<float2>(sp2, M);
        }
        RS_LAUNCH(ctx, "rf_bvh_leaves", k_bvh_leaves, T, TQ, 0, L, nd, (const int64_t *)bo, boxes, ms,
                  (const float4 *)wpos, (const float4 *)wvel);
        RS_LAUNCH(ctx, "rf_bvh_build", k_bvh_build, K, 256, 0, L, nd, (const int64_t *)bo, boxes);
        // ---- random member subsets of the nodes above sub_n (Sec. 3.2) ----
        int2 *sub_q = nullptr;
        int *sub_len = ctr + 13;
        int64_t QN = 0, qcap = 0;
        if (sub_n > 0) {
            qcap = std::min<int64_t>(LM, K * sub_n);
            RS_WS(ctx, int2, sq, WS_RF_SUBQ, qcap + 1);
            sub_q = sq;
            RS_CUDA(ctx, cudaMemsetAsync(sub_len, 0, sizeof(int), ctx->stream));
            RS_LAUNCH(ctx, "rf_sub_init", k_sub_init, ceil_div(K, 128), 128, 0, L, nd, (int)sub_n);
            for (int stage = 0; stage < 2; stage++) {
                for (int pass = 0; pass < 3; pass++) {
                    RS_LAUNCH(ctx, "rf_sub_hist", k_sub_hist, T, TQ, 0, L, nd, (const int *)widx,
                              (unsigned long long)sub_seed, (int)sub_n, stage, pass);
                    RS_LAUNCH(ctx, "rf_lvl_pick", k_lvl_pick, K, 32, 0, L, pass);
                }
                RS_LAUNCH(ctx, "rf_sub_stage", k_sub_stage, ceil_div(K, 128), 128, 0, L, stage);
            }
            RS_LAUNCH(ctx, "rf_sub_mark", k_sub_mark, T, TQ, 0, L, nd, (const int *)widx,
                      (unsigned long long)sub_seed, (int)sub_n, dnn, sub_q, sub_len, (int)qcap, ctx->d_status);
            RS_LAUNCH(ctx, "rf_sub_check", k_sub_check, ceil_div(K, 128), 128, 0, L, nd, (int)sub_n, ctx->d_status);
            RS_TRY(rs_read_i64(ctx, sub_len, 1, &QN, "rs_refine6d"));
            QN = std::min<int64_t>(QN & 0xffffffffll, qcap);
        }
        // ---- linking length: sampled bracket, bounded nearest neighbours, exact select ----
        RS_WS(ctx, int64_t, ch, WS_RF_MISC4, 2 * (K + 1) + 8);
        int64_t *nsm = ch, *stot = ch + (K + 1);
        RS_LAUNCH(ctx, "rf_smp_prep", k_smp_prep, ceil_div(K, 256), 256, 0, (const int *)cur, (int)K, nd, nsm,
                  (int)sub_n, (int)ctx->tune.bracket_min);
        RS_CUDA(ctx, cudaMemsetAsync(nsm + K, 0, sizeof(int64_t), ctx->stream));
        RS_TRY(rs_scan_i64(ctx, nsm, K + 1, stot));
        int64_t SS;
        RS_TRY(rs_read_i64(ctx, stot, 1, &SS, "rs_refine6d"));
        RS_WS(ctx, float, sdnn, WS_RF_SDNN, SS + 32);
        RS_WS(ctx, float, R2, WS_RF_R2, 2 * K + 8);
        float *STOP = R2 + K;
        if (SS > 0) {
            dim3 grid((unsigned)ceil_div(SMP_MAX, W_WARPS), (unsigned)K);
            int pr = rs_prof_begin(ctx, "rf_smp_nn");
            k_bvh_nn_sample<<<grid, W_WARPS * 32, 0, ctx->stream>>>(L, nd, (const int64_t *)bo, boxes, ms,
                                                                    (const int64_t *)nsm, sdnn, ctx->d_status);
            ctx->launches++;
            rs_prof_end(ctx, pr);
            RS_CUDA(ctx, cudaGetLastError());
        }
        RS_LAUNCH(ctx, "rf_smp_thresh", k_smp_thresh, K, 256, 0, L, nd, (const int64_t *)nsm, (const float *)sdnn, f,
                  R2, STOP);
        int *fallback = ctr + 7;
        RS_CUDA(ctx, cudaMemsetAsync(ctr + 7, 0, sizeof(int), ctx->stream));
        // every member's nearest-neighbour distance, searched from the radius
        RS_WS(ctx, int64_t, fw, WS_RF_MISC5, 2 * (K + 1) + 8);
        int64_t *nw = fw, *wtot = fw + (K + 1);
        RS_LAUNCH(ctx, "rf_full_prep", k_full_prep, ceil_div(K, 256), 256, 0, (const int *)cur, (int)K, nd, nw,
                  (int)sub_n);
        RS_CUDA(ctx, cudaMemsetAsync(nw + K, 0, sizeof(int64_t), ctx->stream));
        RS_TRY(rs_scan_i64(ctx, nw, K + 1, wtot));
        int64_t W;
        RS_TRY(rs_read_i64(ctx, wtot, 1, &W, "rs_refine6d"));
        RS_WS(ctx, int, jf, WS_RF_JOBS2, 3 * W + 8);
        WarpJobs JF;
        JF.rank = jf;
        JF.q0 = jf + W;
        JF.out = jf + 2 * W;
        JF.count = W;
        RS_LAUNCH(ctx, "rf_full_jobs", k_full_jobs, K, 128, 0, (const int *)cur, (int)K, nd, (const int64_t *)nw, jf,
                  jf + W, jf + 2 * W);
        RS_TRY(launch_nn(ctx, "rf_lvl_nn", W, L, JF, nd, bo, boxes, ms, R2, STOP, 0, dnn));
        if (QN > 0)
            RS_LAUNCH(ctx, "rf_sub_nn", k_bvh_nn_list, ceil_div(QN, W_WARPS), W_WARPS * 32, 0, L, nd,
                      (const int64_t *)bo, boxes, ms, (const int2 *)sub_q, (const int *)sub_len, (int)qcap, dnn,
                      ctx->d_status);
        RS_LAUNCH(ctx, "rf_lvl_initk", k_lvl_initk, ceil_div(K, 128), 128, 0, L, nd, f, (int)sub_n);
        for (int pass = 0; pass < 3; pass++) {
            RS_LAUNCH(ctx, "rf_lvl_hist", k_lvl_hist, T, TQ, 0, L, nd, (const float *)dnn, pass);
            RS_LAUNCH(ctx, "rf_lvl_pick", k_lvl_pick, K, 32, 0, L, pass);
        }
        RS_LAUNCH(ctx, "rf_bracket_check", k_bracket_check, ceil_div(K, 128), 128, 0, L, R2,
                  (const float *)STOP, fallback, rs_fault("bracket") ? 1 : 0);
        int64_t fo;
        RS_TRY(rs_read_i64(ctx, ctr + 6, 1, &fo, "rs_refine6d"));
        if ((fo >> 32) != 0) {
            // the bracket did not hold for some node: unbounded search of
            // those nodes (the others keep their values and selection)
            RS_TRY(launch_nn(ctx, "rf_lvl_nn_full", W, L, JF, nd, bo, boxes, ms, R2, nullptr, 1, dnn));
            RS_LAUNCH(ctx, "rf_lvl_initk", k_lvl_initk, ceil_div(K, 128), 128, 0, L, nd, f, (int)sub_n);
            for (int pass = 0; pass < 3; pass++) {
                RS_LAUNCH(ctx, "rf_lvl_hist", k_lvl_hist, T, TQ, 0, L, nd, (const float *)dnn, pass);
                RS_LAUNCH(ctx, "rf_lvl_pick", k_lvl_pick, K, 32, 0, L, pass);
            }
            n_fallback_levels++;
        }
        RS_LAUNCH(ctx, "rf_lvl_band", k_lvl_band, T, TQ, 0, L, nd, (const float *)dnn);
        int64_t NB;
        RS_TRY(rs_read_i64(ctx, ctr + 4, 1, &NB, "rs_refine6d"));
        const int nbv = (int)(NB & 0xffffffffll);
        RS_LAUNCH(ctx, "rf_lvl_band_exact", k_lvl_band_exact, ceil_div(nbv, W_WARPS), W_WARPS * 32, 0, L, nd,
                  (const int64_t *)bo, boxes, ms, (const float *)dnn, ctx->d_status);
        RS_LAUNCH(ctx, "rf_lvl_l2", k_lvl_l2, K, 128, 0, L, nd, f, (int)sub_n, ctx->d_status);
        RS_LAUNCH(ctx, "rf_lvl_iota", k_lvl_iota, T, TQ, 0, L, nd, uf, csize, cmin);
        RS_LAUNCH(ctx, "rf_bvh_linkbox", k_bvh_linkbox, K, 256, 0, L, nd, (const int64_t *)bo, boxes,
                  (const float4 *)wpos, (const float4 *)wvel, (const float *)dnn, uf, ctx->d_status);
        {
            // one warp per leaf job, LK_WARPS to a block; compiled for 8 x
            // rs_tuning::link_blocks_per_sm resident warps per SM
            const int64_t njobs = T * (TQ / 32), lg = ceil_div(njobs, LK_WARPS);
            switch (ctx->tune.link_blocks_per_sm) {
            case 4:
                RS_LAUNCH(ctx, "rf_lvl_link", k_bvh_link<4>, lg, LK_WARPS * 32, 0, L, nd, (const int64_t *)bo, boxes,
                          ms, (const float *)dnn, uf, ctx->d_status);
                break;
            case 6:
                RS_LAUNCH(ctx, "rf_lvl_link", k_bvh_link<6>, lg, LK_WARPS * 32, 0, L, nd, (const int64_t *)bo, boxes,
                          ms, (const float *)dnn, uf, ctx->d_status);
                break;
            default:
                RS_LAUNCH(ctx, "rf_lvl_link", k_bvh_link<5>, lg, LK_WARPS * 32, 0, L, nd, (const int64_t *)bo, boxes,
                          ms, (const float *)dnn, uf, ctx->d_status);
            }
        }
        RS_LAUNCH(ctx, "rf_lvl_comp", k_lvl_comp, T, TQ, 0, L, nd, (const int *)widx, uf, csize, cmin,
                  ctx->d_status);
        // reorder: children first, by smallest particle index, then the rest
        RS_LAUNCH(ctx, "rf_lvl_keys", k_lvl_keys, T, TQ, 0, L, nd, uf, (const int *)csize, (const int *)cmin,
                  (unsigned long long *)k0, v0, (int)min_n, ctx->d_status);
        bool alt = false;
        RS_TRY(rs_radix_sort_u64(ctx, k0, k1, v0, v1, LM, 32 + rbits, &alt, "sort_child"));
        const unsigned long long *sk = (const unsigned long long *)(alt ? k1 : k0);
        const unsigned *sv = alt ? v1 : v0;
        unsigned *dest = (unsigned *)(alt ? v0 : v1);
        RS_LAUNCH(ctx, "rf_lvl_children", k_lvl_children, ceil_div(LM, 256), 256, 0, L, nd, LM, sk, sv, uf,
                  (const int *)csize, nxt, nxt_len, small_q, ctr + 2, ctx->d_status);
        RS_LAUNCH(ctx, "rf_lvl_scatter", k_lvl_scatter, ceil_div(LM, 256), 256, 0, L, nd, LM, sk, sv,
                  (const float4 *)wpos, (const float4 *)wvel, (const int *)widx, wpos2, wvel2, widx2, dest, 32);
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
    // three size classes, each forwarding its smaller subtrees to the next
    {
        auto kbig = k_small_subtree<SMALL_N, SMALL_THREADS, 2>;
        auto kmid = k_small_subtree<MID_N, MID_THREADS, 8>;
        const size_t sbig = sizeof(SmallShared<SMALL_N, SMALL_THREADS>);
        const size_t smid = sizeof(SmallShared<MID_N, MID_THREADS>);
        RS_CUDA(ctx, cudaFuncSetAttribute(kbig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sbig));
        RS_CUDA(ctx, cudaFuncSetAttribute(kmid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smid));
        const rs_tuning &tu = ctx->tune;
        RS_LAUNCH(ctx, "rf_small_subtree", kbig, (int64_t)ctx->num_sms * tu.small_ctas_per_sm, SMALL_THREADS, sbig,
                  (const int *)small_q, (const int *)(ctr + 2), ctr + 3, wpos, wvel, widx,
                  std::min(tu.mid_max, MID_N), mid_q, ctr + 11, nd, box, f, (int)min_n, ctx->d_status);
        RS_LAUNCH(ctx, "rf_mid_subtree", kmid, (int64_t)ctx->num_sms * tu.mid_ctas_per_sm, MID_THREADS, smid,
                  (const int *)mid_q, (const int *)(ctr + 11), ctr + 12, wpos, wvel, widx,
                  std::min(tu.tiny_max, TINY_N), tiny_q, ctr + 8, nd, box, f, (int)min_n, ctx->d_status);
    }
    RS_LAUNCH(ctx, "rf_tiny_subtree", k_tiny_subtree, (int64_t)ctx->num_sms * ctx->tune.tiny_ctas_per_sm,
              TINY_WARPS * 32, 0,
              (const int *)tiny_q, (const int *)(ctr + 8), ctr + 9, (const float4 *)wpos, (const float4 *)wvel, widx,
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
    t->sum_big_level_members = sum_level;
    t->n_fallback_levels = n_fallback_levels;
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

extern "C" rs_status rs_refine6d_sampled(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n,
                                         double box, const int32_t *perm, const int64_t *group_offsets,
                                         int64_t n_groups, double f, int32_t min_n, int64_t subset_n,
                                         uint64_t subset_seed, rs_tree **out)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    if (!out) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_refine6d: out is NULL");
    *out = nullptr;
    if (n < 0 || n_groups < 0 || (stride != 3 && stride != 4) || !(box > 0) || !(f > 0 && f < 1) || min_n < 2 ||
        !group_offsets || (n > 0 && (!pos || !vel)) || (n_groups > 0 && !perm))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_refine6d: bad argument");
    if (subset_n != 0 && (subset_n < SMALL_N || subset_n >= ((int64_t)1 << 31)))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_refine6d: subset size must be 0 or in [1024, 2^31)");
    if (n >= ((int64_t)1 << 31)) return rs_fail(ctx, RS_ERR_TOO_LARGE, "rs_refine6d: n >= 2^31");
    if ((double)(float)box != box) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_refine6d: box must be a float32 value");
    RsRange range("rs_refine6d");
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
        rs_status s = refine_impl(ctx, pos, vel, stride, n, box, perm, group_offsets, n_groups, f, min_n, subset_n,
                                  subset_seed, cap, &t);
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

extern "C" rs_status rs_refine6d(rs_ctx *ctx, const float *pos, const float *vel, int32_t stride, int64_t n,
                                 double box, const int32_t *perm, const int64_t *group_offsets, int64_t n_groups,
                                 double f, int32_t min_n, rs_tree **out)
{
    return rs_refine6d_sampled(ctx, pos, vel, stride, n, box, perm, group_offsets, n_groups, f, min_n, 0, 0, out);
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

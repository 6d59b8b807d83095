// rs_halo.cu -- halo centres, the host/subhalo relation (Sec. 3.4, 3.5.1)
// and single-pass unbinding (Sec. 3.4, App. B), after the assignment.
//
// Centres.  A node "belongs" to a halo when every seed under it does; the
// halo's centre is the mean position and velocity of its node with the
// smallest Poisson error sigma_x / sqrt(n) (ties: smaller smallest member,
// then smaller level).  Seeds carry their halo; the property is pushed up
// the tree one level at a time with atomic compare-and-swap.
//
// Hosts.  Each halo's centre is measured with the metric of Eq. 3 against
// the halos of its 3D group with more assigned particles; the nearest is its
// host (ties to the smaller id).  Halos are sorted by group so that each
// scans only its own group.
//
// Unbinding.  A halo's set is its own particles and those of every halo
// below it in the host relation.  Sets are gathered as (set, particle) keys
// and radix-sorted, so each set is a contiguous run.  The bulk velocity is a
// float64 block reduction.  The potential per unit mass is either a direct
// sum over the set (one CTA per 256 targets, sources staged through shared
// memory, float32 pair terms added per 256-source chunk, chunk sums in
// float64), or, for sets above UB_DIRECT_MAX members when theta > 0, a tree
// walk (App. B): each set is put in Morton order of its unwrapped positions,
// cut into 32-member leaves under a 32-ary box hierarchy whose boxes keep
// their mass centre x0, sigma^2 = mean |x - x0|^2 and r_max; a box stands for
// its particles (monopole) beyond d(theta) = r_max/2 + sqrt((r_max/2)^2 +
// sigma^2/theta) from x0, which bounds the relative error of each accepted
// term, hence of the sum, by theta (Salmon & Warren 1994).  One warp walks
// the tree for the 32 targets of a leaf, accepting a box only when the whole
// leaf lies beyond d(theta).  Periodic differences take the far-side
// coordinate minus the box first (exact for x >= box/2).
#include <algorithm>
#include <cmath>

#include "rs_refine.cuh"

namespace {

constexpr int HP_THREADS = 256;
constexpr int UB_TILE = 256;          // targets per CTA and sources per shared-memory chunk
constexpr int UB_DIRECT_MAX = 4096;   // sets up to this size are summed directly
constexpr int UT_LEAF = 32;           // members per leaf, children per box
constexpr int UT_WARPS = 8;           // warps per CTA in the tree walk
constexpr int UT_STACK = 256;         // boxes on a warp's stack
constexpr int UT_MAX_LEVELS = 8;      // 32^8 > 2^31 members

__global__ void k_hp_init(NodeArrays nd, int nn, const int *leaf_halo, int *pure)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    pure[i] = nd.nchild[i] == 0 ? leaf_halo[i] : -2;
}

// nodes of one level hand their halo (or -1, several) to their parent
__global__ void k_hp_up(NodeArrays nd, int nn, int level, int *pure)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn || nd.level[i] != level) return;
    const int p = nd.parent[i];
    if (p < 0) return;
    const int v = pure[i];
    const int old = atomicCAS(&pure[p], -2, v);
    if (old != -2 && old != v) atomicExch(&pure[p], -1);
}

// squared Poisson error of a node, float64 (sigma_x >= 0, so its bits order as the value)
__device__ __forceinline__ unsigned long long poisson_bits(const NodeArrays &nd, int i)
{
    const double e = __ddiv_rn(__dmul_rn(nd.sigx[i], nd.sigx[i]), (double)nd.count[i]);
    return (unsigned long long)__double_as_longlong(e);
}

__global__ void k_hp_best(NodeArrays nd, int nn, const int *pure, int pass, unsigned long long *ebest,
                          unsigned long long *tbest, int *centre_node, double *xc, double *vc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const int h = pure[i];
    if (h < 0) return;
    const unsigned long long e = poisson_bits(nd, i);
    if (pass == 0) {
        atomicMin(&ebest[h], e);
        return;
    }
    if (e != ebest[h]) return;
    const unsigned long long key = ((unsigned long long)(unsigned)nd.minidx[i] << 32) | (unsigned)nd.level[i];
    if (pass == 1) {
        atomicMin(&tbest[h], key);
        return;
    }
    if (key != tbest[h]) return;
    centre_node[h] = i;
    for (int d = 0; d < 3; d++) {
        xc[3 * h + d] = nd.xbar[3 * i + d];
        vc[3 * h + d] = nd.vbar[3 * i + d];
    }
}

__global__ void k_hp_fill_u64(unsigned long long *p, int64_t n, unsigned long long v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_hp_keys(int H, const int *id, const int *root, unsigned *kid, unsigned *vid, unsigned *kroot,
                          unsigned *vroot)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    kid[r] = (unsigned)id[r];
    vid[r] = (unsigned)r;
    kroot[r] = (unsigned)root[r];
    vroot[r] = (unsigned)r;
}

__device__ __forceinline__ int lower_bound_u(const unsigned *a, int n, unsigned x)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// rank of a halo id (ids sorted with their ranks), -1 if absent
__device__ __forceinline__ int rank_of(const unsigned *sid, const unsigned *srank, int H, int id)
{
    const int k = lower_bound_u(sid, H, (unsigned)id);
    return (k < H && sid[k] == (unsigned)id) ? (int)srank[k] : -1;
}

__global__ void k_hp_count(int64_t n, const int32_t *halo_id, const unsigned *sid, const unsigned *srank, int H,
                           unsigned long long *n_assigned, rs_dev_status *st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || halo_id[i] < 0) return;
    const int r = rank_of(sid, srank, H, halo_id[i]);
    if (r < 0) {
        dev_fail(st, DEV_BADARG, 70, i);
        return;
    }
    atomicAdd(&n_assigned[r], 1ull);
}

__device__ __forceinline__ double ratio2_h(double num, double den)
{
    if (den > 0) return __ddiv_rn(num, den);
    return num > 0 ? INFINITY : 0.0;
}

__device__ __forceinline__ double min_image_h(double d, double box)
{
    if (d > 0.5 * box) d = f64_sub(d, box);
    else if (d < -0.5 * box) d = f64_add(d, box);
    return d;
}

// host of every halo: the Eq. 3 nearest larger halo of its group
__global__ void k_hp_host(int H, rs_halos hs, const double *xc, const double *vc,
                          const unsigned long long *n_assigned, const unsigned *groot, const unsigned *grank,
                          double box, int *host)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= H) return;
    const unsigned g = (unsigned)hs.root[s];
    const int a = lower_bound_u(groot, H, g);
    double best = INFINITY;
    int bid = -1;
    for (int k = a; k < H && groot[k] == g; k++) {
        const int h = (int)grank[k];
        if (n_assigned[h] <= n_assigned[s]) continue;
        double dx2 = 0, dv2 = 0;
        for (int d = 0; d < 3; d++) {
            const double dx = min_image_h(f64_sub(xc[3 * h + d], xc[3 * s + d]), box);
            const double dv = f64_sub(vc[3 * h + d], vc[3 * s + d]);
            dx2 = f64_add(dx2, f64_mul(dx, dx));
            dv2 = f64_add(dv2, f64_mul(dv, dv));
        }
        const double d2 = f64_add(ratio2_h(dx2, hs.rdyn2[h]), ratio2_h(dv2, f64_mul(hs.sigv[h], hs.sigv[h])));
        if (d2 < best || (d2 == best && bid >= 0 && hs.id[h] < bid)) {
            best = d2;
            bid = hs.id[h];
        }
    }
    host[s] = bid;
}

// ---- unbinding ----
// host ranks of the halos (-1: none)
__global__ void k_ub_up(int H, const int32_t *host, const unsigned *sid, const unsigned *srank, int *up,
                        rs_dev_status *st)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    int u = -1;
    if (host[r] >= 0) {
        u = rank_of(sid, srank, H, host[r]);
        if (u < 0 || u == r) {
            dev_fail(st, DEV_BADARG, 71, r);
            u = -1;
        }
    }
    up[r] = u;
}

// number of sets each particle joins (its halo and every halo up the chain);
// a chain longer than H is a cycle
__global__ void k_ub_count(int64_t n, const int32_t *halo_id, const unsigned *sid, const unsigned *srank, int H,
                           const int *up, unsigned long long *total, rs_dev_status *st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (i < n && halo_id[i] >= 0) {
        int r = rank_of(sid, srank, H, halo_id[i]);
        if (r < 0) dev_fail(st, DEV_BADARG, 72, i);
        for (int guard = 0; r >= 0; r = up[r], guard++) {
            if (guard > H) {
                dev_fail(st, DEV_BADARG, 73, i);
                break;
            }
            c++;
        }
    }
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(total, c);
}

// (set rank, particle) keys, written through a global cursor
__global__ void k_ub_keys(int64_t n, const int32_t *halo_id, const unsigned *sid, const unsigned *srank, int H,
                          const int *up, unsigned long long *cursor, int64_t cap, uint64_t *keys, uint32_t *vals,
                          rs_dev_status *st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || halo_id[i] < 0) return;
    int r = rank_of(sid, srank, H, halo_id[i]);
    for (int guard = 0; r >= 0 && guard <= H; r = up[r], guard++) {
        const unsigned long long k = atomicAdd(cursor, 1ull);
        if ((int64_t)k >= cap) {
            dev_fail(st, DEV_OVERFLOW, 74, i);
            return;
        }
        keys[k] = ((uint64_t)(unsigned)r << 32) | (uint64_t)i;
        vals[k] = (uint32_t)i;
    }
}

// set boundaries from the sorted keys: off[r] = first position of set r
__global__ void k_ub_bounds(int64_t total, const uint64_t *keys, int64_t *off, int H)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    const int r = (int)(keys[k] >> 32);
    const int rp = k == 0 ? -1 : (int)(keys[k - 1] >> 32);
    for (int q = rp + 1; q <= r; q++) off[q] = k;
    if (k == total - 1)
        for (int q = r + 1; q <= H; q++) off[q] = total;
}

// bulk velocity of every set: one block per set, float64 reduction in a fixed order
__global__ void __launch_bounds__(HP_THREADS) k_ub_bulk(int H, const int64_t *off, const uint32_t *mem,
                                                        const float *vel, int stride, double *vbulk)
{
    __shared__ double red[3][HP_THREADS];
    for (int r = blockIdx.x; r < H; r += gridDim.x) {
        const int64_t a = off[r], b = off[r + 1];
        double s[3] = {0, 0, 0};
        for (int64_t k = a + threadIdx.x; k < b; k += HP_THREADS) {
            const float *v = vel + (int64_t)stride * mem[k];
            for (int d = 0; d < 3; d++) s[d] += (double)v[d];
        }
        for (int d = 0; d < 3; d++) red[d][threadIdx.x] = s[d];
        __syncthreads();
        for (int w = HP_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w)
                for (int d = 0; d < 3; d++) red[d][threadIdx.x] += red[d][threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0)
            for (int d = 0; d < 3; d++) vbulk[3 * r + d] = b > a ? red[d][0] / (double)(b - a) : 0.0;
        __syncthreads();
    }
}

__device__ __forceinline__ bool ub_tree_set(int64_t n, int tree_on) { return tree_on && n > UB_DIRECT_MAX; }

// direct-sum tiles of every set summed directly
__global__ void k_ub_tiles(int H, const int64_t *off, int tree_on, int64_t *tiles)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const int64_t n = off[r + 1] - off[r];
    tiles[r] = ub_tree_set(n, tree_on) ? 0 : (n + UB_TILE - 1) / UB_TILE;
}

__global__ void k_ub_npart(int H, const int64_t *off, int64_t *n_part)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    n_part[r] = off[r + 1] - off[r];
}

__global__ void k_ub_tilemap(int H, const int64_t *toff, int *trank, int *tq0)
{
    const int r = blockIdx.x;
    if (r >= H) return;
    for (int64_t t = toff[r] + threadIdx.x; t < toff[r + 1]; t += blockDim.x) {
        trank[t] = r;
        tq0[t] = (int)((t - toff[r]) * UB_TILE);
    }
}

// b - a for one axis with the periodic image nearest a (x - box is exact
// for x >= box/2, so only the final subtraction rounds)
__device__ __forceinline__ float pdiff(float a, float b, float box)
{
    const float d = b - a;
    if (d > 0.5f * box) return (b - box) - a;
    if (d < -0.5f * box) return b - (a - box);
    return d;
}

// the bound test of particle i in set r, given its potential per unit mass
__device__ __forceinline__ void ub_finish(uint32_t i, int r, double phi, const float *vel, int stride,
                                          const double *vbulk, const int32_t *halo_id, const int *hid,
                                          unsigned long long *n_bound, int8_t *bound_own, double *phi_own)
{
    const float *vi = vel + (int64_t)stride * i;
    double ke = 0;
    for (int d = 0; d < 3; d++) {
        const double dv = (double)vi[d] - vbulk[3 * r + d];
        ke += dv * dv;
    }
    const bool bound = 0.5 * ke + phi < 0.0;
    if (bound) atomicAdd(&n_bound[r], 1ull);
    if (halo_id[i] == hid[r]) {
        bound_own[i] = bound ? 1 : 0;
        if (phi_own) phi_own[i] = phi;
    }
}

// potential and bound flag of every member of a set tile
__global__ void __launch_bounds__(UB_TILE) k_ub_phi(const int *trank, const int *tq0, const int64_t *off,
                                                    const uint32_t *mem, const float *pos, const float *vel,
                                                    int stride, float boxf, double gm, float eps2f,
                                                    const double *vbulk, const int32_t *halo_id, const int *hid,
                                                    unsigned long long *n_bound, int8_t *bound_own,
                                                    double *phi_own)
{
    __shared__ float4 src[UB_TILE];
    const int r = trank[blockIdx.x];
    const int64_t a = off[r], n = off[r + 1] - a;
    const int q = tq0[blockIdx.x] + threadIdx.x;
    const bool mine = q < n;
    const uint32_t i = mine ? mem[a + q] : 0u;
    const float *pi = pos + (int64_t)stride * i;
    const float px = pi[0], py = pi[1], pz = pi[2];
    double phi = 0.0;
    for (int64_t c0 = 0; c0 < n; c0 += UB_TILE) {
        const int64_t cj = c0 + threadIdx.x;
        if (cj < n) {
            const uint32_t j = mem[a + cj];
            const float *pj = pos + (int64_t)stride * j;
            src[threadIdx.x] = make_float4(pj[0], pj[1], pj[2], __int_as_float((int)j));
        }
        __syncthreads();
        const int m = (int)(n - c0 < UB_TILE ? n - c0 : UB_TILE);
        float part = 0.f;
        if (mine)
            for (int k = 0; k < m; k++) {
                const float4 s = src[k];
                if ((uint32_t)__float_as_int(s.w) == i) continue;
                const float dx = pdiff(px, s.x, boxf), dy = pdiff(py, s.y, boxf), dz = pdiff(pz, s.z, boxf);
                const float r2 = dx * dx + dy * dy + dz * dz + eps2f;
                if (r2 > 0.f) part -= rsqrtf(r2);
            }
        phi += (double)part;
        __syncthreads();
    }
    if (!mine) return;
    ub_finish(i, r, phi * gm, vel, stride, vbulk, halo_id, hid, n_bound, bound_own, phi_own);
}

// ---- tree walk for large sets ----
// Boxes of one set: level 0 holds the leaves (32 consecutive members in
// Morton order), level h the boxes over 32 consecutive boxes of level h-1,
// up to one root; levels are stored one after another from level 0.
struct UTView {
    int H;                   // levels
    int cnt[UT_MAX_LEVELS];  // boxes per level
    int off[UT_MAX_LEVELS];  // first box of each level
};

__device__ __forceinline__ void ut_view(UTView &V, int64_t n)
{
    int c = (int)((n + UT_LEAF - 1) / UT_LEAF), o = 0, h = 0;
    for (;;) {
        V.cnt[h] = c;
        V.off[h] = o;
        o += c;
        h++;
        if (c == 1 || h == UT_MAX_LEVELS) break;
        c = (c + UT_LEAF - 1) / UT_LEAF;
    }
    V.H = h;
}

__device__ __forceinline__ int64_t ut_boxes(int64_t n)
{
    int64_t c = (n + UT_LEAF - 1) / UT_LEAF, t = 0;
    for (;;) {
        t += c;
        if (c == 1) break;
        c = (c + UT_LEAF - 1) / UT_LEAF;
    }
    return t;
}

// a box: mass centre and count (c), sigma^2, r_max and the opening distance (s)
struct UBoxes {
    float4 *c;
    float4 *s;
};

__global__ void k_ub_ref(int H, const int64_t *off, const uint32_t *mem, const float *pos, int stride, float4 *ref)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H || off[r + 1] == off[r]) return;
    const float *p = pos + (int64_t)stride * mem[off[r]];
    ref[r] = make_float4(p[0], p[1], p[2], 0.f);
}

// positions relative to the set's first member, nearest periodic image
__global__ void k_ub_upos(int64_t total, const uint64_t *keys, const uint32_t *mem, const float *pos, int stride,
                          const float4 *ref, float boxf, float4 *upos)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    const int r = (int)(keys[k] >> 32);
    const uint32_t i = mem[k];
    const float *p = pos + (int64_t)stride * i;
    const float4 a = ref[r];
    upos[k] = make_float4(pdiff(a.x, p[0], boxf), pdiff(a.y, p[1], boxf), pdiff(a.z, p[2], boxf),
                          __int_as_float((int)i));
}

// bounding cube of every tree set: lower corner and 1024 / side
__global__ void __launch_bounds__(HP_THREADS) k_ub_bbox(int H, const int64_t *off, int tree_on, const float4 *upos,
                                                        float4 *cube)
{
    __shared__ float lo[3][HP_THREADS], hi[3][HP_THREADS];
    for (int r = blockIdx.x; r < H; r += gridDim.x) {
        const int64_t a = off[r], b = off[r + 1];
        if (!ub_tree_set(b - a, tree_on)) continue;  // uniform over the block
        float l[3] = {INFINITY, INFINITY, INFINITY}, u[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t k = a + threadIdx.x; k < b; k += HP_THREADS) {
            const float4 p = upos[k];
            l[0] = fminf(l[0], p.x);
            l[1] = fminf(l[1], p.y);
            l[2] = fminf(l[2], p.z);
            u[0] = fmaxf(u[0], p.x);
            u[1] = fmaxf(u[1], p.y);
            u[2] = fmaxf(u[2], p.z);
        }
        for (int d = 0; d < 3; d++) {
            lo[d][threadIdx.x] = l[d];
            hi[d][threadIdx.x] = u[d];
        }
        __syncthreads();
        for (int w = HP_THREADS / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w)
                for (int d = 0; d < 3; d++) {
                    lo[d][threadIdx.x] = fminf(lo[d][threadIdx.x], lo[d][threadIdx.x + w]);
                    hi[d][threadIdx.x] = fmaxf(hi[d][threadIdx.x], hi[d][threadIdx.x + w]);
                }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const float side = fmaxf(fmaxf(hi[0][0] - lo[0][0], hi[1][0] - lo[1][0]), hi[2][0] - lo[2][0]);
            cube[r] = make_float4(lo[0][0], lo[1][0], lo[2][0], side > 0.f ? 1024.f / side : 0.f);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v)
{
    v &= 1023u;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t cell10(float x, float lo, float scale)
{
    const float q = (x - lo) * scale;
    return q <= 0.f ? 0u : (q >= 1023.f ? 1023u : (uint32_t)q);
}

// (set, Morton code) keys of every entry; sets summed directly keep code 0
__global__ void k_ub_morton(int64_t total, const uint64_t *keys, const int64_t *off, int tree_on, const float4 *upos,
                            const float4 *cube, uint64_t *mkeys, uint32_t *mvals)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    const int r = (int)(keys[k] >> 32);
    uint32_t code = 0;
    if (ub_tree_set(off[r + 1] - off[r], tree_on)) {
        const float4 c = cube[r], p = upos[k];
        code = (spread10(cell10(p.z, c.z, c.w)) << 2) | (spread10(cell10(p.y, c.y, c.w)) << 1) |
               spread10(cell10(p.x, c.x, c.w));
    }
    mkeys[k] = ((uint64_t)(uint32_t)r << 30) | code;
    mvals[k] = (uint32_t)k;
}

__global__ void k_ub_gather(int64_t total, const uint32_t *perm, const float4 *upos, const uint32_t *mem,
                            float4 *tpos, uint32_t *tmem)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    const uint32_t s = perm[k];
    tpos[k] = upos[s];
    tmem[k] = mem[s];
}

// boxes and leaves of every set (zero for sets summed directly)
__global__ void k_ub_boxcount(int H, const int64_t *off, int tree_on, int64_t *nbox, int64_t *nleaf)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const int64_t n = off[r + 1] - off[r];
    const bool t = ub_tree_set(n, tree_on);
    nbox[r] = t ? ut_boxes(n) : 0;
    nleaf[r] = t ? (n + UT_LEAF - 1) / UT_LEAF : 0;
}

__global__ void k_ub_leafjobs(int H, const int64_t *loff, int *jset, int *jleaf)
{
    const int r = blockIdx.x;
    if (r >= H) return;
    for (int64_t j = loff[r] + threadIdx.x; j < loff[r + 1]; j += blockDim.x) {
        jset[j] = r;
        jleaf[j] = (int)(j - loff[r]);
    }
}

__device__ __forceinline__ float ut_dopen(float sig2, float rmax, float theta)
{
    const float h = 0.5f * rmax;
    return h + sqrtf(h * h + sig2 / theta);
}

// leaf boxes: one warp per leaf, a member per lane
__global__ void __launch_bounds__(UT_WARPS * 32) k_ub_leafbox(int64_t njobs, const int *jset, const int *jleaf,
                                                             const int64_t *off, const int64_t *bbase,
                                                             const float4 *tpos, float theta, UBoxes B)
{
    const int64_t j = (int64_t)blockIdx.x * UT_WARPS + warp_id();
    if (j >= njobs) return;
    const int lane = lane_id();
    const int r = jset[j], leaf = jleaf[j];
    const int64_t a = off[r], n = off[r + 1] - a;
    const int64_t m = (int64_t)leaf * UT_LEAF + lane;
    const bool have = m < n;
    const float4 p = have ? tpos[a + m] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float cnt = warp_sum(have ? 1.f : 0.f);
    const float x0 = warp_sum(have ? p.x : 0.f) / cnt, y0 = warp_sum(have ? p.y : 0.f) / cnt,
                z0 = warp_sum(have ? p.z : 0.f) / cnt;
    const float dx = p.x - x0, dy = p.y - y0, dz = p.z - z0;
    const float d2 = have ? dx * dx + dy * dy + dz * dz : 0.f;
    const float sig2 = warp_sum(d2) / cnt;
    float rm = sqrtf(d2);
    for (int o = 16; o > 0; o >>= 1) rm = fmaxf(rm, __shfl_xor_sync(0xffffffffu, rm, o));
    if (lane == 0) {
        const int64_t b = bbase[r] + leaf;
        B.c[b] = make_float4(x0, y0, z0, cnt);
        B.s[b] = make_float4(sig2, rm, ut_dopen(sig2, rm, theta), 0.f);
    }
}

// upper levels of every tree set, one block per set (parallel-axis sums for
// sigma^2; r_max bounded by the children's distance plus their r_max)
__global__ void __launch_bounds__(HP_THREADS) k_ub_upper(int H, const int64_t *off, int tree_on,
                                                         const int64_t *bbase, float theta, UBoxes B)
{
    for (int r = blockIdx.x; r < H; r += gridDim.x) {
        const int64_t n = off[r + 1] - off[r];
        if (!ub_tree_set(n, tree_on)) continue;  // uniform over the block
        UTView V;
        ut_view(V, n);
        const int64_t base = bbase[r];
        for (int h = 1; h < V.H; h++) {
            for (int b = threadIdx.x; b < V.cnt[h]; b += HP_THREADS) {
                const int c0 = b * UT_LEAF, c1 = min(c0 + UT_LEAF, V.cnt[h - 1]);
                float cnt = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
                for (int c = c0; c < c1; c++) {
                    const float4 q = B.c[base + V.off[h - 1] + c];
                    cnt += q.w;
                    sx += q.w * q.x;
                    sy += q.w * q.y;
                    sz += q.w * q.z;
                }
                const float x0 = sx / cnt, y0 = sy / cnt, z0 = sz / cnt;
                float s2 = 0.f, rm = 0.f;
                for (int c = c0; c < c1; c++) {
                    const float4 q = B.c[base + V.off[h - 1] + c];
                    const float4 w = B.s[base + V.off[h - 1] + c];
                    const float dx = q.x - x0, dy = q.y - y0, dz = q.z - z0;
                    const float g2 = dx * dx + dy * dy + dz * dz;
                    s2 += q.w * (w.x + g2);
                    rm = fmaxf(rm, sqrtf(g2) + w.y);
                }
                s2 /= cnt;
                B.c[base + V.off[h] + b] = make_float4(x0, y0, z0, cnt);
                B.s[base + V.off[h] + b] = make_float4(s2, rm, ut_dopen(s2, rm, theta), 0.f);
            }
            __syncthreads();
        }
    }
}

// tree walk: one warp per leaf of targets, a target per lane
__global__ void __launch_bounds__(UT_WARPS * 32) k_ub_walk(int64_t njobs, const int *jset, const int *jleaf,
                                                          const int64_t *off, const int64_t *bbase,
                                                          const float4 *tpos, const uint32_t *tmem, UBoxes B,
                                                          double gm, float eps2f, const float *vel, int stride,
                                                          const double *vbulk, const int32_t *halo_id, const int *hid,
                                                          unsigned long long *n_bound, int8_t *bound_own,
                                                          double *phi_own, rs_dev_status *st)
{
    __shared__ int stk[UT_WARPS][UT_STACK];
    const unsigned FULL = 0xffffffffu;
    const int64_t j = (int64_t)blockIdx.x * UT_WARPS + warp_id();
    if (j >= njobs) return;
    const int w = warp_id(), lane = lane_id();
    const int r = jset[j], leaf = jleaf[j];
    const int64_t a = off[r], n = off[r + 1] - a;
    UTView V;
    ut_view(V, n);
    const int64_t base = bbase[r];
    const int64_t m = (int64_t)leaf * UT_LEAF + lane;
    const bool have = m < n;
    const float4 t = have ? tpos[a + m] : make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t ti = (uint32_t)__float_as_int(t.w);
    // the group: this leaf's centre and radius
    const float4 gc = B.c[base + leaf], gs = B.s[base + leaf];
    float acc = 0.f;    // current chunk of terms
    double phi = 0.0;   // chunks
    int terms = 0;
    int *S = stk[w];
    if (lane == 0) S[0] = ((V.H - 1) << 24) | 0;  // the root
    int sp = 1;
    __syncwarp();
    for (int it = 0; sp > 0 && it < (1 << 24); it++) {
        sp--;
        const int ent = S[sp];
        __syncwarp();
        const int h = ent >> 24, b = ent & 0xffffff;
        if (h == 0) {  // a leaf: every member directly
            const int64_t l0 = (int64_t)b * UT_LEAF;
            const int64_t mm = l0 + lane;
            const float4 q = mm < n ? tpos[a + mm] : make_float4(0.f, 0.f, 0.f, 0.f);
            const int cnt = (int)(n - l0 < UT_LEAF ? n - l0 : UT_LEAF);
            for (int k = 0; k < cnt; k++) {
                const float qx = __shfl_sync(FULL, q.x, k), qy = __shfl_sync(FULL, q.y, k),
                            qz = __shfl_sync(FULL, q.z, k);
                const uint32_t qi = (uint32_t)__shfl_sync(FULL, __float_as_int(q.w), k);
                const float dx = qx - t.x, dy = qy - t.y, dz = qz - t.z;
                const float r2 = dx * dx + dy * dy + dz * dz + eps2f;
                if (have && qi != ti && r2 > 0.f) acc -= rsqrtf(r2);
            }
            terms += cnt;
        } else {
            const int c = b * UT_LEAF + lane;
            const bool ex = c < V.cnt[h - 1];
            float4 cc = make_float4(0.f, 0.f, 0.f, 0.f), cs = cc;
            if (ex) {
                cc = B.c[base + V.off[h - 1] + c];
                cs = B.s[base + V.off[h - 1] + c];
            }
            const float gx = cc.x - gc.x, gy = cc.y - gc.y, gz = cc.z - gc.z;
            const bool acc_ok = ex && sqrtf(gx * gx + gy * gy + gz * gz) - gs.y > cs.z;
            unsigned am = __ballot_sync(FULL, acc_ok);
            while (am) {  // accepted boxes: a monopole term for every target
                const int src = __ffs(am) - 1;
                am &= am - 1;
                const float bx = __shfl_sync(FULL, cc.x, src), by = __shfl_sync(FULL, cc.y, src),
                            bz = __shfl_sync(FULL, cc.z, src), bn = __shfl_sync(FULL, cc.w, src);
                const float dx = bx - t.x, dy = by - t.y, dz = bz - t.z;
                if (have) acc -= bn * rsqrtf(dx * dx + dy * dy + dz * dz + eps2f);
                terms++;
            }
            const unsigned om = __ballot_sync(FULL, ex && !acc_ok);
            // stack entries hold a box index in 24 bits (sets below 2^29 members)
            if (sp + __popc(om) > UT_STACK || __any_sync(FULL, ex && !acc_ok && c >= (1 << 24))) {
                if (lane == 0) dev_fail(st, DEV_OVERFLOW, 75, r);
                break;
            }
            if (ex && !acc_ok) S[sp + __popc(om & ((1u << lane) - 1u))] = ((h - 1) << 24) | c;
            sp += __popc(om);
            __syncwarp();
        }
        if (terms >= 256) {
            phi += (double)acc;
            acc = 0.f;
            terms = 0;
        }
    }
    phi += (double)acc;
    // a walk that ran out of iterations with boxes still pending has a
    // partial potential: record it like every other bounded loop
    if (sp > 0 && lane == 0) dev_fail(st, DEV_TIMEOUT, 76, r);
    if (!have) return;
    ub_finish(tmem[a + m], r, phi * gm, vel, stride, vbulk, halo_id, hid, n_bound, bound_own, phi_own);
}

__global__ void k_ub_fill_i8(int8_t *p, int64_t n, int8_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ids sorted with their ranks, in the workspace
rs_status sorted_ids(rs_ctx *ctx, const rs_halos *hs, unsigned **sid, unsigned **srank, unsigned **groot,
                     unsigned **grank)
{
    const int64_t H = hs->n_halos;
    RS_WS(ctx, unsigned, kb, WS_HL_IDS, 8 * H + 16);
    unsigned *k0 = kb, *v0 = kb + H, *k1 = kb + 2 * H, *v1 = kb + 3 * H;
    unsigned *g0 = kb + 4 * H, *w0 = kb + 5 * H, *g1 = kb + 6 * H, *w1 = kb + 7 * H;
    RS_LAUNCH(ctx, "hp_keys", k_hp_keys, ceil_div(H, 256), 256, 0, (int)H, (const int *)hs->id,
              (const int *)hs->root, k0, v0, g0, w0);
    bool alt = false;
    RS_TRY(rs_radix_sort_u32(ctx, k0, k1, v0, v1, H, 31, &alt));
    *sid = alt ? k1 : k0;
    *srank = alt ? v1 : v0;
    bool galt = false;
    RS_TRY(rs_radix_sort_u32(ctx, g0, g1, w0, w1, H, 31, &galt));
    *groot = galt ? g1 : g0;
    *grank = galt ? w1 : w0;
    return RS_OK;
}

}  // namespace

extern "C" rs_status rs_halo_props(rs_ctx *ctx, const rs_tree *t, const rs_halos *hs, const int32_t *halo_id,
                                   int64_t n, int32_t *centre_node, double *xc, double *vc, int64_t *n_assigned,
                                   int32_t *host)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    RsRange range("rs_halo_props");
    if (!t || !hs || n != t->n_total || hs->n_nodes != t->n_nodes || (n > 0 && !halo_id))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_halo_props: bad argument");
    const int64_t H = hs->n_halos;
    if (H == 0) return RS_OK;
    if (!centre_node || !xc || !vc || !n_assigned || !host)
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_halo_props: an output is NULL");
    const NodeArrays &nd = t->nd;
    const int nn = (int)t->n_nodes;
    RS_WS(ctx, int, pure, WS_HL_PURE, nn);
    RS_WS(ctx, unsigned long long, eb, WS_HL_BEST, 2 * H);
    RS_LAUNCH(ctx, "hp_init", k_hp_init, ceil_div(nn, 256), 256, 0, nd, nn, (const int *)hs->leaf_halo, pure);
    for (int level = t->n_levels - 1; level >= 1; level--)
        RS_LAUNCH(ctx, "hp_up", k_hp_up, ceil_div(nn, 256), 256, 0, nd, nn, level, pure);
    RS_LAUNCH(ctx, "hp_fill", k_hp_fill_u64, ceil_div(2 * H, 256), 256, 0, eb, 2 * H, ~0ull);
    for (int pass = 0; pass < 3; pass++)
        RS_LAUNCH(ctx, "hp_best", k_hp_best, ceil_div(nn, 256), 256, 0, nd, nn, (const int *)pure, pass, eb, eb + H,
                  centre_node, xc, vc);
    unsigned *sid, *srank, *groot, *grank;
    RS_TRY(sorted_ids(ctx, hs, &sid, &srank, &groot, &grank));
    unsigned long long *na = (unsigned long long *)n_assigned;
    RS_CUDA(ctx, cudaMemsetAsync(na, 0, sizeof(int64_t) * H, ctx->stream));
    RS_LAUNCH(ctx, "hp_count", k_hp_count, ceil_div(n, 256), 256, 0, n, halo_id, (const unsigned *)sid,
              (const unsigned *)srank, (int)H, na, ctx->d_status);
    RS_LAUNCH(ctx, "hp_host", k_hp_host, ceil_div(H, 128), 128, 0, (int)H, *hs, (const double *)xc,
              (const double *)vc, (const unsigned long long *)na, (const unsigned *)groot, (const unsigned *)grank,
              t->box, host);
    return rs_sync_check(ctx, "rs_halo_props");
}

extern "C" rs_status rs_unbind(rs_ctx *ctx, const rs_tree *t, const rs_halos *hs, const int32_t *halo_id,
                               const int32_t *host, const float *pos, const float *vel, int32_t stride, int64_t n,
                               double gm, double eps, double theta, int64_t *n_part, int64_t *n_bound,
                               double *vbulk, int8_t *bound_own, double *phi_own)
{
    RsRange range("rs_unbind");
    if (!ctx) return RS_ERR_INVALID_ARG;
    if (!t || !hs || n != t->n_total || (stride != 3 && stride != 4) || !(gm >= 0) || !(eps >= 0) ||
        !(theta >= 0 && theta < 1) || (n > 0 && (!halo_id || !pos || !vel || !bound_own)))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_unbind: bad argument");
    const int tree_on = theta > 0 ? 1 : 0;
    if (n == 0) return RS_OK;
    RS_LAUNCH(ctx, "ub_fill", k_ub_fill_i8, std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->num_sms * 16), 256, 0,
              bound_own, n, (int8_t)-1);
    const int64_t H = hs->n_halos;
    if (H == 0) return RS_OK;
    if (!host || !n_part || !n_bound || !vbulk)
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_unbind: an output is NULL");
    unsigned *sid, *srank, *groot, *grank;
    RS_TRY(sorted_ids(ctx, hs, &sid, &srank, &groot, &grank));
    RS_WS(ctx, int, up, WS_HL_PURE, H + 8);
    RS_LAUNCH(ctx, "ub_up", k_ub_up, ceil_div(H, 256), 256, 0, (int)H, host, (const unsigned *)sid,
              (const unsigned *)srank, up, ctx->d_status);
    RS_WS(ctx, unsigned long long, cnt, WS_HL_BEST, 4);
    RS_CUDA(ctx, cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), ctx->stream));
    RS_LAUNCH(ctx, "ub_count", k_ub_count, ceil_div(n, 256), 256, 0, n, halo_id, (const unsigned *)sid,
              (const unsigned *)srank, (int)H, (const int *)up, cnt, ctx->d_status);
    int64_t total = 0;
    RS_TRY(rs_read_i64(ctx, cnt, 1, &total, "rs_unbind"));
    if (total >= ((int64_t)1 << 32)) return rs_fail(ctx, RS_ERR_TOO_LARGE, "rs_unbind: sets hold 2^32 entries");
    RS_WS(ctx, uint64_t, k0, WS_SORT_K0, total);
    RS_WS(ctx, uint64_t, k1, WS_SORT_K1, total);
    RS_WS(ctx, uint32_t, v0, WS_SORT_V0, total);
    RS_WS(ctx, uint32_t, v1, WS_SORT_V1, total);
    RS_LAUNCH(ctx, "ub_keys", k_ub_keys, ceil_div(n, 256), 256, 0, n, halo_id, (const unsigned *)sid,
              (const unsigned *)srank, (int)H, (const int *)up, cnt + 1, total, k0, v0, ctx->d_status);
    RS_TRY(rs_sync_check(ctx, "rs_unbind"));
    int rbits = 0;
    while (rbits < 32 && ((uint64_t)(H - 1) >> rbits) != 0) rbits++;
    bool alt = false;
    if (total > 0) RS_TRY(rs_radix_sort_u64(ctx, k0, k1, v0, v1, total, 32 + rbits, &alt));
    const uint64_t *sk = alt ? k1 : k0;
    const uint32_t *smem = alt ? v1 : v0;
    RS_WS(ctx, int64_t, ob, WS_HL_OFF, 2 * (H + 1) + 8);
    int64_t *off = ob, *toff = ob + (H + 1);
    if (total > 0)
        RS_LAUNCH(ctx, "ub_bounds", k_ub_bounds, ceil_div(total, 256), 256, 0, total, sk, off, (int)H);
    else
        RS_CUDA(ctx, cudaMemsetAsync(off, 0, sizeof(int64_t) * (H + 1), ctx->stream));
    RS_LAUNCH(ctx, "ub_bulk", k_ub_bulk, std::min<int64_t>(H, (int64_t)ctx->num_sms * 8), HP_THREADS, 0, (int)H,
              (const int64_t *)off, smem, vel, stride, vbulk);
    RS_LAUNCH(ctx, "ub_tiles", k_ub_tiles, ceil_div(H, 256), 256, 0, (int)H, (const int64_t *)off, tree_on, toff);
    RS_CUDA(ctx, cudaMemsetAsync(toff + H, 0, sizeof(int64_t), ctx->stream));
    RS_TRY(rs_scan_i64(ctx, toff, H + 1, nullptr));
    int64_t T = 0;
    RS_TRY(rs_read_i64(ctx, toff + H, 1, &T, "rs_unbind"));
    RS_WS(ctx, int, tm, WS_HL_TILES, 2 * T + 8);
    RS_LAUNCH(ctx, "ub_tilemap", k_ub_tilemap, H, 128, 0, (int)H, (const int64_t *)toff, tm, tm + T);
    RS_CUDA(ctx, cudaMemsetAsync(n_bound, 0, sizeof(int64_t) * H, ctx->stream));
    if (T > 0)
        RS_LAUNCH(ctx, "ub_phi", k_ub_phi, T, UB_TILE, 0, (const int *)tm, (const int *)(tm + T),
                  (const int64_t *)off, smem, pos, vel, stride, (float)t->box, gm, (float)(eps * eps),
                  (const double *)vbulk, halo_id, (const int *)hs->id, (unsigned long long *)n_bound, bound_own,
                  phi_own);
    if (tree_on && total > 0) {
        // the sets above UB_DIRECT_MAX members: Morton order, boxes, tree walk
        RS_WS(ctx, int64_t, tb, WS_HL_TREE, 2 * (H + 1) + 8);
        int64_t *nbox = tb, *nleaf = tb + (H + 1);
        RS_LAUNCH(ctx, "ub_boxcount", k_ub_boxcount, ceil_div(H, 256), 256, 0, (int)H, (const int64_t *)off,
                  tree_on, nbox, nleaf);
        RS_CUDA(ctx, cudaMemsetAsync(nbox + H, 0, sizeof(int64_t), ctx->stream));
        RS_CUDA(ctx, cudaMemsetAsync(nleaf + H, 0, sizeof(int64_t), ctx->stream));
        RS_TRY(rs_scan_i64(ctx, nbox, H + 1, nullptr));
        RS_TRY(rs_scan_i64(ctx, nleaf, H + 1, nullptr));
        int64_t NB = 0, NJ = 0;
        RS_TRY(rs_read_i64(ctx, nbox + H, 1, &NB, "rs_unbind"));
        RS_TRY(rs_read_i64(ctx, nleaf + H, 1, &NJ, "rs_unbind"));
        if (NJ > 0) {
            const float boxf = (float)t->box;
            RS_WS(ctx, float4, rc, WS_HL_REF, 2 * H + 2);
            float4 *ref = rc, *cube = rc + H;
            RS_WS(ctx, float4, upos, WS_HL_UPOS, total);
            RS_WS(ctx, float4, tpos, WS_HL_TPOS, total);
            RS_WS(ctx, uint32_t, tmem, WS_HL_TMEM, total);
            RS_WS(ctx, uint64_t, mk0, WS_HL_MK0, total);
            RS_WS(ctx, uint64_t, mk1, WS_HL_MK1, total);
            RS_WS(ctx, uint32_t, mv0, WS_HL_MV0, total);
            RS_WS(ctx, uint32_t, mv1, WS_HL_MV1, total);
            RS_LAUNCH(ctx, "ub_ref", k_ub_ref, ceil_div(H, 256), 256, 0, (int)H, (const int64_t *)off, smem, pos,
                      stride, ref);
            RS_LAUNCH(ctx, "ub_upos", k_ub_upos, ceil_div(total, 256), 256, 0, total, sk, smem, pos, stride,
                      (const float4 *)ref, boxf, upos);
            RS_LAUNCH(ctx, "ub_bbox", k_ub_bbox, std::min<int64_t>(H, (int64_t)ctx->num_sms * 4), HP_THREADS, 0,
                      (int)H, (const int64_t *)off, tree_on, (const float4 *)upos, cube);
            RS_LAUNCH(ctx, "ub_morton", k_ub_morton, ceil_div(total, 256), 256, 0, total, sk, (const int64_t *)off,
                      tree_on, (const float4 *)upos, (const float4 *)cube, mk0, mv0);
            bool malt = false;
            RS_TRY(rs_radix_sort_u64(ctx, mk0, mk1, mv0, mv1, total, 30 + rbits, &malt));
            RS_LAUNCH(ctx, "ub_gather", k_ub_gather, ceil_div(total, 256), 256, 0, total,
                      (const uint32_t *)(malt ? mv1 : mv0), (const float4 *)upos, smem, tpos, tmem);
            RS_WS(ctx, float4, bx, WS_HL_BOX, 2 * NB + 2);
            UBoxes B;
            B.c = bx;
            B.s = bx + NB;
            RS_WS(ctx, int, jb, WS_HL_JOBS, 2 * NJ + 8);
            int *jset = jb, *jleaf = jb + NJ;
            RS_LAUNCH(ctx, "ub_leafjobs", k_ub_leafjobs, H, 128, 0, (int)H, (const int64_t *)nleaf, jset, jleaf);
            RS_LAUNCH(ctx, "ub_leafbox", k_ub_leafbox, ceil_div(NJ, UT_WARPS), UT_WARPS * 32, 0, NJ,
                      (const int *)jset, (const int *)jleaf, (const int64_t *)off, (const int64_t *)nbox,
                      (const float4 *)tpos, (float)theta, B);
            RS_LAUNCH(ctx, "ub_upper", k_ub_upper, std::min<int64_t>(H, (int64_t)ctx->num_sms * 4), HP_THREADS, 0,
                      (int)H, (const int64_t *)off, tree_on, (const int64_t *)nbox, (float)theta, B);
            RS_LAUNCH(ctx, "ub_walk", k_ub_walk, ceil_div(NJ, UT_WARPS), UT_WARPS * 32, 0, NJ, (const int *)jset,
                      (const int *)jleaf, (const int64_t *)off, (const int64_t *)nbox, (const float4 *)tpos,
                      (const uint32_t *)tmem, B, gm, (float)(eps * eps), vel, stride, (const double *)vbulk,
                      halo_id, (const int *)hs->id, (unsigned long long *)n_bound, bound_own, phi_own,
                      ctx->d_status);
        }
    }
    RS_LAUNCH(ctx, "ub_npart", k_ub_npart, ceil_div(H, 256), 256, 0, (int)H, (const int64_t *)off, n_part);
    return rs_sync_check(ctx, "rs_unbind");
}

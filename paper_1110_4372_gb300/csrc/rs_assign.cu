// rs_assign.cu -- seeds, seed merge and hierarchical assignment (Sec. 3.3).
//
//  1. Seeds are the tree's leaves, sorted by their first member slot; the
//     seeds under any node are then a contiguous run of that list.
//  2. Merge (Eq. 2): every pair of seeds of one 3D group is tested in
//     float64 with the unmerged properties; merges are closed by union-find.
//  3. Halo properties: exact moments over the union of a halo's seed
//     members; r_dyn,vir^2 = max_k (k / r_(k)) / (4/3 pi delta nbar) (Eq. 4,
//     G and the particle mass cancel) from the sorted float64 member radii.
//  4. Assignment: every member slot is decided at the deepest node holding
//     it -- the node whose range holds the slot outside all of its children.
//     One halo among the node's seeds: that halo.  Several: the Eq. 3
//     nearest, found in float32 with every halo inside a 2^-20 band of the
//     best re-evaluated in float64 (ties to the smaller halo id).
#include <cmath>
#include <new>

#include "rs_refine.cuh"

namespace {

constexpr int AS_THREADS = 256;
constexpr int RDYN_SMEM_N = 4096;

__device__ __forceinline__ double min_image64(double d, double box)
{
    if (d > 0.5 * box) d = f64_sub(d, box);
    else if (d < -0.5 * box) d = f64_add(d, box);
    return d;
}

// zero-dispersion reading: 0/0 contributes 0, x/0 is infinite
__device__ __forceinline__ double ratio2(double num, double den)
{
    if (den > 0) return __ddiv_rn(num, den);
    return num > 0 ? INFINITY : 0.0;
}

struct AsBufs {
    int L;                 // seeds
    const int *leaf_node;  // by rank of first slot
    const unsigned *leaf_first;
    int *uf;               // union-find over seeds
    int *hid;              // per root seed: halo id (smallest particle index)
    MomAcc *hacc;
    float4 *href;          // per root seed: reference position, velocity
    unsigned long long *hcount;
    double *hx, *hv, *hsigv, *hrdyn2;  // per root seed (hx, hv: 3 each)
    float *hfast;          // per root seed: 12 floats (centre hi/lo, velocity hi/lo) + 2 factors
    int *hrank;            // per root seed: dense halo rank
    int *span;             // per node: members held by its children
};

__device__ __forceinline__ float4 unwrap_pos(const float *pos, int stride, int i, int shift, float boxf)
{
    const float *p = pos + (int64_t)stride * i;
    float x = p[0], y = p[1], z = p[2];
    if ((shift & 1) && x >= 0.5f * boxf) x = x - boxf;
    if ((shift & 2) && y >= 0.5f * boxf) y = y - boxf;
    if ((shift & 4) && z >= 0.5f * boxf) z = z - boxf;
    return make_float4(x, y, z, 0.f);
}

__device__ __forceinline__ float4 load_vel(const float *vel, int stride, int i)
{
    const float *p = vel + (int64_t)stride * i;
    return make_float4(p[0], p[1], p[2], 0.f);
}

__global__ void k_as_leafflag(NodeArrays nd, int nn, unsigned *flag, int *span)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    flag[i] = nd.nchild[i] == 0 ? 1u : 0u;
    span[i] = 0;
}

__global__ void k_as_span(NodeArrays nd, int nn, int *span)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int p = nd.parent[i];
    if (p >= 0) atomicAdd(&span[p], nd.count[i]);
}

__global__ void k_as_leafcompact(NodeArrays nd, int nn, const unsigned *flag, const unsigned *scan, unsigned *keys,
                                 unsigned *vals)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn || !flag[i]) return;
    keys[scan[i]] = (unsigned)nd.first[i];
    vals[scan[i]] = (unsigned)i;
}

__global__ void k_as_init(AsBufs A)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.L) return;
    A.uf[a] = a;
    A.hid[a] = 0x7fffffff;
    A.hcount[a] = 0;
    A.hrank[a] = -1;
}

// Eq. 2 separation with the smaller seed's Poisson uncertainties
__device__ double merge_distance(const NodeArrays &nd, int a, int b, double box)
{
    const int na = nd.count[a], nb = nd.count[b];
    const bool a_small = (na != nb) ? (na < nb) : (nd.minidx[a] > nd.minidx[b]);
    const int s = a_small ? a : b;
    const double rn = sqrt((double)nd.count[s]);
    const double mux = __ddiv_rn(nd.sigx[s], rn), muv = __ddiv_rn(nd.sigv[s], rn);
    double dx2 = 0, dv2 = 0;
    for (int d = 0; d < 3; d++) {
        double dx = min_image64(f64_sub(nd.xbar[3 * a + d], nd.xbar[3 * b + d]), box);
        double dv = f64_sub(nd.vbar[3 * a + d], nd.vbar[3 * b + d]);
        dx2 = f64_add(dx2, f64_mul(dx, dx));
        dv2 = f64_add(dv2, f64_mul(dv, dv));
    }
    return sqrt(f64_add(ratio2(dx2, f64_mul(mux, mux)), ratio2(dv2, f64_mul(muv, muv))));
}

// A float32 lower bound of the squared Eq. 2 separation: each coordinate gap
// is shrunk by a bound on the rounding of the float32 copies (2^-22 of the
// coordinates' size covers both roundings and the subtraction), and the
// comparison keeps a 2^-10 relative margin for the float32 products and
// sums.  Returns false when the pair may be within the threshold (or a
// dispersion is zero): the float64 test then decides.
__device__ __forceinline__ bool merge_far_f32(const NodeArrays &nd, int a, int b, float boxf, float thresh2)
{
    const int na = nd.count[a], nb = nd.count[b];
    const bool a_small = (na != nb) ? (na < nb) : (nd.minidx[a] > nd.minidx[b]);
    const int s = a_small ? a : b;
    const float sx = (float)nd.sigx[s], sv = (float)nd.sigv[s];
    if (!(sx > 1e-30f) || !(sv > 1e-30f)) return false;
    float gx2 = 0.f, gv2 = 0.f;
    for (int d = 0; d < 3; d++) {
        const float xa = (float)nd.xbar[3 * a + d], xb = (float)nd.xbar[3 * b + d];
        float dx = fabsf(xa - xb);
        dx = fminf(dx, boxf - dx);
        const float ex = 2.384185791015625e-07f * (fabsf(xa) + fabsf(xb) + boxf);
        const float lx = fmaxf(0.f, dx - ex);
        gx2 += lx * lx;
        const float va = (float)nd.vbar[3 * a + d], vb = (float)nd.vbar[3 * b + d];
        const float ev = 2.384185791015625e-07f * (fabsf(va) + fabsf(vb));
        const float lv = fmaxf(0.f, fabsf(va - vb) - ev);
        gv2 += lv * lv;
    }
    const float ns = (float)nd.count[s];
    const float d2 = gx2 * ns / (sx * sx) + gv2 * ns / (sv * sv);
    return d2 > thresh2 * 1.0009765625f;
}

__global__ void k_as_merge(AsBufs A, NodeArrays nd, double box, double thresh, rs_dev_status *st)
{
    const float boxf = (float)box, thresh2 = (float)(thresh * thresh);
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < A.L; a += gridDim.x * blockDim.x) {
        const int na = A.leaf_node[a];
        const int ra = nd.root[na];
        for (int b = a + 1; b < A.L; b++) {
            const int nb = A.leaf_node[b];
            if (nd.root[nb] != ra) break;
            if (merge_far_f32(nd, na, nb, boxf, thresh2)) continue;
            if (merge_distance(nd, na, nb, box) < thresh) uf_union(A.uf, a, b, st);
        }
    }
}

__global__ void k_as_roots(AsBufs A, NodeArrays nd, const int *members, const float *pos, const float *vel,
                           int stride, float boxf, rs_dev_status *st)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.L) return;
    const int node = A.leaf_node[a];
    const int r = uf_find(A.uf, a, st);
    atomicMin(&A.hid[r], nd.minidx[node]);
    atomicAdd(&A.hcount[r], (unsigned long long)nd.count[node]);
    if (r == a) {
        const int i = members[nd.first[node]];
        A.href[2 * a] = unwrap_pos(pos, stride, i, nd.shift[node], boxf);
        A.href[2 * a + 1] = load_vel(vel, stride, i);
    }
}

__global__ void __launch_bounds__(AS_THREADS) k_as_hmom(AsBufs A, NodeArrays nd, const int *members, const float *pos,
                                                        const float *vel, int stride, float boxf, rs_dev_status *st)
{
    __shared__ MomAcc w[AS_THREADS / 32];
    for (int a = blockIdx.x; a < A.L; a += gridDim.x) {
        const int node = A.leaf_node[a];
        const int r = uf_find(A.uf, a, st);
        const MomRef ref = mom_ref(A.href[2 * r], A.href[2 * r + 1]);
        const int first = nd.first[node], cnt = nd.count[node], sh = nd.shift[node];
        MomAcc acc;
        mom_zero(acc);
        for (int m = threadIdx.x; m < cnt; m += AS_THREADS) {
            const int i = members[first + m];
            mom_add(acc, unwrap_pos(pos, stride, i, sh, boxf), load_vel(vel, stride, i), ref);
        }
        mom_warp_reduce(acc);
        if (lane_id() == 0) w[warp_id()] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            MomAcc t = w[0];
            for (int k = 1; k < AS_THREADS / 32; k++) mom_merge(t, w[k]);
            mom_atomic_add(&A.hacc[r], t);
        }
        __syncthreads();
    }
}

__global__ void k_as_hfin(AsBufs A, double box, unsigned *rootflag)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.L) return;
    const bool is_root = A.uf[a] == a;
    rootflag[a] = is_root ? 1u : 0u;
    if (!is_root) return;
    const float4 pr = A.href[2 * a], vr = A.href[2 * a + 1];
    MomOut o = mom_finalize(A.hacc[a], pr, vr, (int64_t)A.hcount[a], box);
    for (int d = 0; d < 3; d++) {
        A.hx[3 * a + d] = o.xbar[d];
        A.hv[3 * a + d] = o.vbar[d];
    }
    A.hsigv[a] = o.sigv;
    // centre in the group's unwrapped frame, as a float pair
    const double cnt = (double)A.hcount[a];
    const float prc[3] = {pr.x, pr.y, pr.z};
    float *f = A.hfast + 16 * (int64_t)a;
    for (int d = 0; d < 3; d++) {
        double xu = (double)prc[d] + s128_to_double(A.hacc[a].s_lo[d], A.hacc[a].s_hi[d]) * RS_FX_INV / cnt;
        float hi = (float)xu;
        f[d] = hi;
        f[3 + d] = (float)(xu - (double)hi);
        float vh = (float)o.vbar[d];
        f[6 + d] = vh;
        f[9 + d] = (float)(o.vbar[d] - (double)vh);
    }
}

__global__ void k_as_hrank(AsBufs A, const unsigned *rootflag, const unsigned *rscan, unsigned long long *hoff)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.L || !rootflag[a]) return;
    const int k = (int)rscan[a];
    A.hrank[a] = k;
    hoff[k] = A.hcount[a];
}

__global__ void k_as_hmembers(AsBufs A, NodeArrays nd, const unsigned long long *hoff, unsigned long long *hfill,
                              int *hmem, rs_dev_status *st)
{
    for (int a = blockIdx.x; a < A.L; a += gridDim.x) {
        __shared__ unsigned long long base;
        const int node = A.leaf_node[a];
        const int cnt = nd.count[node], first = nd.first[node];
        if (threadIdx.x == 0) {
            const int k = A.hrank[uf_find(A.uf, a, st)];
            base = hoff[k] + atomicAdd(&hfill[k], (unsigned long long)cnt);
        }
        __syncthreads();
        for (int m = threadIdx.x; m < cnt; m += blockDim.x) hmem[base + m] = first + m;
        __syncthreads();
    }
}

// r_dyn,vir (Eq. 4): one block per halo
__global__ void __launch_bounds__(AS_THREADS) k_as_rdyn(AsBufs A, int n_halos, const int *root_of_rank,
                                                        const unsigned long long *hoff, const int *hmem,
                                                        const int *members, const float *pos, int stride,
                                                        double box, double rho_term)
{
    __shared__ unsigned long long key[RDYN_SMEM_N];
    __shared__ double wbest[AS_THREADS / 32];
    for (int k = blockIdx.x; k < n_halos; k += gridDim.x) {
        const int r = root_of_rank[k];
        const unsigned long long a0 = hoff[k], s = hoff[k + 1] - hoff[k];
        const double xb[3] = {A.hx[3 * r], A.hx[3 * r + 1], A.hx[3 * r + 2]};
        double best = 0.0;
        auto radius = [&](unsigned long long m) {
            const int i = members[hmem[a0 + m]];
            const float *p = pos + (int64_t)stride * i;
            double acc = 0.0;
            for (int d = 0; d < 3; d++) {
                double dx = min_image64(f64_sub((double)p[d], xb[d]), box);
                acc = f64_add(acc, f64_mul(dx, dx));
            }
            return sqrt(acc);
        };
        if (s <= RDYN_SMEM_N) {
            int P = 1;
            while ((unsigned long long)P < s) P <<= 1;
            for (int m = threadIdx.x; m < P; m += AS_THREADS)
                key[m] = (unsigned long long)m < s ? (unsigned long long)__double_as_longlong(radius(m)) : ~0ull;
            __syncthreads();
            for (int kk = 2; kk <= P; kk <<= 1)
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    for (int t = threadIdx.x; t < P / 2; t += AS_THREADS) {
                        int i = 2 * j * (t / j) + (t % j), l = i + j;
                        bool up = (i & kk) == 0;
                        unsigned long long x = key[i], y = key[l];
                        if ((x > y) == up) {
                            key[i] = y;
                            key[l] = x;
                        }
                    }
                    __syncthreads();
                }
            for (int m = threadIdx.x; (unsigned long long)m < s; m += AS_THREADS) {
                double rr = __longlong_as_double((long long)key[m]);
                if (rr > 0) best = fmax(best, __ddiv_rn((double)(m + 1), rr));
            }
        } else {
            continue;  // large halo: handled by the sort-based kernels below
        }
        best = warp_max(best);
        if (lane_id() == 0) wbest[warp_id()] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = wbest[0];
            for (int w = 1; w < AS_THREADS / 32; w++) b = fmax(b, wbest[w]);
            const double r2 = __ddiv_rn(b, rho_term);
            A.hrdyn2[r] = r2;
            const double sv2 = f64_mul(A.hsigv[r], A.hsigv[r]);
            float *f = A.hfast + 16 * (int64_t)r;
            f[12] = r2 > 0 ? (float)(1.0 / r2) : -1.f;   // -1: zero denominator, float64 only
            f[13] = sv2 > 0 ? (float)(1.0 / sv2) : -1.f;
        }
        __syncthreads();
    }
}

// ---- r_dyn of halos above RDYN_SMEM_N members: one global sort ----
// Members of large halos get keys (large-halo rank, float32 radius) -- float32
// rounding is monotone, so the order is the float64 order up to runs of
// equal float32 keys, inside which each member's exact float64 rank is
// counted directly.  max_k k / r_(k) is then taken per halo with a 64-bit
// atomic max on the (positive) double's bits.
__global__ void k_as_large_flag(int n_halos, const unsigned long long *hoff, unsigned *lflag)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_halos) return;
    lflag[k] = (hoff[k + 1] - hoff[k]) > (unsigned long long)RDYN_SMEM_N ? 1u : 0u;
}

__global__ void k_as_large_size(int n_halos, const unsigned long long *hoff, const unsigned *lflag,
                                const unsigned *lscan, long long *lsize, int *lhalo)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_halos || !lflag[k]) return;
    lsize[lscan[k]] = (long long)(hoff[k + 1] - hoff[k]);
    lhalo[lscan[k]] = k;
}

__global__ void k_as_large_keys(int nlarge, const long long *loff, const int *lhalo, const int *root_of_rank,
                                const unsigned long long *hoff, const int *hmem, const int *members, const float *pos,
                                int stride, double box, AsBufs A, unsigned long long *keys, unsigned *vals,
                                double *r64)
{
    for (int li = blockIdx.x; li < nlarge; li += gridDim.x) {
        const int k = lhalo[li];
        const int r = root_of_rank[k];
        const unsigned long long a0 = hoff[k], s = hoff[k + 1] - hoff[k];
        const long long o = loff[li];
        for (unsigned long long m = threadIdx.x; m < s; m += blockDim.x) {
            const int i = members[hmem[a0 + m]];
            const float *p = pos + (int64_t)stride * i;
            double acc = 0.0;
            for (int d = 0; d < 3; d++) {
                double dx = min_image64(f64_sub((double)p[d], A.hx[3 * r + d]), box);
                acc = f64_add(acc, f64_mul(dx, dx));
            }
            const double rr = sqrt(acc);
            r64[o + m] = rr;
            keys[o + m] = ((unsigned long long)li << 32) | __float_as_uint((float)rr);
            vals[o + m] = (unsigned)(o + m);
        }
    }
}

__global__ void k_as_large_max(long long total, const long long *loff, const unsigned long long *keys,
                               const unsigned *vals, const double *r64, unsigned long long *best_bits)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const unsigned long long key = keys[t];
    const int li = (int)(key >> 32);
    const long long start = loff[li];
    const double r = r64[vals[t]];
    if (!(r > 0)) return;
    // bounds of the run of equal keys holding t
    long long a = t, b = t + 1;
    while (a > start && keys[a - 1] == key) a--;
    while (b < total && keys[b] == key) b++;
    long long rank = a - start;
    for (long long u = a; u < b; u++) rank += r64[vals[u]] <= r ? 1 : 0;
    const double v = __ddiv_rn((double)rank, r);
    atomicMax(&best_bits[li], (unsigned long long)__double_as_longlong(v));
}

__global__ void k_as_large_fin(int nlarge, const int *lhalo, const int *root_of_rank,
                               const unsigned long long *best_bits, AsBufs A, double rho_term)
{
    int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nlarge) return;
    const int r = root_of_rank[lhalo[li]];
    const double b = __longlong_as_double((long long)best_bits[li]);
    const double r2 = __ddiv_rn(b, rho_term);
    A.hrdyn2[r] = r2;
    const double sv2 = f64_mul(A.hsigv[r], A.hsigv[r]);
    float *f = A.hfast + 16 * (int64_t)r;
    f[12] = r2 > 0 ? (float)(1.0 / r2) : -1.f;
    f[13] = sv2 > 0 ? (float)(1.0 / sv2) : -1.f;
}

__global__ void k_as_tiles_prep(NodeArrays nd, int nn, const int *span, int64_t *tiles)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    tiles[i] = ceil_div(nd.count[i] - span[i], AS_THREADS);
}

__global__ void k_as_tiles_fill(int nn, const int64_t *toff, int *tnode, int *tq0)
{
    for (int i = blockIdx.x; i < nn; i += gridDim.x) {
        const int64_t a = toff[i], b = toff[i + 1];
        for (int64_t t = a + threadIdx.x; t < b; t += blockDim.x) {
            tnode[t] = i;
            tq0[t] = (int)((t - a) * AS_THREADS);
        }
    }
}

__device__ __forceinline__ int lower_bound_u32(const unsigned *a, int n, unsigned v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

constexpr int AS_CAND = 4096;  // seeds deduplicated in shared memory per node

__global__ void k_as_leafroot(AsBufs A, int *leaf_root, rs_dev_status *st)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.L) return;
    leaf_root[a] = uf_find(A.uf, a, st);
}

__device__ __forceinline__ float as_d2_32(float4 p, float4 v, const float *f)
{
    float dx = (p.x - f[0]) - f[3], dy = (p.y - f[1]) - f[4], dz = (p.z - f[2]) - f[5];
    float ux = (v.x - f[6]) - f[9], uy = (v.y - f[7]) - f[10], uz = (v.z - f[8]) - f[11];
    return (dx * dx + dy * dy + dz * dz) * f[12] + (ux * ux + uy * uy + uz * uz) * f[13];
}

// One block per tile of a node's own members (those outside its children).
// The node's seeds are the seed-list run [la, lb); their halos are
// deduplicated in shared memory, then each member takes the only halo or the
// Eq. 3 nearest one (float32 pass, float64 over the float32 band).
// Seeds under each node: the first (la) and how many (nl).
__global__ void k_as_nl(AsBufs A, NodeArrays nd, int nn, int *node_la, int64_t *nlv)
{
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= nn) return;
    const int first = nd.first[node], cnt = nd.count[node];
    const int la = lower_bound_u32(A.leaf_first, A.L, (unsigned)first);
    const int lb = lower_bound_u32(A.leaf_first, A.L, (unsigned)(first + cnt));
    node_la[node] = la;
    nlv[node] = lb - la;
}

// The distinct candidate halos (roots of the seeds under a node), once per
// node: the node's first tile sorts the seeds' roots in shared memory and
// keeps the first of each run, into the node's own region cand_g[coff ..).
// ncand[node] = the list's length, or -(seeds) - 1 when there are too many
// seeds to stage, in which case the raw roots stand in (repeats only cost
// time).
__global__ void __launch_bounds__(AS_THREADS) k_as_cand(AsBufs A, NodeArrays nd, const int *leaf_root,
                                                        const int *tnode, const int *tq0, const int *node_la,
                                                        const int64_t *coff, int *cand_g, int *ncand)
{
    __shared__ int cand[AS_CAND];
    __shared__ int wsum[AS_THREADS / 32];
    if (tq0[blockIdx.x] != 0) return;
    const int node = tnode[blockIdx.x];
    const int la = node_la[node];
    const int nl = (int)(coff[node + 1] - coff[node]);
    int *out = cand_g + coff[node];
    if (nl > AS_CAND || nl <= 0) {
        if (threadIdx.x == 0) ncand[node] = -nl - 1;
        return;
    }
    int P = 1;
    while (P < nl) P <<= 1;
    for (int i = threadIdx.x; i < P; i += AS_THREADS) cand[i] = i < nl ? leaf_root[la + i] : 0x7fffffff;
    __syncthreads();
    for (int kk = 2; kk <= P; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += AS_THREADS) {
                int i = 2 * j * (t / j) + (t % j), l = i + j;
                bool up = (i & kk) == 0;
                int x = cand[i], y = cand[l];
                if ((x > y) == up) {
                    cand[i] = y;
                    cand[l] = x;
                }
            }
            __syncthreads();
        }
    // first of each run: a block-wide exclusive scan of the run-start flags
    const int per = (nl + AS_THREADS - 1) / AS_THREADS;
    const int i0 = threadIdx.x * per, i1 = min(nl, i0 + per);
    int c = 0;
    for (int i = i0; i < i1; i++) c += (i == 0 || cand[i] != cand[i - 1]) ? 1 : 0;
    int x = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane_id() >= o) x += y;
    }
    if (lane_id() == 31) wsum[warp_id()] = x;
    __syncthreads();
    int pre = 0;
    for (int w = 0; w < warp_id(); w++) pre += wsum[w];
    int o = pre + x - c;
    for (int i = i0; i < i1; i++)
        if (i == 0 || cand[i] != cand[i - 1]) out[o++] = cand[i];
    if (threadIdx.x == AS_THREADS - 1) ncand[node] = pre + x;
}

__global__ void __launch_bounds__(AS_THREADS) k_as_assign(AsBufs A, NodeArrays nd, const int *leaf_root,
                                                          const int *cand_g, const int *node_la, const int64_t *coff,
                                                          const int *ncand,
                                                          const int *tnode, const int *tq0, const int *members,
                                                          const float *pos, const float *vel, int stride,
                                                          double box, float boxf, int32_t *halo_id,
                                                          rs_dev_status *st)
{
    const int node = tnode[blockIdx.x];
    const int q0 = tq0[blockIdx.x];
    const int first = nd.first[node], cnt = nd.count[node];
    const int tail0 = first + A.span[node];
    const int la = node_la[node], nq = ncand[node];
    // candidate halo roots: the distinct list, or the raw roots (with repeats)
    const int nc = nq >= 0 ? nq : -nq - 1;
    const int *cl = nq >= 0 ? cand_g + coff[node] : leaf_root + la;
    const int m = tail0 + q0 + threadIdx.x;
    if (m >= first + cnt) return;
    const int i = members[m];
    if (nc <= 0) {
        dev_fail(st, DEV_INTERNAL, 60, node);
        return;
    }
    if (nc == 1) {
        halo_id[i] = A.hid[cl[0]];
        return;
    }
    const float4 p = unwrap_pos(pos, stride, i, nd.shift[node], boxf);
    const float4 v = load_vel(vel, stride, i);
    float best = INFINITY;
    bool need64 = false;
    for (int c = 0; c < nc; c++) {
        const float *f = A.hfast + 16 * (int64_t)cl[c];
        if (f[12] < 0.f || f[13] < 0.f) {
            need64 = true;
            continue;
        }
        best = fminf(best, as_d2_32(p, v, f));
    }
    const float lim = best * (float)(1.0 + 2.0 * RS_BAND);
    double b64 = INFINITY;
    int bid = 0x7fffffff;
    const float *pr = pos + (int64_t)stride * i;
    const float *vr = vel + (int64_t)stride * i;
    for (int c = 0; c < nc; c++) {
        const int r = cl[c];
        const float *f = A.hfast + 16 * (int64_t)r;
        const bool zero = f[12] < 0.f || f[13] < 0.f;
        if (!zero) {
            if (as_d2_32(p, v, f) > lim) continue;
        } else if (!need64) {
            continue;
        }
        double dx2 = 0, dv2 = 0;
        for (int d = 0; d < 3; d++) {
            double dx = min_image64(f64_sub(A.hx[3 * r + d], (double)pr[d]), box);
            double dv = f64_sub(A.hv[3 * r + d], (double)vr[d]);
            dx2 = f64_add(dx2, f64_mul(dx, dx));
            dv2 = f64_add(dv2, f64_mul(dv, dv));
        }
        const double sv = A.hsigv[r];
        const double d2 = f64_add(ratio2(dx2, A.hrdyn2[r]), ratio2(dv2, f64_mul(sv, sv)));
        const int id = A.hid[r];
        if (d2 < b64 || (d2 == b64 && id < bid)) {
            b64 = d2;
            bid = id;
        }
    }
    halo_id[i] = bid;
}

__global__ void k_fill_i32v(int32_t *p, int64_t n, int32_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_as_root_of_rank(AsBufs A, int *root_of_rank)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.L) return;
    if (A.hrank[a] >= 0) root_of_rank[A.hrank[a]] = a;
}

// per-halo results in rank order, and every seed's halo rank
__global__ void k_as_export(AsBufs A, NodeArrays nd, int H, const int *root_of_rank, rs_halos out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const int s = root_of_rank[r];
    out.id[r] = A.hid[s];
    for (int d = 0; d < 3; d++) {
        out.xbar[3 * r + d] = A.hx[3 * s + d];
        out.vbar[3 * r + d] = A.hv[3 * s + d];
    }
    out.sigv[r] = A.hsigv[s];
    out.rdyn2[r] = A.hrdyn2[s];
    out.root[r] = nd.root[A.leaf_node[s]];
}

__global__ void k_as_export_leaf(AsBufs A, const int *leaf_root, int *leaf_halo)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.L) return;
    leaf_halo[A.leaf_node[a]] = A.hrank[leaf_root[a]];
}

rs_status empty_halos(rs_halos **out)
{
    *out = new (std::nothrow) rs_halos();
    return *out ? RS_OK : RS_ERR_OOM;
}

template <typename T>
T *carve(char *&p, int64_t count)
{
    T *r = (T *)p;
    size_t b = sizeof(T) * (size_t)(count > 0 ? count : 1);
    p += (b + 255) / 256 * 256;
    return r;
}

rs_status large_rdyn(rs_ctx *ctx, AsBufs A, int H, const int *root_of_rank, const unsigned long long *hoff,
                     const int *hmem, const int *members, const float *pos, int stride, double box, double rho_term)
{
    if (H == 0) return RS_OK;
    RS_WS(ctx, unsigned, lfl, WS_RF_MISC0, 2 * (int64_t)H + 8);
    unsigned *lflag = lfl, *lscan = lfl + H, *ltot = lfl + 2 * H;
    RS_LAUNCH(ctx, "as_large_flag", k_as_large_flag, ceil_div(H, 256), 256, 0, H, hoff, lflag);
    RS_CUDA(ctx, cudaMemcpyAsync(lscan, lflag, sizeof(unsigned) * H, cudaMemcpyDeviceToDevice, ctx->stream));
    RS_TRY(rs_scan_u32(ctx, lscan, H, ltot));
    RS_CUDA(ctx, cudaMemcpyAsync(ctx->h_scratch, ltot, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    RS_TRY(rs_sync_check(ctx, "rs_assign"));
    const int NL = (int)(*(unsigned *)ctx->h_scratch);
    if (NL == 0) return RS_OK;
    RS_WS(ctx, long long, lo, WS_RF_MISC1, 2 * (int64_t)NL + 8);
    long long *lsize = lo, *ltot2 = lo + NL + 1;
    int *lhalo = (int *)(lo + NL + 4);
    RS_CUDA(ctx, cudaMemsetAsync(lsize + NL, 0, sizeof(long long), ctx->stream));
    RS_LAUNCH(ctx, "as_large_size", k_as_large_size, ceil_div(H, 256), 256, 0, H, hoff, (const unsigned *)lflag,
              (const unsigned *)lscan, lsize, lhalo);
    RS_TRY(rs_scan_i64(ctx, (int64_t *)lsize, NL + 1, (int64_t *)ltot2));
    int64_t total;
    RS_TRY(rs_read_i64(ctx, lsize + NL, 1, &total, "rs_assign"));
    RS_WS(ctx, uint64_t, k0, WS_SORT_K0, total);
    RS_WS(ctx, uint64_t, k1, WS_SORT_K1, total);
    RS_WS(ctx, uint32_t, v0, WS_SORT_V0, total);
    RS_WS(ctx, uint32_t, v1, WS_SORT_V1, total);
    RS_WS(ctx, double, r64, WS_RF_DNN, total);
    RS_WS(ctx, unsigned long long, bb, WS_RF_MISC2, NL);
    RS_CUDA(ctx, cudaMemsetAsync(bb, 0, sizeof(unsigned long long) * NL, ctx->stream));
    RS_LAUNCH(ctx, "as_large_keys", k_as_large_keys, std::min<int64_t>(NL, (int64_t)ctx->num_sms * 4), 256, 0, NL,
              (const long long *)lsize, (const int *)lhalo, root_of_rank, hoff, hmem, members, pos, stride, box, A,
              (unsigned long long *)k0, v0, r64);
    int bits = 32;
    while (bits < 64 && ((uint64_t)(NL - 1) >> (bits - 32)) != 0) bits++;
    bool alt = false;
    RS_TRY(rs_radix_sort_u64(ctx, k0, k1, v0, v1, total, bits, &alt, "sort_as"));
    RS_LAUNCH(ctx, "as_large_max", k_as_large_max, ceil_div(total, 256), 256, 0, (long long)total,
              (const long long *)lsize, (const unsigned long long *)(alt ? k1 : k0), (const unsigned *)(alt ? v1 : v0),
              (const double *)r64, bb);
    RS_LAUNCH(ctx, "as_large_fin", k_as_large_fin, ceil_div(NL, 256), 256, 0, NL, (const int *)lhalo, root_of_rank,
              (const unsigned long long *)bb, A, rho_term);
    return RS_OK;
}

}  // namespace

extern "C" rs_status rs_assign_ex(rs_ctx *ctx, const rs_tree *t, const float *pos, const float *vel, int32_t stride,
                                  int64_t n, double box, const rs_params *params, int32_t *halo_id, int64_t *n_halos,
                                  rs_halos **halos_out)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    RsRange range("rs_assign");
    if (halos_out) *halos_out = nullptr;
    if (!t || !params || n < 0 || (stride != 3 && stride != 4) || !(box > 0) || (n > 0 && (!pos || !vel || !halo_id)))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_assign: bad argument");
    if (n != t->n_total) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_assign: n differs from the tree's");
    if (!(params->delta_vir > 0) || !(params->merge_thresh > 0))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_assign: delta_vir and merge_thresh must be positive");
    if (n == 0) {
        if (n_halos) *n_halos = 0;
        return halos_out ? empty_halos(halos_out) : RS_OK;
    }
    const double nbar = params->nbar > 0 ? params->nbar : (double)n / (box * box * box);
    const double rho_term = (4.0 / 3.0) * M_PI * params->delta_vir * nbar;
    const float boxf = (float)box;
    const NodeArrays &nd = t->nd;
    const int nn = (int)t->n_nodes;
    RS_LAUNCH(ctx, "as_fill", k_fill_i32v, std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->num_sms * 16), 256, 0,
              halo_id, n, -1);
    if (nn == 0) {
        if (n_halos) *n_halos = 0;
        return halos_out ? empty_halos(halos_out) : RS_OK;
    }
    // seeds
    RS_WS(ctx, unsigned, fl, WS_AS_0, 2 * (int64_t)nn + 8);
    unsigned *flag = fl, *scan = fl + nn, *tot = fl + 2 * nn;
    RS_WS(ctx, int, span, WS_AS_1, nn);
    RS_LAUNCH(ctx, "as_leafflag", k_as_leafflag, ceil_div(nn, 256), 256, 0, nd, nn, flag, span);
    RS_LAUNCH(ctx, "as_span", k_as_span, ceil_div(nn, 256), 256, 0, nd, nn, span);
    RS_CUDA(ctx, cudaMemcpyAsync(scan, flag, sizeof(unsigned) * nn, cudaMemcpyDeviceToDevice, ctx->stream));
    RS_TRY(rs_scan_u32(ctx, scan, nn, tot));
    int64_t Lh;
    {
        RS_CUDA(ctx, cudaMemcpyAsync(ctx->h_scratch, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        RS_TRY(rs_sync_check(ctx, "rs_assign"));
        Lh = (int64_t)(*(unsigned *)ctx->h_scratch);
    }
    const int L = (int)Lh;
    RS_WS(ctx, unsigned, lk, WS_AS_2, 4 * (int64_t)L + 8);
    unsigned *k0 = lk, *k1 = lk + L, *v0 = lk + 2 * L, *v1 = lk + 3 * L;
    RS_LAUNCH(ctx, "as_leafcompact", k_as_leafcompact, ceil_div(nn, 256), 256, 0, nd, nn, (const unsigned *)flag,
              (const unsigned *)scan, k0, v0);
    int bits = 0;
    while (bits < 32 && ((uint64_t)(t->n_members > 0 ? t->n_members - 1 : 0) >> bits) != 0) bits++;
    bool alt = false;
    RS_TRY(rs_radix_sort_u32(ctx, k0, k1, v0, v1, L, bits, &alt, "sort_as"));
    AsBufs A;
    A.L = L;
    A.leaf_first = alt ? k1 : k0;
    A.leaf_node = (const int *)(alt ? v1 : v0);
    A.span = span;
    size_t per = sizeof(int) * 3 + sizeof(MomAcc) + 2 * sizeof(float4) + sizeof(unsigned long long) +
                 8 * sizeof(double) + 16 * sizeof(float) + 64 * 8;
    RS_WS(ctx, char, hb, WS_AS_3, (int64_t)(per * (L + 1)) + 65536);
    char *hp = hb;
    A.uf = carve<int>(hp, L);
    A.hid = carve<int>(hp, L);
    A.hrank = carve<int>(hp, L);
    A.hacc = carve<MomAcc>(hp, L);
    A.href = carve<float4>(hp, 2 * L);
    A.hcount = carve<unsigned long long>(hp, L);
    A.hx = carve<double>(hp, 3 * L);
    A.hv = carve<double>(hp, 3 * L);
    A.hsigv = carve<double>(hp, L);
    A.hrdyn2 = carve<double>(hp, L);
    A.hfast = carve<float>(hp, 16 * (int64_t)L);
    RS_CUDA(ctx, cudaMemsetAsync(A.hacc, 0, sizeof(MomAcc) * (size_t)L, ctx->stream));
    const int64_t gl = ceil_div(L, 256);
    RS_LAUNCH(ctx, "as_init", k_as_init, gl, 256, 0, A);
    RS_LAUNCH(ctx, "as_merge", k_as_merge, gl, 256, 0, A, nd, box, params->merge_thresh, ctx->d_status);
    RS_LAUNCH(ctx, "as_roots", k_as_roots, gl, 256, 0, A, nd, (const int *)t->members, pos, vel, stride, boxf,
              ctx->d_status);
    RS_WS(ctx, int, leaf_root, WS_AS_7, L);
    RS_LAUNCH(ctx, "as_leafroot", k_as_leafroot, gl, 256, 0, A, leaf_root, ctx->d_status);
    const int64_t gblk = std::min<int64_t>(L, (int64_t)ctx->num_sms * 8);
    RS_LAUNCH(ctx, "as_hmom", k_as_hmom, gblk, AS_THREADS, 0, A, nd, (const int *)t->members, pos, vel, stride, boxf,
              ctx->d_status);
    RS_WS(ctx, unsigned, rf, WS_AS_4, 2 * (int64_t)L + 8);
    unsigned *rootflag = rf, *rscan = rf + L, *rtot = rf + 2 * L;
    RS_LAUNCH(ctx, "as_hfin", k_as_hfin, gl, 256, 0, A, box, rootflag);
    RS_CUDA(ctx, cudaMemcpyAsync(rscan, rootflag, sizeof(unsigned) * L, cudaMemcpyDeviceToDevice, ctx->stream));
    RS_TRY(rs_scan_u32(ctx, rscan, L, rtot));
    int64_t H;
    {
        RS_CUDA(ctx, cudaMemcpyAsync(ctx->h_scratch, rtot, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        RS_TRY(rs_sync_check(ctx, "rs_assign"));
        H = (int64_t)(*(unsigned *)ctx->h_scratch);
    }
    RS_WS(ctx, unsigned long long, ho, WS_AS_5, 2 * (H + 1) + 8);
    unsigned long long *hoff = ho, *hfill = ho + (H + 1);
    RS_CUDA(ctx, cudaMemsetAsync(ho, 0, sizeof(unsigned long long) * (2 * (H + 1)), ctx->stream));
    RS_LAUNCH(ctx, "as_hrank", k_as_hrank, gl, 256, 0, A, (const unsigned *)rootflag, (const unsigned *)rscan, hoff);
    RS_TRY(rs_scan_i64(ctx, (int64_t *)hoff, H + 1, nullptr));
    int64_t hm_total;
    RS_TRY(rs_read_i64(ctx, hoff + H, 1, &hm_total, "rs_assign"));
    RS_WS(ctx, int, hm, WS_AS_6, hm_total + H + 8);
    int *hmem = hm, *root_of_rank = hm + hm_total;
    RS_LAUNCH(ctx, "as_root_of_rank", k_as_root_of_rank, gl, 256, 0, A, root_of_rank);
    RS_LAUNCH(ctx, "as_hmembers", k_as_hmembers, gblk, AS_THREADS, 0, A, nd, (const unsigned long long *)hoff, hfill,
              hmem, ctx->d_status);
    RS_LAUNCH(ctx, "as_rdyn", k_as_rdyn, std::min<int64_t>(H, (int64_t)ctx->num_sms * 8), AS_THREADS, 0, A, (int)H,
              (const int *)root_of_rank, (const unsigned long long *)hoff, (const int *)hmem,
              (const int *)t->members, pos, stride, box, rho_term);
    // r_dyn of the halos too large for one block's shared memory
    RS_TRY(large_rdyn(ctx, A, (int)H, (const int *)root_of_rank, (const unsigned long long *)hoff, (const int *)hmem,
                      (const int *)t->members, pos, stride, box, rho_term));
    // assignment tiles over every node's own members (outside its children)
    RS_WS(ctx, int64_t, tl, WS_RF_MISC1, (int64_t)nn + 8);
    RS_LAUNCH(ctx, "as_tiles_prep", k_as_tiles_prep, ceil_div(nn, 256), 256, 0, nd, nn, (const int *)span, tl);
    RS_CUDA(ctx, cudaMemsetAsync(tl + nn, 0, sizeof(int64_t), ctx->stream));
    RS_TRY(rs_scan_i64(ctx, tl, nn + 1, tl + nn + 2));
    int64_t T;
    RS_TRY(rs_read_i64(ctx, tl + nn, 1, &T, "rs_assign"));
    RS_WS(ctx, int, tt, WS_RF_MISC2, 2 * T + 8);
    RS_LAUNCH(ctx, "as_tiles_fill", k_as_tiles_fill, std::min<int64_t>(nn, 65535), 128, 0, nn, (const int64_t *)tl, tt,
              tt + T);
    // distinct candidate halos of every node, once per node
    RS_WS(ctx, int64_t, cw, WS_AS_8, 2 * (int64_t)nn + 8);
    int64_t *coff = cw;
    int *node_la = (int *)(cw + nn + 4), *ncand = node_la + nn;
    RS_LAUNCH(ctx, "as_nl", k_as_nl, ceil_div(nn, 256), 256, 0, A, nd, (int)nn, node_la, coff);
    RS_CUDA(ctx, cudaMemsetAsync(coff + nn, 0, sizeof(int64_t), ctx->stream));
    RS_TRY(rs_scan_i64(ctx, coff, nn + 1, coff + nn + 2));
    int64_t CT;
    RS_TRY(rs_read_i64(ctx, coff + nn, 1, &CT, "rs_assign"));
    RS_WS(ctx, int, cand_g, WS_AS_9, CT + 8);
    RS_LAUNCH(ctx, "as_cand", k_as_cand, T, AS_THREADS, 0, A, nd, (const int *)leaf_root, (const int *)tt,
              (const int *)(tt + T), (const int *)node_la, (const int64_t *)coff, cand_g, ncand);
    RS_LAUNCH(ctx, "as_assign", k_as_assign, T, AS_THREADS, 0, A, nd, (const int *)leaf_root, (const int *)cand_g,
              (const int *)node_la, (const int64_t *)coff, (const int *)ncand, (const int *)tt, (const int *)(tt + T),
              (const int *)t->members, pos, vel, stride, box, boxf, halo_id, ctx->d_status);
    if (halos_out) {
        rs_halos *hs = new (std::nothrow) rs_halos();
        if (!hs) return RS_ERR_OOM;
        hs->n_halos = H;
        hs->n_nodes = nn;
        const size_t bytes = (size_t)(H + 1) * (4 + 48 + 8 + 8 + 4) + (size_t)(nn + 1) * 4 + 8 * 256;
        if (cudaMalloc(&hs->block, bytes) != cudaSuccess) {
            cudaGetLastError();
            delete hs;
            return rs_fail(ctx, RS_ERR_OOM, "rs_assign: halo table allocation failed");
        }
        char *b = (char *)hs->block;
        hs->id = carve<int>(b, H);
        hs->xbar = carve<double>(b, 3 * H);
        hs->vbar = carve<double>(b, 3 * H);
        hs->sigv = carve<double>(b, H);
        hs->rdyn2 = carve<double>(b, H);
        hs->root = carve<int>(b, H);
        hs->leaf_halo = carve<int>(b, nn);
        RS_LAUNCH(ctx, "as_export_fill", k_fill_i32v, ceil_div(nn, 256), 256, 0, (int32_t *)hs->leaf_halo, (int64_t)nn,
                  -1);
        if (H > 0)
            RS_LAUNCH(ctx, "as_export", k_as_export, ceil_div(H, 256), 256, 0, A, nd, (int)H,
                      (const int *)root_of_rank, *hs);
        RS_LAUNCH(ctx, "as_export_leaf", k_as_export_leaf, gl, 256, 0, A, (const int *)leaf_root, hs->leaf_halo);
        *halos_out = hs;
    }
    if (n_halos) {
        *n_halos = H;
        RS_TRY(rs_sync_check(ctx, "rs_assign"));
    }
    return RS_OK;
}

extern "C" rs_status rs_assign(rs_ctx *ctx, const rs_tree *t, const float *pos, const float *vel, int32_t stride,
                               int64_t n, double box, const rs_params *params, int32_t *halo_id, int64_t *n_halos)
{
    return rs_assign_ex(ctx, t, pos, vel, stride, n, box, params, halo_id, n_halos, nullptr);
}

extern "C" void rs_halos_free(rs_halos *h)
{
    if (!h) return;
    if (h->block) cudaFree(h->block);
    delete h;
}

extern "C" int64_t rs_halos_count(const rs_halos *h) { return h ? h->n_halos : 0; }

extern "C" rs_status rs_halos_export(rs_ctx *ctx, const rs_halos *h, int32_t *id, double *xbar, double *vbar,
                                     double *sigv, double *rdyn2)
{
    if (!ctx || !h) return RS_ERR_INVALID_ARG;
    const size_t H = (size_t)h->n_halos;
    if (H == 0) return RS_OK;
    if (id) RS_CUDA(ctx, cudaMemcpyAsync(id, h->id, 4 * H, cudaMemcpyDeviceToDevice, ctx->stream));
    if (xbar) RS_CUDA(ctx, cudaMemcpyAsync(xbar, h->xbar, 24 * H, cudaMemcpyDeviceToDevice, ctx->stream));
    if (vbar) RS_CUDA(ctx, cudaMemcpyAsync(vbar, h->vbar, 24 * H, cudaMemcpyDeviceToDevice, ctx->stream));
    if (sigv) RS_CUDA(ctx, cudaMemcpyAsync(sigv, h->sigv, 8 * H, cudaMemcpyDeviceToDevice, ctx->stream));
    if (rdyn2) RS_CUDA(ctx, cudaMemcpyAsync(rdyn2, h->rdyn2, 8 * H, cudaMemcpyDeviceToDevice, ctx->stream));
    return RS_OK;
}

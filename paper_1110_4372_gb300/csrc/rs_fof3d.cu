// rs_fof3d.cu -- periodic 3D friends-of-friends (Sec. 3.1) and the group CSR.
//
// Particles are binned into fine cells of side s <= l / sqrt(3) (with a
// margin that covers the float32 rounding of the cell index), so any two
// particles of one fine cell are friends and a fine cell can stand for all
// of its particles in the union-find.  Fine cells are grouped 4 x 4 x 4 into
// coarse cells; particles are radix-sorted by (coarse cell, fine sub-cell),
// a dense table maps each coarse cell to its first fine cell, and a 64-bit
// mask stored at that first fine cell tells which of the 64 sub-cells are
// occupied.  Every friend of a particle lies within two fine cells per axis,
// which is inside at most 2 x 2 x 2 coarse cells; the fine cells within
// reach of a fine cell follow from the masks by bit operations, and their
// indices by a popcount, with no scan.  Two fine cells are joined as soon as
// one pair between them is within l; pairs already in one set are skipped.
//
// Distances: float32 with the periodic shift applied to the coordinate near
// the top of the box (x - box is exact there), compared against l^2 (1 -+
// 2^-20); pairs inside that band are re-tested in float64 with the same
// separate multiplies and adds as the definition, so the partition is the
// float64 one.
#include <cmath>
#include <utility>

#include "rs_internal.cuh"

namespace {

constexpr int FOF_THREADS = 256;
constexpr double BAND_REL = 9.5367431640625e-07;  // 2^-20, relative on d^2

struct FofGeom {
    int32_t Gc;      // coarse cells per side
    int32_t Gf;      // fine cells per side (4 Gc)
    float inv_sf;    // Gf / box (float32)
    float boxf;
    double box;
    double l, l2;
    float lo32, hi32;  // float32 thresholds on d^2 around l^2
};

__device__ __forceinline__ void load_pos(const float *pos, int stride, int64_t i, float &x, float &y, float &z)
{
    const float *p = pos + (int64_t)stride * i;
    x = p[0];
    y = p[1];
    z = p[2];
}

__device__ __forceinline__ int fine_coord(float x, float inv, int Gf)
{
    int f = (int)floorf(x * inv);
    f = f < 0 ? 0 : f;
    f = f >= Gf ? Gf - 1 : f;
    return f;
}

__global__ void k_fof_keys(const float *pos, int stride, int64_t n, FofGeom g, uint64_t *keys, uint32_t *vals,
                           rs_dev_status *st)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x, y, z;
    load_pos(pos, stride, i, x, y, z);
    if (!(x >= 0.f && x < g.boxf && y >= 0.f && y < g.boxf && z >= 0.f && z < g.boxf))
        dev_fail(st, DEV_BADARG, 10, i);
    int fx = fine_coord(x, g.inv_sf, g.Gf), fy = fine_coord(y, g.inv_sf, g.Gf), fz = fine_coord(z, g.inv_sf, g.Gf);
    uint64_t c = ((uint64_t)(fz >> 2) * (uint64_t)g.Gc + (uint64_t)(fy >> 2)) * (uint64_t)g.Gc + (uint64_t)(fx >> 2);
    uint32_t sub = (uint32_t)(((fz & 3) << 4) | ((fy & 3) << 2) | (fx & 3));
    keys[i] = (c << 6) | sub;
    vals[i] = (uint32_t)i;
}

// sorted positions as float4 and cell-start flags
__global__ void k_fof_gather(const float *pos, int stride, int64_t n, const uint64_t *keys, const uint32_t *idx,
                             float4 *spos, uint32_t *flag)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    float x, y, z;
    load_pos(pos, stride, idx[q], x, y, z);
    spos[q] = make_float4(x, y, z, 0.f);
    flag[q] = (q == 0 || keys[q] != keys[q - 1]) ? 1u : 0u;
}

// after an exclusive scan of flag: cell_of[q] = scan[q] + flag[q] - 1
__global__ void k_fof_cells(int64_t n, const uint64_t *keys, const uint32_t *scan, const uint32_t *flag,
                            uint32_t *cell_of, uint32_t *cell_start, uint64_t *cell_key, uint32_t *table,
                            const uint32_t *n_cells)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    uint32_t c = scan[q] + flag[q] - 1u;
    cell_of[q] = c;
    if (flag[q]) {
        cell_start[c] = (uint32_t)q;
        cell_key[c] = keys[q];
        uint64_t coarse = keys[q] >> 6;
        if (q == 0 || (keys[q - 1] >> 6) != coarse) table[coarse] = c;
    }
    if (q == n - 1) cell_start[*n_cells] = (uint32_t)n;
}

// occupancy mask of each coarse cell, kept at its first fine cell
__global__ void k_fof_occ(const uint32_t *n_cells_p, const uint64_t *cell_key, const uint32_t *table, uint64_t *occ)
{
    const int64_t M = *n_cells_p;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = cell_key[c];
        atomicOr((unsigned long long *)&occ[table[k >> 6]], 1ull << (k & 63));
    }
}

__global__ void k_fill_u32(uint32_t *p, int64_t n, uint32_t v)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) p[i] = v;
}

__global__ void k_iota_i32(int *p, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int)i;
}

// sub-cells (4 per axis, bit (z << 4) | (y << 2) | x) of the coarse cell at
// coarse offset d (per axis) whose fine offset from sub-cell u of the query's
// coarse cell is at most R on every axis
__device__ __forceinline__ unsigned axis_range(int u, int d, int R)
{
    const int lo = max(u - R - 4 * d, 0), hi = min(u + R - 4 * d, 3);
    return lo > hi ? 0u : ((2u << hi) - 1u) & ~((1u << lo) - 1u);
}

__device__ __forceinline__ uint64_t reach_mask(int ux, int uy, int uz, int dx, int dy, int dz, int R)
{
    const unsigned mx = axis_range(ux, dx, R), my = axis_range(uy, dy, R), mz = axis_range(uz, dz, R);
    unsigned m16 = 0;
    for (int y = 0; y < 4; y++)
        if ((my >> y) & 1u) m16 |= mx << (4 * y);
    uint64_t m = 0;
    for (int z = 0; z < 4; z++)
        if ((mz >> z) & 1u) m |= (uint64_t)m16 << (16 * z);
    return m;
}

__device__ __forceinline__ void coarse_coords(uint64_t c, int Gc, int &cx, int &cy, int &cz)
{
    const uint32_t cc = (uint32_t)c, G = (uint32_t)Gc;  // fewer than 2^32 coarse cells
    const uint32_t r = cc / G;
    cx = (int)(cc - r * G);
    cz = (int)(r / G);
    cy = (int)(r - (uint32_t)cz * G);
}

// wrapped fine-cell offset b - a in [-Gf/2, Gf/2); shift tells which point
// sits on the far side of the periodic face (+1: b near the top, -1: a)
__device__ __forceinline__ int fine_offset(int a, int b, int Gf, int &shift)
{
    int d = b - a;
    shift = 0;
    if (d > Gf / 2) {
        d -= Gf;
        shift = 1;
    } else if (d < -(Gf / 2)) {
        d += Gf;
        shift = -1;
    }
    return d;
}

__device__ __forceinline__ float sdiff(float a, float b, int shift, float box)
{
    // b - a with the periodic image chosen by shift; x - box is exact for x >= box/2
    if (shift > 0) return (b - box) - a;
    if (shift < 0) return b - (a - box);
    return b - a;
}

__device__ __forceinline__ double ddiff(float a, float b, int shift, double box)
{
    if (shift > 0) return f64_sub(f64_sub((double)b, box), (double)a);
    if (shift < 0) return f64_sub((double)b, f64_sub((double)a, box));
    return f64_sub((double)b, (double)a);
}

// 0 = not friends, 1 = friends
__device__ __forceinline__ int pair_link(const float4 &pa, const float4 &pb, int sx, int sy, int sz,
                                         const FofGeom &g)
{
    float dx = sdiff(pa.x, pb.x, sx, g.boxf), dy = sdiff(pa.y, pb.y, sy, g.boxf), dz = sdiff(pa.z, pb.z, sz, g.boxf);
    float d2 = dx * dx + dy * dy + dz * dz;
    if (d2 <= g.lo32) return 1;
    if (d2 > g.hi32) return 0;
    double ex = ddiff(pa.x, pb.x, sx, g.box), ey = ddiff(pa.y, pb.y, sy, g.box), ez = ddiff(pa.z, pb.z, sz, g.box);
    double e2 = f64_add(f64_add(f64_mul(ex, ex), f64_mul(ey, ey)), f64_mul(ez, ez));
    return e2 <= g.l2 ? 1 : 0;
}

// position of the j-th (0-based) set bit of a 64-bit mask with at least j + 1 bits
__device__ __forceinline__ int nth_bit64(uint64_t m, int j)
{
    const unsigned lo = (unsigned)m, hi = (unsigned)(m >> 32);
    const int nlo = __popc(lo);
    return j < nlo ? (int)__fns(lo, 0, j + 1) : 32 + (int)__fns(hi, 0, j - nlo + 1);
}

// Join fine cell A with every fine cell of larger index within two fine cells
// per axis that has a friend pair with it.  Pass 0 takes the 26 adjacent
// cells (offsets of at most 1 per axis), where pairs are friends almost at
// once in dense regions; pass 1 takes the cells two apart on some axis, by
// which time dense regions are mostly one set: a coarse cell whose fine cells
// all had one root after pass 0 (uroot at its first fine cell, else -1) is
// skipped whole when that root is A's, and the same-set check skips the
// rest.  Coarse cells numbered below A's hold only fine cells of smaller
// index and are not visited.
//
// A warp takes 32 consecutive fine cells, a lane each.  For each of the
// eight coarse cells around them every lane forms its mask of candidate fine
// cells; the warp then numbers all lanes' candidates (a prefix sum of the
// mask popcounts) and deals them out 32 at a time, so each lane tests one
// candidate pair per round whatever the spread of candidates over the cells.
__global__ void __launch_bounds__(FOF_THREADS, 6) k_fof_link(const uint32_t *n_cells_p, const uint64_t *cell_key,
                                                            const uint32_t *cell_start, const uint32_t *table,
                                                            const uint64_t *occ, const float4 *spos, int *parent,
                                                            const int *uroot, FofGeom g, int pass, rs_dev_status *st)
{
    const unsigned FULL = 0xffffffffu;
    const int64_t M = *n_cells_p;
    const int lane = lane_id();
    const int64_t wfirst = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31));
    for (int64_t wb = wfirst; wb < M; wb += (int64_t)gridDim.x * blockDim.x) {
        const int64_t A = wb + lane;
        const bool va = A < M;
        uint64_t ca = 0;
        int sa = 0, ux = 0, uy = 0, uz = 0, ccx = 0, ccy = 0, ccz = 0;
        uint32_t a0 = 0, a1 = 0;
        if (va) {
            const uint64_t ka = cell_key[A];
            ca = ka >> 6;
            sa = (int)(ka & 63);
            ux = sa & 3;
            uy = (sa >> 2) & 3;
            uz = sa >> 4;
            coarse_coords(ca, g.Gc, ccx, ccy, ccz);
            a0 = cell_start[A];
            a1 = cell_start[A + 1];
        }
        const int ax = 4 * ccx + ux, ay = 4 * ccy + uy, az = 4 * ccz + uz;
        const int lox = ux < 2 ? -1 : 0, loy = uy < 2 ? -1 : 0, loz = uz < 2 ? -1 : 0;
        // a root of A's set (sets only grow, so a coarse cell whose common
        // root equals it is in A's set for the rest of the pass)
        const int ra = (va && uroot) ? uf_find(parent, (int)A, st) : -1;
        for (int s8 = 0; s8 < 8; s8++) {
            const int dz = loz + (s8 >> 2), dy = loy + ((s8 >> 1) & 1), dx = lox + (s8 & 1);
            int cz = ccz + dz, cy = ccy + dy, cx = ccx + dx;
            cz = cz < 0 ? cz + g.Gc : (cz >= g.Gc ? cz - g.Gc : cz);
            cy = cy < 0 ? cy + g.Gc : (cy >= g.Gc ? cy - g.Gc : cy);
            cx = cx < 0 ? cx + g.Gc : (cx >= g.Gc ? cx - g.Gc : cx);
            uint64_t cand = 0, om = 0;
            uint32_t b0c = 0;
            if (va) {
                const uint64_t cc = ((uint64_t)cz * g.Gc + cy) * g.Gc + cx;
                if (cc >= ca) {  // coarse cells below A's hold only fine cells of smaller index
                    b0c = table[cc];
                    if (b0c != 0xffffffffu && !(ra >= 0 && uroot[b0c] == ra)) {
                        om = occ[b0c];
                        const uint64_t near = reach_mask(ux, uy, uz, dx, dy, dz, 1);
                        cand = om & (pass == 0 ? near : reach_mask(ux, uy, uz, dx, dy, dz, 2) & ~near);
                        if (cc == ca) cand &= ~((2ull << sa) - 1ull);  // sub-cells after A's
                    }
                }
            }
            for (int guard = 0; guard < 4096; guard++) {
                const int cnt = __popcll(cand);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                const int total = __shfl_sync(FULL, incl, 31);
                if (total == 0) break;
                const int excl = incl - cnt;
                // this lane's candidate: number `lane` in the warp's order
                int lo = 0, hi = 31;
#pragma unroll
                for (int it = 0; it < 5; it++) {
                    const int mid = (lo + hi) >> 1;
                    if (__shfl_sync(FULL, incl, mid) > lane) hi = mid;
                    else lo = mid + 1;
                }
                const int src = lo;
                const int j = lane - __shfl_sync(FULL, excl, src);
                const uint64_t smask = __shfl_sync(FULL, cand, src), som = __shfl_sync(FULL, om, src);
                const uint32_t sb0 = __shfl_sync(FULL, b0c, src), sa0 = __shfl_sync(FULL, a0, src),
                               sa1 = __shfl_sync(FULL, a1, src);
                const int sax = __shfl_sync(FULL, ax, src), say = __shfl_sync(FULL, ay, src),
                          saz = __shfl_sync(FULL, az, src);
                const int scx = __shfl_sync(FULL, cx, src), scy = __shfl_sync(FULL, cy, src),
                          scz = __shfl_sync(FULL, cz, src);
                const int sA = (int)(wb + src);
                if (lane < total) {
                    const int sb = nth_bit64(smask, j);
                    const int B = (int)(sb0 + __popcll(som & ((1ull << sb) - 1ull)));
                    const int bx = 4 * scx + (sb & 3), by = 4 * scy + ((sb >> 2) & 3), bz = 4 * scz + (sb >> 4);
                    int sx, sy, sz;
                    fine_offset(sax, bx, g.Gf, sx);
                    fine_offset(say, by, g.Gf, sy);
                    fine_offset(saz, bz, g.Gf, sz);
                    if (uf_find(parent, sA, st) != uf_find(parent, B, st)) {
                        const uint32_t b0 = cell_start[B], b1 = cell_start[B + 1];
                        bool linked = false;
                        for (uint32_t i = sa0; i < sa1 && !linked; i++) {
                            const float4 pa = spos[i];
                            for (uint32_t q = b0; q < b1; q++)
                                if (pair_link(pa, spos[q], sx, sy, sz, g)) {
                                    linked = true;
                                    break;
                                }
                        }
                        if (linked) uf_union(parent, sA, B, st);
                    }
                }
                // drop the candidates dealt out this round (the lowest ones of each lane)
                const int used = max(0, min(incl, 32) - excl);
                for (int u = 0; u < used; u++) cand &= cand - 1ull;
            }
        }
    }
}

// the root of every coarse cell's first fine cell, kept at that cell
__global__ void k_fof_uroot_first(const uint32_t *n_cells_p, const uint64_t *cell_key, const uint32_t *table,
                                  int *parent, int *uroot, rs_dev_status *st)
{
    const int64_t M = *n_cells_p;
    for (int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; A < M; A += (int64_t)gridDim.x * blockDim.x)
        if (table[cell_key[A] >> 6] == (uint32_t)A) uroot[A] = uf_find(parent, (int)A, st);
}

// -1 at the first fine cell of every coarse cell whose fine cells do not all
// share that root (no unions run meanwhile, so roots are fixed)
__global__ void k_fof_uroot_check(const uint32_t *n_cells_p, const uint64_t *cell_key, const uint32_t *table,
                                  int *parent, int *uroot, rs_dev_status *st)
{
    const int64_t M = *n_cells_p;
    for (int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; A < M; A += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b0 = table[cell_key[A] >> 6];
        if (b0 != (uint32_t)A && uf_find(parent, (int)A, st) != uroot[b0]) uroot[b0] = -1;
    }
}

// (find_limit bounds each find; it is RS_SPIN_LIMIT except under the
// injected fault RS_FAULT=timeout1, where it is 1)
__global__ void k_fof_rootmin(const uint32_t *n_cells_p, const uint32_t *cell_start, const uint32_t *idx,
                              int *parent, int *root_min, int find_limit, rs_dev_status *st)
{
    const int64_t M = *n_cells_p;
    for (int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; A < M; A += (int64_t)gridDim.x * blockDim.x) {
        uint32_t m = 0xffffffffu;
        for (uint32_t q = cell_start[A]; q < cell_start[A + 1]; q++) m = min(m, idx[q]);
        int r = uf_find_n(parent, (int)A, st, find_limit);
        atomicMin(&root_min[r], (int)m);
    }
}

__global__ void k_fof_labels(int64_t n, const uint32_t *idx, const uint32_t *cell_of, int *parent,
                             const int *root_min, int32_t *labels, rs_dev_status *st)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    labels[idx[q]] = root_min[uf_find(parent, (int)cell_of[q], st)];
}

__global__ void k_fof_count_roots(const uint32_t *n_cells_p, const int *parent, unsigned long long *count)
{
    const int64_t M = *n_cells_p;
    unsigned long long c = 0;
    for (int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; A < M; A += (int64_t)gridDim.x * blockDim.x)
        c += parent[A] == (int)A ? 1ull : 0ull;
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(count, c);
}

// Tie-band census: every pair (i < j in sorted order) within the fine-cell
// reach whose float64 distance satisfies |d - l| <= 1e-6 l.
__global__ void __launch_bounds__(FOF_THREADS) k_fof_tieband(const uint32_t *n_cells_p, const uint64_t *cell_key,
                                                               const uint32_t *cell_start, const uint32_t *table,
                                                               const uint64_t *occ, const float4 *spos, FofGeom g,
                                                               unsigned long long *count)
{
    const int64_t M = *n_cells_p;
    const float flo = (float)(g.l2 * (1.0 - 4e-6)), fhi = (float)(g.l2 * (1.0 + 4e-6));
    unsigned long long c = 0;
    for (int64_t A = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; A < M; A += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ka = cell_key[A], ca = ka >> 6;
        const int sa = (int)(ka & 63), ux = sa & 3, uy = (sa >> 2) & 3, uz = sa >> 4;
        int ccx, ccy, ccz;
        coarse_coords(ca, g.Gc, ccx, ccy, ccz);
        const int ax = 4 * ccx + ux, ay = 4 * ccy + uy, az = 4 * ccz + uz;
        const uint32_t a0 = cell_start[A], a1 = cell_start[A + 1];
        const int lox = ux < 2 ? -1 : 0, loy = uy < 2 ? -1 : 0, loz = uz < 2 ? -1 : 0;
        for (int dz = loz; dz <= loz + 1; dz++)
            for (int dy = loy; dy <= loy + 1; dy++)
                for (int dx = lox; dx <= lox + 1; dx++) {
                    int cx = ccx + dx, cy = ccy + dy, cz = ccz + dz;
                    cx = cx < 0 ? cx + g.Gc : (cx >= g.Gc ? cx - g.Gc : cx);
                    cy = cy < 0 ? cy + g.Gc : (cy >= g.Gc ? cy - g.Gc : cy);
                    cz = cz < 0 ? cz + g.Gc : (cz >= g.Gc ? cz - g.Gc : cz);
                    const uint64_t cc = ((uint64_t)cz * g.Gc + cy) * g.Gc + cx;
                    if (cc < ca) continue;
                    const uint32_t b0c = table[cc];
                    if (b0c == 0xffffffffu) continue;
                    const uint64_t om = occ[b0c];
                    uint64_t cand = om & reach_mask(ux, uy, uz, dx, dy, dz, 2);
                    if (cc == ca) cand &= ~((1ull << sa) - 1ull);  // A itself and the sub-cells after it
                    while (cand) {
                        const int sb = __ffsll((long long)cand) - 1;
                        cand &= cand - 1ull;
                        const int64_t B = (int64_t)b0c + __popcll(om & ((1ull << sb) - 1ull));
                        const int bx = 4 * cx + (sb & 3), by = 4 * cy + ((sb >> 2) & 3), bz = 4 * cz + (sb >> 4);
                        int sx, sy, sz;
                        fine_offset(ax, bx, g.Gf, sx);
                        fine_offset(ay, by, g.Gf, sy);
                        fine_offset(az, bz, g.Gf, sz);
                        for (uint32_t i = a0; i < a1; i++) {
                            const float4 pa = spos[i];
                            for (uint32_t j = (B == A ? i + 1 : cell_start[B]); j < cell_start[B + 1]; j++) {
                                const float4 pb = spos[j];
                                float ddx = sdiff(pa.x, pb.x, sx, g.boxf), ddy = sdiff(pa.y, pb.y, sy, g.boxf),
                                      ddz = sdiff(pa.z, pb.z, sz, g.boxf);
                                float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
                                if (d2 < flo || d2 > fhi) continue;
                                double ex = ddiff(pa.x, pb.x, sx, g.box), ey = ddiff(pa.y, pb.y, sy, g.box),
                                       ez = ddiff(pa.z, pb.z, sz, g.box);
                                double d = sqrt(f64_add(f64_add(f64_mul(ex, ex), f64_mul(ey, ey)), f64_mul(ez, ez)));
                                if (fabs(d - g.l) <= 1e-6 * g.l) c++;
                            }
                        }
                    }
                }
    }
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(count, c);
}

// ---- accelerated variant (Sec. 3.1) ----
// The paper's faster FOF visits particles one by one: a particle with more
// than dense_n neighbours within l joins every particle within 2l, and its
// neighbours skip their own search.  Taking the visit order to be the
// particle index, the groups have a closed form that needs no order: call a
// dense particle a centre when no centre of smaller index lies within l (the
// index-greedy maximal independent set of the dense particles); the groups
// are the components of the plain FOF graph plus an edge from every centre
// to every particle within 2l of it (a skipped particle lies within l of a
// centre, so its own FOF edges end within 2l of that centre).  So the plain
// FOF runs first, then: neighbour counts up to dense_n + 1; rounds that
// decide the centres (a dense particle becomes a centre once every dense
// neighbour of smaller index is decided and none is a centre, and drops out
// once one is a centre); and the 2l joins of the centres' fine cells.
enum : uint8_t { ACC_SPARSE = 0, ACC_UNDECIDED = 1, ACC_CENTRE = 2, ACC_OUT = 3 };

// Calls f(B, b0, b1, sx, sy, sz) for every occupied fine cell B within R fine
// cells per axis of the fine cell at fine coordinates (ax, ay, az) (coarse
// cell (ccx, ccy, ccz), sub-cell (ux, uy, uz)), with B's particle range and
// the periodic shifts; stops when f returns true.  Visits the 27 coarse
// cells around the query's, which hold every fine cell within R <= 4.
template <typename F>
__device__ __forceinline__ void acc_cells(int ccx, int ccy, int ccz, int ux, int uy, int uz, int R,
                                          const uint32_t *cell_start, const uint32_t *table, const uint64_t *occ,
                                          const FofGeom &g, F f)
{
    const int ax = 4 * ccx + ux, ay = 4 * ccy + uy, az = 4 * ccz + uz;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                uint64_t cand = reach_mask(ux, uy, uz, dx, dy, dz, R);
                if (!cand) continue;
                int cx = ccx + dx, cy = ccy + dy, cz = ccz + dz;
                cx = cx < 0 ? cx + g.Gc : (cx >= g.Gc ? cx - g.Gc : cx);
                cy = cy < 0 ? cy + g.Gc : (cy >= g.Gc ? cy - g.Gc : cy);
                cz = cz < 0 ? cz + g.Gc : (cz >= g.Gc ? cz - g.Gc : cz);
                const uint64_t cc = ((uint64_t)cz * g.Gc + cy) * g.Gc + cx;
                const uint32_t b0c = table[cc];
                if (b0c == 0xffffffffu) continue;
                const uint64_t om = occ[b0c];
                cand &= om;
                while (cand) {
                    const int sb = __ffsll((long long)cand) - 1;
                    cand &= cand - 1ull;
                    const uint32_t B = b0c + (uint32_t)__popcll(om & ((1ull << sb) - 1ull));
                    const int bx = 4 * cx + (sb & 3), by = 4 * cy + ((sb >> 2) & 3), bz = 4 * cz + (sb >> 4);
                    int sx, sy, sz;
                    fine_offset(ax, bx, g.Gf, sx);
                    fine_offset(ay, by, g.Gf, sy);
                    fine_offset(az, bz, g.Gf, sz);
                    if (f(B, cell_start[B], cell_start[B + 1], sx, sy, sz)) return;
                }
            }
}

__device__ __forceinline__ void acc_where(const uint64_t *cell_key, uint32_t A, const FofGeom &g, int &ccx, int &ccy,
                                          int &ccz, int &ux, int &uy, int &uz)
{
    const uint64_t k = cell_key[A];
    const int sa = (int)(k & 63);
    ux = sa & 3;
    uy = (sa >> 2) & 3;
    uz = sa >> 4;
    coarse_coords(k >> 6, g.Gc, ccx, ccy, ccz);
}

// dense flag of every particle (sorted slot q): more than dense_n others
// within l.  The own fine cell is a clique; other cells are tested pair by
// pair until the count is exceeded.
__global__ void __launch_bounds__(FOF_THREADS) k_acc_count(int64_t n, const uint32_t *cell_of, const uint64_t *cell_key,
                                                           const uint32_t *cell_start, const uint32_t *table,
                                                           const uint64_t *occ, const float4 *spos, FofGeom g,
                                                           int dense_n, uint8_t *state)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint32_t A = cell_of[q];
    int cnt = (int)(cell_start[A + 1] - cell_start[A]) - 1;
    if (cnt <= dense_n) {
        int ccx, ccy, ccz, ux, uy, uz;
        acc_where(cell_key, A, g, ccx, ccy, ccz, ux, uy, uz);
        const float4 p = spos[q];
        acc_cells(ccx, ccy, ccz, ux, uy, uz, 2, cell_start, table, occ, g,
                  [&](uint32_t B, uint32_t b0, uint32_t b1, int sx, int sy, int sz) {
                      if (B == A) return false;
                      for (uint32_t r = b0; r < b1; r++)
                          if (pair_link(p, spos[r], sx, sy, sz, g) && ++cnt > dense_n) return true;
                      return false;
                  });
    }
    state[q] = cnt > dense_n ? ACC_UNDECIDED : ACC_SPARSE;
}

// one round of the centre choice; `left` counts the particles still undecided
__global__ void __launch_bounds__(FOF_THREADS) k_acc_round(int64_t n, const uint32_t *cell_of, const uint64_t *cell_key,
                                                           const uint32_t *cell_start, const uint32_t *table,
                                                           const uint64_t *occ, const float4 *spos, const uint32_t *idx,
                                                           FofGeom g, const uint8_t *sin, uint8_t *sout,
                                                           unsigned long long *left)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint8_t s0 = sin[q];
    if (s0 != ACC_UNDECIDED) {
        sout[q] = s0;
        return;
    }
    const uint32_t A = cell_of[q], me = idx[q];
    int ccx, ccy, ccz, ux, uy, uz;
    acc_where(cell_key, A, g, ccx, ccy, ccz, ux, uy, uz);
    const float4 p = spos[q];
    bool blocked = false, out = false;
    acc_cells(ccx, ccy, ccz, ux, uy, uz, 2, cell_start, table, occ, g,
              [&](uint32_t B, uint32_t b0, uint32_t b1, int sx, int sy, int sz) {
                  for (uint32_t r = b0; r < b1; r++) {
                      const uint8_t sr = sin[r];
                      if ((sr != ACC_UNDECIDED && sr != ACC_CENTRE) || idx[r] >= me) continue;
                      // the own fine cell is a clique
                      if (B != A && !pair_link(p, spos[r], sx, sy, sz, g)) continue;
                      if (sr == ACC_CENTRE) {
                          out = true;
                          return true;
                      }
                      blocked = true;
                  }
                  return false;
              });
    const uint8_t s1 = out ? ACC_OUT : (blocked ? ACC_UNDECIDED : ACC_CENTRE);
    sout[q] = s1;
    if (s1 == ACC_UNDECIDED) atomicAdd(left, 1ull);
}

// every centre joins the fine cells that hold a particle within 2l of it
// (a fine cell is one set already, so one such particle joins it); g2 is the
// geometry with the thresholds of 2l
__global__ void __launch_bounds__(FOF_THREADS) k_acc_join(int64_t n, const uint32_t *cell_of, const uint64_t *cell_key,
                                                          const uint32_t *cell_start, const uint32_t *table,
                                                          const uint64_t *occ, const float4 *spos, FofGeom g2,
                                                          const uint8_t *state, int *parent,
                                                          unsigned long long *centres, rs_dev_status *st)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool mine = q < n && state[q] == ACC_CENTRE;
    const unsigned m = __ballot_sync(0xffffffffu, mine);
    if (lane_id() == 0 && m) atomicAdd(centres, (unsigned long long)__popc(m));
    if (!mine) return;
    const uint32_t A = cell_of[q];
    int ccx, ccy, ccz, ux, uy, uz;
    acc_where(cell_key, A, g2, ccx, ccy, ccz, ux, uy, uz);
    const float4 p = spos[q];
    acc_cells(ccx, ccy, ccz, ux, uy, uz, 4, cell_start, table, occ, g2,
              [&](uint32_t B, uint32_t b0, uint32_t b1, int sx, int sy, int sz) {
                  if (uf_find(parent, (int)A, st) == uf_find(parent, (int)B, st)) return false;
                  for (uint32_t r = b0; r < b1; r++)
                      if (pair_link(p, spos[r], sx, sy, sz, g2)) {
                          uf_union(parent, (int)A, (int)B, st);
                          break;
                      }
                  return false;
              });
}

rs_status fof_geometry(rs_ctx *ctx, int64_t n, double box, double b, FofGeom *g)
{
    // fine side s with sqrt(3) s (1 + 2 err) < l, err = float32 error of the
    // fine-cell coordinate in cell units (2.0001 u Gf)
    const FofGridSize gs = fof_grid_size(n, box, b);
    const double l = gs.l, gf_est = gs.gf_est, err = gs.err, gc = gs.gc;
    if (!(l > 0)) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_fof3d: linking length must be positive");
    if (gc < 3) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_fof3d: box narrower than about seven linking lengths");
    if (gc * gc * gc >= 4294967295.0) return rs_fail(ctx, RS_ERR_TOO_LARGE, "rs_fof3d: more than 2^32 coarse cells");
    g->Gc = (int32_t)gc;
    g->Gf = 4 * g->Gc;
    if (g->Gf > gf_est) return rs_fail(ctx, RS_ERR_INTERNAL, "rs_fof3d: grid estimate");
    // the link kernels look two fine cells per axis around a cell: two
    // friends' fine indices differ by less than 1 + l/s + 2 err, so l/s must
    // not exceed 2 - 2 err.  With s rounded down to box / (4 Gc) this fails
    // only in narrow windows of box/l below 14 (e.g. 6.9-8, 11.55-12).
    if (l * (double)g->Gf / box > 2.0 - 2.0 * err)
        return rs_fail(ctx, RS_ERR_INVALID_ARG,
                       "rs_fof3d: no cell grid fits this box and linking length (cells of side between l/2 and "
                       "l/sqrt(3) that divide the box 4k times); use a box of at least 14 linking lengths");
    g->inv_sf = (float)((double)g->Gf / box);
    g->boxf = (float)box;
    g->box = box;
    g->l = l;
    g->l2 = l * l;
    g->lo32 = (float)(g->l2 * (1.0 - BAND_REL));
    g->hi32 = (float)(g->l2 * (1.0 + BAND_REL));
    if ((double)g->boxf != box) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_fof3d: box must be a float32 value");
    return RS_OK;
}

int key_bits(const FofGeom &g)
{
    uint64_t maxkey = (((uint64_t)g.Gc * g.Gc * g.Gc) << 6);
    int bits = 0;
    while (bits < 64 && (maxkey >> bits) != 0) bits++;
    return bits;
}

}  // namespace

namespace {

constexpr int ACC_MAX_ROUNDS = 1 << 16;  // bound on the centre-choice rounds

// plain FOF (dense_n < 0) or the accelerated variant (dense_n >= 0)
rs_status fof_run(rs_ctx *ctx, const float *pos, int32_t stride, int64_t n, double box, double b, int32_t dense_n,
                  int32_t *labels, int64_t *n_groups, int64_t *n_tieband, int64_t *n_centres)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!pos || !labels)) || (stride != 3 && stride != 4) || !(box > 0) || !(b > 0))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_fof3d: bad argument");
    if (n >= ((int64_t)1 << 31)) return rs_fail(ctx, RS_ERR_TOO_LARGE, "rs_fof3d: n >= 2^31");
    if (n == 0) {
        if (n_groups) *n_groups = 0;
        if (n_tieband) *n_tieband = 0;
        if (n_centres) *n_centres = 0;
        return RS_OK;
    }
    RsStageGuard running(&ctx->in_fof);
    RsRange range(dense_n >= 0 ? "rs_fof3d_accel" : "rs_fof3d");
    FofGeom g;
    RS_TRY(fof_geometry(ctx, n, box, b, &g));
    const int64_t T = FOF_THREADS;
    const int64_t nb = ceil_div(n, T);
    const int64_t ncoarse = (int64_t)g.Gc * g.Gc * g.Gc;

    RS_WS(ctx, uint64_t, k0, WS_SORT_K0, n);
    RS_WS(ctx, uint64_t, k1, WS_SORT_K1, n);
    RS_WS(ctx, uint32_t, v0, WS_SORT_V0, n);
    RS_WS(ctx, uint32_t, v1, WS_SORT_V1, n);
    RS_LAUNCH(ctx, "fof_keys", k_fof_keys, nb, T, 0, pos, stride, n, g, k0, v0, ctx->d_status);
    bool alt = false;
    RS_TRY(rs_radix_sort_u64(ctx, k0, k1, v0, v1, n, key_bits(g), &alt, "sort_fof"));
    uint64_t *keys = alt ? k1 : k0;
    uint32_t *idx = alt ? v1 : v0;

    RS_WS(ctx, float4, spos, WS_FOF_POS4, n);
    RS_WS(ctx, uint32_t, flag, WS_FOF_MISC, 2 * n + 8);
    uint32_t *scan = flag + n;
    uint32_t *n_cells = flag + 2 * n;  // device scalar
    RS_LAUNCH(ctx, "fof_gather", k_fof_gather, nb, T, 0, pos, stride, n, (const uint64_t *)keys,
              (const uint32_t *)idx, spos, flag);
    RS_CUDA(ctx, cudaMemcpyAsync(scan, flag, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    RS_TRY(rs_scan_u32(ctx, scan, n, n_cells));

    RS_WS(ctx, uint32_t, cell_of, WS_FOF_CELLOF, n);
    RS_WS(ctx, uint32_t, cell_start, WS_FOF_CELLSTART, n + 1);
    RS_WS(ctx, uint64_t, cell_key, WS_FOF_CELLKEY, n);
    RS_WS(ctx, uint32_t, table, WS_FOF_TABLE, ncoarse);
    int fill_blocks = (int)std::min<int64_t>(ceil_div(ncoarse, T), (int64_t)ctx->num_sms * 16);
    RS_LAUNCH(ctx, "fof_table_clear", k_fill_u32, fill_blocks, T, 0, table, ncoarse, 0xffffffffu);
    RS_LAUNCH(ctx, "fof_cells", k_fof_cells, nb, T, 0, n, (const uint64_t *)keys, (const uint32_t *)scan,
              (const uint32_t *)flag, cell_of, cell_start, cell_key, table, (const uint32_t *)n_cells);
    RS_WS(ctx, uint64_t, occ, WS_FOF_OCC, n);
    RS_CUDA(ctx, cudaMemsetAsync(occ, 0, sizeof(uint64_t) * n, ctx->stream));
    const int64_t grid = std::min<int64_t>(nb, (int64_t)ctx->num_sms * ctx->tune.fof_link_ctas_per_sm);
    RS_LAUNCH(ctx, "fof_occ", k_fof_occ, grid, T, 0, (const uint32_t *)n_cells, (const uint64_t *)cell_key,
              (const uint32_t *)table, occ);

    RS_WS(ctx, int, parent, WS_FOF_PARENT, n);
    RS_WS(ctx, int, root_min, WS_FOF_ROOTMIN, n);
    RS_LAUNCH(ctx, "fof_iota", k_iota_i32, nb, T, 0, parent, n);
    RS_LAUNCH(ctx, "fof_fill", k_fill_u32, std::min<int64_t>(nb, (int64_t)ctx->num_sms * 16), T, 0,
              (uint32_t *)root_min, n, 0x7fffffffu);
    // (flag's first n words are free once the cells are numbered: they hold
    // the common root of each coarse cell between the passes)
    int *uroot = (int *)flag;
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            RS_LAUNCH(ctx, "fof_uroot_first", k_fof_uroot_first, grid, T, 0, (const uint32_t *)n_cells,
                      (const uint64_t *)cell_key, (const uint32_t *)table, parent, uroot, ctx->d_status);
            RS_LAUNCH(ctx, "fof_uroot_check", k_fof_uroot_check, grid, T, 0, (const uint32_t *)n_cells,
                      (const uint64_t *)cell_key, (const uint32_t *)table, parent, uroot, ctx->d_status);
        }
        RS_LAUNCH(ctx, "fof_link", k_fof_link, grid, T, 0, (const uint32_t *)n_cells, (const uint64_t *)cell_key,
                  (const uint32_t *)cell_start, (const uint32_t *)table, (const uint64_t *)occ, (const float4 *)spos,
                  parent, pass == 1 ? (const int *)uroot : nullptr, g, pass, ctx->d_status);
    }
    if (dense_n >= 0) {
        // accelerated variant: dense flags, centre rounds, 2l joins
        RS_WS(ctx, uint8_t, acc, WS_FOF_ACC, 2 * n + 64);
        uint8_t *sa = acc, *sb = acc + n;
        unsigned long long *acnt = (unsigned long long *)(acc + (2 * n + 7) / 8 * 8);
        RS_LAUNCH(ctx, "fof_acc_count", k_acc_count, nb, T, 0, n, (const uint32_t *)cell_of,
                  (const uint64_t *)cell_key, (const uint32_t *)cell_start, (const uint32_t *)table,
                  (const uint64_t *)occ, (const float4 *)spos, g, (int)dense_n, sa);
        for (int round = 0;; round++) {
            if (round >= ACC_MAX_ROUNDS)
                return rs_fail(ctx, RS_ERR_INTERNAL, "rs_fof3d_accel: the centre choice did not settle");
            RS_CUDA(ctx, cudaMemsetAsync(acnt, 0, sizeof(unsigned long long), ctx->stream));
            RS_LAUNCH(ctx, "fof_acc_round", k_acc_round, nb, T, 0, n, (const uint32_t *)cell_of,
                      (const uint64_t *)cell_key, (const uint32_t *)cell_start, (const uint32_t *)table,
                      (const uint64_t *)occ, (const float4 *)spos, (const uint32_t *)idx, g, (const uint8_t *)sa, sb,
                      acnt);
            int64_t left = 0;
            RS_TRY(rs_read_i64(ctx, acnt, 1, &left, "rs_fof3d_accel"));
            std::swap(sa, sb);
            if (left == 0) break;
        }
        // the same tests at 2l: every threshold scales by exactly 2 or 4
        FofGeom g2 = g;
        g2.l = 2.0 * g.l;
        g2.l2 = 4.0 * g.l2;
        g2.lo32 = 4.0f * g.lo32;
        g2.hi32 = 4.0f * g.hi32;
        RS_CUDA(ctx, cudaMemsetAsync(acnt + 1, 0, sizeof(unsigned long long), ctx->stream));
        RS_LAUNCH(ctx, "fof_acc_join", k_acc_join, nb, T, 0, n, (const uint32_t *)cell_of, (const uint64_t *)cell_key,
                  (const uint32_t *)cell_start, (const uint32_t *)table, (const uint64_t *)occ, (const float4 *)spos,
                  g2, (const uint8_t *)sa, parent, acnt + 1, ctx->d_status);
        if (n_centres) RS_TRY(rs_read_i64(ctx, acnt + 1, 1, n_centres, "rs_fof3d_accel"));
    }
    RS_LAUNCH(ctx, "fof_rootmin", k_fof_rootmin, grid, T, 0, (const uint32_t *)n_cells,
              (const uint32_t *)cell_start, (const uint32_t *)idx, parent, root_min,
              rs_fault("timeout1") ? 1 : RS_SPIN_LIMIT, ctx->d_status);
    RS_LAUNCH(ctx, "fof_labels", k_fof_labels, nb, T, 0, n, (const uint32_t *)idx, (const uint32_t *)cell_of,
              parent, (const int *)root_min, labels, ctx->d_status);
    if (n_groups || n_tieband) {
        unsigned long long *cnt = (unsigned long long *)(flag + 2 * n + 2);
        RS_CUDA(ctx, cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), ctx->stream));
        if (n_groups)
            RS_LAUNCH(ctx, "fof_count_roots", k_fof_count_roots, grid, T, 0, (const uint32_t *)n_cells,
                      (const int *)parent, cnt);
        if (n_tieband)
            RS_LAUNCH(ctx, "fof_tieband", k_fof_tieband, grid, T, 0, (const uint32_t *)n_cells,
                      (const uint64_t *)cell_key, (const uint32_t *)cell_start, (const uint32_t *)table,
                      (const uint64_t *)occ, (const float4 *)spos, g, cnt + 1);
        int64_t h[2];
        RS_TRY(rs_read_i64(ctx, cnt, 2, h, "rs_fof3d"));
        if (n_groups) *n_groups = h[0];
        if (n_tieband) *n_tieband = h[1];
    }
    return RS_OK;
}

}  // namespace

extern "C" rs_status rs_fof3d(rs_ctx *ctx, const float *pos, int32_t stride, int64_t n, double box, double b,
                              int32_t *labels, int64_t *n_groups, int64_t *n_tieband)
{
    return fof_run(ctx, pos, stride, n, box, b, -1, labels, n_groups, n_tieband, nullptr);
}

extern "C" rs_status rs_fof3d_accel(rs_ctx *ctx, const float *pos, int32_t stride, int64_t n, double box, double b,
                                    int32_t dense_n, int32_t *labels, int64_t *n_groups, int64_t *n_centres)
{
    if (ctx && dense_n < 0) return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_fof3d_accel: dense_n must be >= 0");
    return fof_run(ctx, pos, stride, n, box, b, dense_n, labels, n_groups, nullptr, n_centres);
}

// ---------------------------------------------------------------------------
// group CSR (App. A work units)
// ---------------------------------------------------------------------------
namespace {

// Members per label.  The lanes of a warp that share a label add together
// (one atomic per distinct label in the warp): neighbours in the input often
// belong to one group, whose counter would otherwise take one atomic per
// member.
__global__ void k_gs_count(int64_t n, const int32_t *labels, uint32_t *count, rs_dev_status *st)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int32_t l = -1;
    if (i < n) {
        l = labels[i];
        if (l < 0 || l > i) {
            dev_fail(st, DEV_BADARG, 20, i);
            l = -1;
        }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, l);
    if (l >= 0 && lane_id() == __ffs(peers) - 1) atomicAdd(&count[l], (uint32_t)__popc(peers));
}

// root flags: groups of >= min_n members, keyed by their label (= root index)
__global__ void k_gs_rootflag(int64_t n, const int32_t *labels, const uint32_t *count, int32_t min_n,
                              uint32_t *rflag)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rflag[i] = (labels[i] == (int32_t)i && count[i] >= (uint32_t)min_n) ? 1u : 0u;  // label i is in range
}

// member flags
__global__ void k_gs_memflag(int64_t n, const int32_t *labels, const uint32_t *count, int32_t min_n,
                             uint32_t *mflag)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t l = labels[i];
    mflag[i] = (l >= 0 && l <= i && count[l] >= (uint32_t)min_n) ? 1u : 0u;
}

__global__ void k_gs_compact(int64_t n, const int32_t *labels, const uint32_t *mflag, const uint32_t *mscan,
                             const uint32_t *rscan, uint32_t *keys, uint32_t *vals)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !mflag[i]) return;
    uint32_t p = mscan[i];
    keys[p] = rscan[labels[i]];
    vals[p] = (uint32_t)i;
}

__global__ void k_gs_sizes(int64_t n, const uint32_t *rflag, const uint32_t *rscan, const uint32_t *count,
                           int64_t *offsets)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !rflag[i]) return;
    offsets[rscan[i]] = count[i];
}

}  // namespace

extern "C" rs_status rs_group_sort(rs_ctx *ctx, const int32_t *labels, int64_t n, int32_t min_n, int32_t *perm,
                                   int64_t *offsets, int64_t offsets_cap, int64_t *n_groups, int64_t *n_members)
{
    if (!ctx) return RS_ERR_INVALID_ARG;
    if (n < 0 || !n_groups || !n_members || min_n < 1 || offsets_cap < 1 || !offsets ||
        (n > 0 && (!labels || !perm)))
        return rs_fail(ctx, RS_ERR_INVALID_ARG, "rs_group_sort: bad argument");
    if (n >= ((int64_t)1 << 31)) return rs_fail(ctx, RS_ERR_TOO_LARGE, "rs_group_sort: n >= 2^31");
    if (n == 0) {
        *n_groups = 0;
        *n_members = 0;
        RS_CUDA(ctx, cudaMemsetAsync(offsets, 0, sizeof(int64_t), ctx->stream));
        return RS_OK;
    }
    RsStageGuard running(&ctx->in_gs);
    RsRange range("rs_group_sort");
    const int64_t T = 256, nb = ceil_div(n, T);
    RS_WS(ctx, uint32_t, count, WS_GS_COUNT, n);
    RS_WS(ctx, uint32_t, fl, WS_GS_FLAG, 4 * n + 8);
    uint32_t *rflag = fl, *rscan = fl + n, *mflag = fl + 2 * n, *mscan = fl + 3 * n;
    uint32_t *tot = fl + 4 * n;  // [0] groups, [1] members
    RS_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(uint32_t) * n, ctx->stream));
    RS_LAUNCH(ctx, "gs_count", k_gs_count, nb, T, 0, n, labels, count, ctx->d_status);
    RS_LAUNCH(ctx, "gs_rootflag", k_gs_rootflag, nb, T, 0, n, labels, (const uint32_t *)count, min_n, rflag);
    RS_LAUNCH(ctx, "gs_memflag", k_gs_memflag, nb, T, 0, n, labels, (const uint32_t *)count, min_n, mflag);
    RS_CUDA(ctx, cudaMemcpyAsync(rscan, rflag, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    RS_CUDA(ctx, cudaMemcpyAsync(mscan, mflag, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    RS_TRY(rs_scan_u32(ctx, rscan, n, tot));
    RS_TRY(rs_scan_u32(ctx, mscan, n, tot + 1));
    uint32_t h2[2];
    RS_CUDA(ctx, cudaMemcpyAsync(ctx->h_scratch, tot, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    RS_TRY(rs_sync_check(ctx, "rs_group_sort"));
    memcpy(h2, ctx->h_scratch, sizeof h2);
    const int64_t G = h2[0], Mm = h2[1];
    *n_groups = G;
    *n_members = Mm;
    if (offsets_cap < G + 1) return rs_fail(ctx, RS_ERR_INTERNAL, "rs_group_sort: offsets capacity too small");
    RS_WS(ctx, uint64_t, kbuf, WS_SORT_K0, 2 * Mm);  // reused as two u32 key arrays
    uint32_t *k0 = (uint32_t *)kbuf, *k1 = (uint32_t *)kbuf + Mm;
    RS_WS(ctx, uint32_t, vtmp, WS_SORT_V1, Mm);
    uint32_t *v0 = (uint32_t *)perm;
    RS_LAUNCH(ctx, "gs_compact", k_gs_compact, nb, T, 0, n, labels, (const uint32_t *)mflag,
              (const uint32_t *)mscan, (const uint32_t *)rscan, k0, v0);
    int bits = 0;
    while (bits < 32 && ((uint64_t)(G > 0 ? G - 1 : 0) >> bits) != 0) bits++;
    bool alt = false;
    RS_TRY(rs_radix_sort_u32(ctx, k0, k1, v0, vtmp, Mm, bits, &alt, "sort_gs"));
    if (alt)
        RS_CUDA(ctx, cudaMemcpyAsync(perm, vtmp, sizeof(uint32_t) * Mm, cudaMemcpyDeviceToDevice, ctx->stream));
    RS_CUDA(ctx, cudaMemsetAsync(offsets, 0, sizeof(int64_t) * (G + 1), ctx->stream));
    RS_LAUNCH(ctx, "gs_sizes", k_gs_sizes, nb, T, 0, n, (const uint32_t *)rflag, (const uint32_t *)rscan,
              (const uint32_t *)count, offsets);
    RS_TRY(rs_scan_i64(ctx, offsets, G + 1, nullptr));
    return rs_sync_check(ctx, "rs_group_sort");
}

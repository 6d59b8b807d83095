// rs_refine.cuh -- pieces of the phase-space hierarchy shared by the
// refinement kernels (rs_refine.cu) and the assignment (rs_assign.cu).
#pragma once

#include "rs_internal.cuh"

// Node table (structure of arrays, device).  A node's members are the
// member slots [first, first + count) of the tree's member array.
struct NodeArrays {
    int *parent, *level, *first, *count, *minidx, *nchild, *tie, *root;
    int *shift;    // periodic unwrap of the node's group: bit a set = axis a shifted
    double *lnk, *xbar, *vbar, *sigx, *sigv;
    int *counter;  // number of nodes allocated (device scalar)
    int cap;
};

struct rs_tree {
    int64_t n_total = 0;     // particles in the catalogue
    int64_t n_members = 0;   // member slots
    int64_t n_nodes = 0, n_seeds = 0, n_tieband = 0, sum_level_members = 0;
    int32_t n_levels = 0;
    int32_t n_fallback_levels = 0;  // big-node levels that needed the full nearest-neighbour search
    int64_t sum_big_level_members = 0;
    double box = 0;
    NodeArrays nd{};
    int *members = nullptr;  // particle index per member slot
    void *block = nullptr;   // single device allocation holding everything
};

// Per-halo results of the assignment, kept for the halo-property steps
// (Sec. 3.4, 3.5.1).  Halos are in the assignment's rank order.
struct rs_halos {
    int64_t n_halos = 0, n_nodes = 0;
    int *id = nullptr;         // halo id: smallest particle index of its seeds
    double *xbar = nullptr;    // 3 per halo: centre of the seeds' members
    double *vbar = nullptr;    // 3 per halo
    double *sigv = nullptr;    // velocity dispersion of the seeds' members
    double *rdyn2 = nullptr;   // r_dyn,vir^2 (Eq. 4)
    int *root = nullptr;       // root node of the halo's 3D group
    int *leaf_halo = nullptr;  // per tree node: the halo of a seed, -1 for inner nodes
    void *block = nullptr;
};

// Fixed-point scale of the exact moment sums: positions and velocities are
// rounded to multiples of 2^-32 (of their units) before summation.
#define RS_FX 4294967296.0f
#define RS_FX_INV 2.3283064365386963e-10

// Relative half-width, on squared distances, of the band within which a
// float32 comparison is re-done in float64: 2^-20 = 16 float32 ulps, twice
// the worst-case error (8 ulps) of the float32 6D distance below.
#define RS_BAND 9.5367431640625e-07

struct Metric6 {
    float ax, av;       // float32 factors on |dx|^2 and |dv|^2 (common scale applied)
    double ax64, av64;  // float64 factors (same scale)
    double scale;       // common factor: metric = scale * Eq. 1
};

__device__ __forceinline__ float d2_32(float4 pa, float4 va, float4 pb, float4 vb, const Metric6 &m)
{
    float dx = pa.x - pb.x, dy = pa.y - pb.y, dz = pa.z - pb.z;
    float ux = va.x - vb.x, uy = va.y - vb.y, uz = va.z - vb.z;
    float sx = dx * dx + dy * dy + dz * dz;
    float sv = ux * ux + uy * uy + uz * uz;
    return sx * m.ax + sv * m.av;
}

__device__ __forceinline__ double d2_64(float4 pa, float4 va, float4 pb, float4 vb, const Metric6 &m)
{
    double dx = f64_sub(pa.x, pb.x), dy = f64_sub(pa.y, pb.y), dz = f64_sub(pa.z, pb.z);
    double ux = f64_sub(va.x, vb.x), uy = f64_sub(va.y, vb.y), uz = f64_sub(va.z, vb.z);
    double sx = f64_add(f64_add(f64_mul(dx, dx), f64_mul(dy, dy)), f64_mul(dz, dz));
    double sv = f64_add(f64_add(f64_mul(ux, ux), f64_mul(uy, uy)), f64_mul(uz, uz));
    return f64_add(f64_mul(sx, m.ax64), f64_mul(sv, m.av64));
}

__device__ __forceinline__ long long fx(float x) { return __float2ll_rn(x * RS_FX); }

// Exact moment accumulator: 128-bit sums of the fixed-point offsets of each
// coordinate from a reference member, and 128-bit sums of their squares over
// the three position and the three velocity axes.  Two's-complement addition
// modulo 2^128 is associative, so partial sums may be combined in any order
// and the result is exact whenever the true sum fits.
struct MomAcc {
    unsigned long long s_lo[6], s_hi[6];  // dx, dy, dz, dvx, dvy, dvz
    unsigned long long qx_lo, qx_hi, qv_lo, qv_hi;
};

__device__ __forceinline__ void mom_zero(MomAcc &a)
{
#pragma unroll
    for (int i = 0; i < 6; i++) a.s_lo[i] = a.s_hi[i] = 0;
    a.qx_lo = a.qx_hi = a.qv_lo = a.qv_hi = 0;
}

__device__ __forceinline__ void add128(unsigned long long &lo, unsigned long long &hi, unsigned long long alo,
                                       unsigned long long ahi)
{
    unsigned long long n = lo + alo;
    hi += ahi + (n < lo ? 1ull : 0ull);
    lo = n;
}

__device__ __forceinline__ void sadd128(unsigned long long &lo, unsigned long long &hi, long long d)
{
    add128(lo, hi, (unsigned long long)d, (unsigned long long)(d >> 63));
}

__device__ __forceinline__ void sq_add(unsigned long long &lo, unsigned long long &hi, long long d)
{
    unsigned long long u = (unsigned long long)(d < 0 ? -d : d);
    add128(lo, hi, u * u, __umul64hi(u, u));
}

struct MomRef {
    long long c[6];
};

__device__ __forceinline__ MomRef mom_ref(float4 p, float4 v)
{
    MomRef r;
    r.c[0] = fx(p.x);
    r.c[1] = fx(p.y);
    r.c[2] = fx(p.z);
    r.c[3] = fx(v.x);
    r.c[4] = fx(v.y);
    r.c[5] = fx(v.z);
    return r;
}

__device__ __forceinline__ void mom_add(MomAcc &a, float4 p, float4 v, const MomRef &r)
{
    const long long d[6] = {fx(p.x) - r.c[0], fx(p.y) - r.c[1], fx(p.z) - r.c[2],
                            fx(v.x) - r.c[3], fx(v.y) - r.c[4], fx(v.z) - r.c[5]};
#pragma unroll
    for (int i = 0; i < 6; i++) sadd128(a.s_lo[i], a.s_hi[i], d[i]);
    sq_add(a.qx_lo, a.qx_hi, d[0]);
    sq_add(a.qx_lo, a.qx_hi, d[1]);
    sq_add(a.qx_lo, a.qx_hi, d[2]);
    sq_add(a.qv_lo, a.qv_hi, d[3]);
    sq_add(a.qv_lo, a.qv_hi, d[4]);
    sq_add(a.qv_lo, a.qv_hi, d[5]);
}

__device__ __forceinline__ void mom_merge(MomAcc &a, const MomAcc &b)
{
#pragma unroll
    for (int i = 0; i < 6; i++) add128(a.s_lo[i], a.s_hi[i], b.s_lo[i], b.s_hi[i]);
    add128(a.qx_lo, a.qx_hi, b.qx_lo, b.qx_hi);
    add128(a.qv_lo, a.qv_hi, b.qv_lo, b.qv_hi);
}

__device__ __forceinline__ void mom_warp_reduce(MomAcc &a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        MomAcc b;
#pragma unroll
        for (int i = 0; i < 6; i++) {
            b.s_lo[i] = __shfl_xor_sync(0xffffffffu, a.s_lo[i], o);
            b.s_hi[i] = __shfl_xor_sync(0xffffffffu, a.s_hi[i], o);
        }
        b.qx_lo = __shfl_xor_sync(0xffffffffu, a.qx_lo, o);
        b.qx_hi = __shfl_xor_sync(0xffffffffu, a.qx_hi, o);
        b.qv_lo = __shfl_xor_sync(0xffffffffu, a.qv_lo, o);
        b.qv_hi = __shfl_xor_sync(0xffffffffu, a.qv_hi, o);
        mom_merge(a, b);
    }
}

__device__ __forceinline__ void atomic_add128(unsigned long long *lo, unsigned long long *hi, unsigned long long alo,
                                              unsigned long long ahi)
{
    unsigned long long old = atomicAdd(lo, alo);
    atomicAdd(hi, ahi + ((old + alo) < old ? 1ull : 0ull));
}

// Atomically adds a partial accumulator into a global one (the carry from
// each low word into its high word is exact).
__device__ __forceinline__ void mom_atomic_add(MomAcc *g, const MomAcc &a)
{
#pragma unroll
    for (int i = 0; i < 6; i++) atomic_add128(&g->s_lo[i], &g->s_hi[i], a.s_lo[i], a.s_hi[i]);
    atomic_add128(&g->qx_lo, &g->qx_hi, a.qx_lo, a.qx_hi);
    atomic_add128(&g->qv_lo, &g->qv_hi, a.qv_lo, a.qv_hi);
}

__device__ __forceinline__ double u128_to_double(unsigned long long lo, unsigned long long hi)
{
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

// Signed 128-bit value to double: convert the magnitude (a small negative
// value has a low word near 2^64, which would cancel against the high word).
__device__ __forceinline__ double s128_to_double(unsigned long long lo, unsigned long long hi)
{
    if ((long long)hi < 0) {
        unsigned long long nlo = ~lo + 1ull;
        unsigned long long nhi = ~hi + (nlo == 0 ? 1ull : 0ull);
        return -u128_to_double(nlo, nhi);
    }
    return u128_to_double(lo, hi);
}

struct MomOut {
    double xbar[3], vbar[3], sigx, sigv;
};

// x wrapped into [0, box).  Inside (-box, 2 box) one add or subtract gives
// what fmod would (x - box is exact there, Sterbenz); fmod takes the rest.
__device__ __forceinline__ double wrap_box(double x, double box)
{
    if (x >= 0 && x < box) return x;
    if (x < 0 && x > -box) {
        x += box;
        return x >= box ? x - box : x;
    }
    if (x >= box && x < 2 * box) return x - box;
    x = fmod(x, box);
    if (x < 0) x += box;
    if (x >= box) x -= box;
    return x;
}

// Mean and 3D dispersions from the exact sums (Sec. 3.2).  The mean is the
// reference member's exact float32 coordinate plus the mean fixed-point
// offset, so members that all share the reference's value give it exactly.
__device__ __forceinline__ MomOut mom_finalize(const MomAcc &a, float4 pref, float4 vref, int64_t n, double box)
{
    MomOut o;
    // float64 is scarce on this part: one reciprocal of n, the rest multiplies
    const double inv_n = 1.0 / (double)n;
    const double ref[6] = {pref.x, pref.y, pref.z, vref.x, vref.y, vref.z};
    double s2x = 0, s2v = 0, mean[6];
    for (int i = 0; i < 6; i++) {
        double s = s128_to_double(a.s_lo[i], a.s_hi[i]) * RS_FX_INV;
        mean[i] = s * inv_n;
        if (i < 3) s2x += s * s;
        else s2v += s * s;
    }
    for (int i = 0; i < 3; i++) {
        o.xbar[i] = wrap_box(ref[i] + mean[i], box);
        o.vbar[i] = ref[3 + i] + mean[3 + i];
    }
    const double q2 = RS_FX_INV * RS_FX_INV;
    double qx = u128_to_double(a.qx_lo, a.qx_hi) * q2;
    double qv = u128_to_double(a.qv_lo, a.qv_hi) * q2;
    double vx = (qx - s2x * inv_n) * inv_n, vv = (qv - s2v * inv_n) * inv_n;
    o.sigx = vx > 0 ? sqrt(vx) : 0.0;
    o.sigv = vv > 0 ? sqrt(vv) : 0.0;
    return o;
}

// Metric of Eq. 1 with a common scale that keeps both factors <= 1.
__device__ __forceinline__ Metric6 metric_of(double sigx, double sigv)
{
    Metric6 m;
    double ax = sigx > 0 ? 1.0 / (sigx * sigx) : 0.0;
    double av = sigv > 0 ? 1.0 / (sigv * sigv) : 0.0;
    double mx = ax > av ? ax : av;
    double c = mx > 0 ? 1.0 / mx : 1.0;
    m.ax64 = ax * c;
    m.av64 = av * c;
    m.ax = (float)m.ax64;
    m.av = (float)m.av64;
    m.scale = c;
    return m;
}

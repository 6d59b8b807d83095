// rs_internal.cuh -- shared internals of the GB300 ROCKSTAR library:
// context, workspace, device status word, launch accounting and small device
// helpers.  Not part of the public ABI (include/rsgpu.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "rsgpu.h"

// NVTX range over a scope: each entry point and stage is named for a
// profiler that attaches (ncu --nvtx, Nsight Systems); without one it costs
// a function-pointer check.
struct RsRange {
    explicit RsRange(const char *name) { nvtxRangePushA(name); }
    ~RsRange() { nvtxRangePop(); }
};

// ---------------------------------------------------------------------------
// Device status word: kernels that hit a bounded wait or a capacity limit
// record a code here instead of trapping; the host reads it at sync points.
// ---------------------------------------------------------------------------
enum rs_dev_code : int32_t {
    DEV_OK = 0,
    DEV_TIMEOUT = 1,     // a bounded loop ran out of iterations
    DEV_OVERFLOW = 2,    // a table, stack or list was too small
    DEV_EXTENT = 3,      // a node spans half the box or more
    DEV_BADARG = 4,      // an input violated a documented precondition
    DEV_INTERNAL = 5,    // a consistency check failed
};

struct rs_dev_status {
    int32_t code;    // first error code recorded
    int32_t site;    // which check recorded it
    int64_t detail;  // site-specific value
};

__device__ __forceinline__ void dev_fail(rs_dev_status *st, int32_t code, int32_t site, int64_t detail)
{
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->site = site;
        st->detail = detail;
    }
}

// Upper bound on iterations of any retry or pointer-chasing loop.
#define RS_SPIN_LIMIT (1 << 22)

// ---------------------------------------------------------------------------
// Workspace slots (grow-only device buffers owned by the context)
// ---------------------------------------------------------------------------
enum rs_ws_slot {
    WS_SCAN_TMP = 0,
    WS_SORT_K0, WS_SORT_K1, WS_SORT_V0, WS_SORT_V1, WS_SORT_HIST,
    WS_FOF_CELLKEY, WS_FOF_CELLSTART, WS_FOF_CELLOF, WS_FOF_PARENT, WS_FOF_ROOTMIN, WS_FOF_TABLE,
    WS_FOF_OCC, WS_FOF_POS4, WS_FOF_MISC, WS_FOF_ACC,
    WS_GS_COUNT, WS_GS_FLAG,
    WS_RF_POS, WS_RF_VEL, WS_RF_POS2, WS_RF_VEL2, WS_RF_IDX2,
    WS_RF_DNN, WS_RF_PARENT, WS_RF_MISC0, WS_RF_MISC1, WS_RF_MISC2, WS_RF_MISC3, WS_RF_NODEQ,
    WS_RF_ACC, WS_RF_HIST, WS_RF_BAND, WS_RF_MISC4, WS_RF_MISC5, WS_RF_JOBS, WS_RF_JOBS2, WS_RF_SDNN, WS_RF_R2,
    WS_RF_SRCH, WS_RF_SUBQ, WS_RF_KDV,
    WS_HL_IDS, WS_HL_PURE, WS_HL_BEST, WS_HL_OFF, WS_HL_TILES, WS_HL_TREE, WS_HL_REF, WS_HL_UPOS, WS_HL_TPOS,
    WS_HL_TMEM, WS_HL_MK0, WS_HL_MK1, WS_HL_MV0, WS_HL_MV1, WS_HL_BOX, WS_HL_JOBS,
    WS_AS_0, WS_AS_1, WS_AS_2, WS_AS_3, WS_AS_4, WS_AS_5, WS_AS_6, WS_AS_7, WS_AS_8, WS_AS_9,
    WS_IO_POS, WS_IO_VEL, WS_IO_LAB, WS_IO_HID, WS_IO_PERM, WS_IO_OFF,
    WS_SELFTEST,
    WS_NUM_SLOTS
};

struct rs_prof_rec {
    int name_id;
    cudaEvent_t a, b;
};

struct rs_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 1;
    std::string last_error;
    void *ws_ptr[WS_NUM_SLOTS] = {};
    size_t ws_size[WS_NUM_SLOTS] = {};
    rs_dev_status *d_status = nullptr;
    rs_dev_status *h_status = nullptr;   // pinned
    int64_t *h_scratch = nullptr;        // pinned, 64 entries
    int prof_on = 0;
    std::vector<std::string> prof_names;
    std::vector<rs_prof_rec> prof_recs;
    std::vector<cudaEvent_t> ev_free;
    int64_t launches = 0;
    // the workspace slots are fixed regions set up by the caller (no device
    // allocation allowed): a slot that is too small is an internal error
    int fixed_ws = 0;
    // set while a 3D FOF or group-sort call runs: its slots are in use and
    // must not be released to make room (see rs_ws)
    int in_fof = 0, in_gs = 0;
    rs_tuning tune;  // launch choices (rs_set_tuning)
    rs_ctx() { rs_tuning_default(&tune); }
    // second stream and events for copies that overlap the kernels of the
    // context's stream (rs_find_halos with host buffers); created on first use
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_io[3] = {nullptr, nullptr, nullptr};
};

// ---------------------------------------------------------------------------
// Host helpers (rs_ctx.cu)
// ---------------------------------------------------------------------------
rs_status rs_fail(rs_ctx *ctx, rs_status s, const std::string &msg);
rs_status rs_cuda_fail(rs_ctx *ctx, cudaError_t e, const char *where);
// Device buffer of at least `bytes` for a slot; contents are kept while the
// slot does not grow.  When the device is out of memory, the slots of the 3D
// FOF and of the group sort (scratch of those calls only) are released if
// neither call is running, and the allocation is tried once more.  Returns
// nullptr (and records RS_ERR_OOM) on failure.
void *rs_ws(rs_ctx *ctx, int slot, size_t bytes);
// Total bytes of the context's workspace slots.
size_t rs_ws_total(const rs_ctx *ctx);

// Marks a 3D FOF or group-sort call as running for its scope.
struct RsStageGuard {
    int *flag;
    explicit RsStageGuard(int *f) : flag(f) { *flag = 1; }
    ~RsStageGuard() { *flag = 0; }
};
int rs_prof_begin(rs_ctx *ctx, const char *name);
void rs_prof_end(rs_ctx *ctx, int rec);
// Synchronises the stream and turns the device status word into an rs_status.
rs_status rs_sync_check(rs_ctx *ctx, const char *where);
// Copies `count` int64 values from device to host scratch and synchronises.
rs_status rs_read_i64(rs_ctx *ctx, const void *dsrc, int count, int64_t *dst, const char *where);
// Host-side fault injection for the failure-detection tests: true when the
// environment variable RS_FAULT, a comma-separated list, names `site`.
// Sites: "alloc" (every workspace allocation fails), "timeout1" (the 3D FOF
// label pass runs with a bound of one step per find), "offsets" (rs_find_halos
// corrupts the group offsets it passes to the refinement), "bracket" (the
// sampled search bracket of every big node of odd rank is treated as failed,
// which sends those nodes to the unbounded fallback search).
bool rs_fault(const char *site);

#define RS_TRY(expr)                         \
    do {                                     \
        rs_status _s = (expr);               \
        if (_s != RS_OK) return _s;          \
    } while (0)

#define RS_CUDA(ctx, call)                                          \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return rs_cuda_fail((ctx), _e, #call); \
    } while (0)

// Launch with accounting and optional event bracketing.  Skips empty grids.
#define RS_LAUNCH(ctx, name, kernel, grid, block, smem, ...)                           \
    do {                                                                               \
        if ((grid) > 0) {                                                              \
            int _pr = rs_prof_begin((ctx), (name));                                    \
            kernel<<<(unsigned)(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__); \
            (ctx)->launches++;                                                         \
            rs_prof_end((ctx), _pr);                                                   \
            cudaError_t _e = cudaGetLastError();                                       \
            if (_e != cudaSuccess) return rs_cuda_fail((ctx), _e, (name));             \
        }                                                                              \
    } while (0)

#define RS_WS(ctx, T, var, slot, count)                                         \
    T *var = (T *)rs_ws((ctx), (slot), sizeof(T) * (size_t)((count) > 0 ? (count) : 1)); \
    if (!var) return (ctx)->fixed_ws ? RS_ERR_INTERNAL : RS_ERR_OOM

__host__ __device__ static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Scan and sort (rs_scan_sort.cu)
// ---------------------------------------------------------------------------
// In-place exclusive prefix sum; *total (device, optional) receives the sum.
rs_status rs_scan_u32(rs_ctx *ctx, uint32_t *data, int64_t n, uint32_t *total);
rs_status rs_scan_i64(rs_ctx *ctx, int64_t *data, int64_t n, int64_t *total);
// keys per radix-sort tile; the histogram workspace holds 256 counts per tile
constexpr int64_t RS_SORT_TILE = 2048;
// Stable LSD radix sort of (key, value) pairs on key bits [0, nbits).  The
// caller provides both ping-pong buffers; *out_in_alt says whether the
// sorted data ended in (k1, v1).
// `tag` names the launches for the per-kernel profile (tag_hist, tag_scatter).
rs_status rs_radix_sort_u64(rs_ctx *ctx, uint64_t *k0, uint64_t *k1, uint32_t *v0, uint32_t *v1, int64_t n,
                            int nbits, bool *out_in_alt, const char *tag = "sort");
rs_status rs_radix_sort_u32(rs_ctx *ctx, uint32_t *k0, uint32_t *k1, uint32_t *v0, uint32_t *v1, int64_t n,
                            int nbits, bool *out_in_alt, const char *tag = "sort");

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// float64 arithmetic without contraction into fused multiply-adds, so a
// recheck evaluates exactly the separate multiplies and adds it writes.
__device__ __forceinline__ double f64_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double f64_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double f64_sub(double a, double b) { return __dsub_rn(a, b); }

// Fine cells per side of the 3D FOF grid for (n, box, b): the side s is the
// largest with sqrt(3) s (1 + 2 err) < l, err being the float32 error of a
// fine-cell coordinate in cell units (2.0001 u Gf), rounded down so that 4 Gc
// cells fill the box.  Returns Gc (coarse cells per side; 0 when l <= 0) and
// the estimate of Gf and err the caller checks the grid against.  Host only;
// every caller of the 3D FOF grid uses it.
struct FofGridSize {
    double gc, gf_est, err, l;
};
static inline FofGridSize fof_grid_size(int64_t n, double box, double b)
{
    FofGridSize r{0.0, 0.0, 0.0, rs_linking_length(n, box, b)};
    if (!(r.l > 0)) return r;
    const double u = 5.9604644775390625e-08;  // 2^-24
    r.gf_est = box * std::sqrt(3.0) / r.l + 16.0;
    r.err = 2.0001 * u * r.gf_est * 1.01;
    const double s_max = r.l * (1.0 - 1e-7) / (std::sqrt(3.0) * (1.0 + 2.0 * r.err));
    r.gc = std::ceil(box / (4.0 * s_max));
    return r;
}

// Lock-free union-find over int32 node ids: every root is the smallest id of
// its set (the larger root is hooked under the smaller one with a CAS, after
// the ECL-CC scheme of Jaiganesh & Burtscher 2018).  Loops are bounded; on
// running out they record DEV_TIMEOUT and give up.
__device__ __forceinline__ int uf_find_n(int *parent, int x, rs_dev_status *st, int limit)
{
    for (int it = 0; it < limit; it++) {
        int p = __ldcg(&parent[x]);
        if (p == x) return x;
        int g = __ldcg(&parent[p]);
        if (g != p) parent[x] = g;  // path halving (benign race: any ancestor is valid)
        x = g;
    }
    dev_fail(st, DEV_TIMEOUT, 1, x);
    return x;
}

__device__ __forceinline__ int uf_find(int *parent, int x, rs_dev_status *st)
{
    return uf_find_n(parent, x, st, RS_SPIN_LIMIT);
}

__device__ __forceinline__ void uf_union(int *parent, int a, int b, rs_dev_status *st)
{
    for (int it = 0; it < RS_SPIN_LIMIT; it++) {
        a = uf_find(parent, a, st);
        b = uf_find(parent, b, st);
        if (a == b) return;
        if (a > b) {
            int t = a;
            a = b;
            b = t;
        }
        int old = atomicCAS(&parent[b], b, a);
        if (old == b) return;
        b = old;
    }
    dev_fail(st, DEV_TIMEOUT, 2, a);
}

// Shared-memory variants (same scheme, block-local ids)
__device__ __forceinline__ int uf_find_s(int *parent, int x)
{
    for (int it = 0; it < 4096; it++) {
        int p = ((volatile int *)parent)[x];
        if (p == x) return x;
        x = p;
    }
    return x;
}

__device__ __forceinline__ void uf_union_s(int *parent, int a, int b, rs_dev_status *st)
{
    for (int it = 0; it < 65536; it++) {
        a = uf_find_s(parent, a);
        b = uf_find_s(parent, b);
        if (a == b) return;
        if (a > b) {
            int t = a;
            a = b;
            b = t;
        }
        int old = atomicCAS(&parent[b], b, a);
        if (old == b) return;
        b = old;
    }
    dev_fail(st, DEV_TIMEOUT, 3, a);
}

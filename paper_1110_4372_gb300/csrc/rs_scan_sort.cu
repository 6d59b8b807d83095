// rs_scan_sort.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Scan: reduce-then-scan over blocks of 4096 elements, recursive on the block
// sums.  Sort: 8-bit digits, tiles of 4096 keys (256 threads x 16); per pass
// a histogram kernel, a scan of the digit-major histogram and a scatter
// kernel that ranks keys stably with warp match-any and per-warp counters.
#include "rs_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int64_t SCAN_PER_BLOCK = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_excl_scan(T v, T *total)
{
    __shared__ T wsum[SCAN_THREADS / 32];
    int lane = lane_id(), w = warp_id();
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        T s = lane < SCAN_THREADS / 32 ? wsum[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) wsum[lane] = s;
    }
    __syncthreads();
    T before = (w > 0 ? wsum[w - 1] : T(0)) + x - v;
    if (total) *total = wsum[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return before;
}

template <typename T>
__global__ void k_scan_reduce(const T *data, int64_t n, T *sums)
{
    int64_t base = (int64_t)blockIdx.x * SCAN_PER_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++)
        if (base + j < n) s += data[base + j];
    __shared__ T wsum[SCAN_THREADS / 32];
    s = warp_sum(s);
    if (lane_id() == 0) wsum[warp_id()] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) t += wsum[w];
        sums[blockIdx.x] = t;
    }
}

template <typename T>
__global__ void k_scan_apply(T *data, int64_t n, const T *offsets, T *total)
{
    int64_t base = (int64_t)blockIdx.x * SCAN_PER_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        v[j] = (base + j < n) ? data[base + j] : T(0);
        s += v[j];
    }
    T btot;
    T run = block_excl_scan(s, &btot);
    if (offsets) run += offsets[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; j++) {
        if (base + j < n) data[base + j] = run;
        run += v[j];
    }
    if (total && gridDim.x == 1 && threadIdx.x == 0) *total = btot;
}

template <typename T>
rs_status scan_rec(rs_ctx *ctx, T *data, int64_t n, T *total, char *tmp, size_t tmp_bytes)
{
    if (n <= 0) {
        if (total) RS_CUDA(ctx, cudaMemsetAsync(total, 0, sizeof(T), ctx->stream));
        return RS_OK;
    }
    int64_t nb = ceil_div(n, SCAN_PER_BLOCK);
    if (nb == 1) {
        RS_LAUNCH(ctx, "scan_apply", k_scan_apply<T>, 1, SCAN_THREADS, 0, data, n, (const T *)nullptr, total);
        return RS_OK;
    }
    size_t need = ((sizeof(T) * (size_t)nb + 255) / 256) * 256;
    if (need > tmp_bytes) return rs_fail(ctx, RS_ERR_INTERNAL, "scan scratch too small");
    T *sums = (T *)tmp;
    RS_LAUNCH(ctx, "scan_reduce", k_scan_reduce<T>, nb, SCAN_THREADS, 0, (const T *)data, n, sums);
    RS_TRY(scan_rec<T>(ctx, sums, nb, total, tmp + need, tmp_bytes - need));
    RS_LAUNCH(ctx, "scan_apply", k_scan_apply<T>, nb, SCAN_THREADS, 0, data, n, (const T *)sums, (T *)nullptr);
    return RS_OK;
}

template <typename T>
rs_status scan_top(rs_ctx *ctx, T *data, int64_t n, T *total)
{
    size_t bytes = 0;
    for (int64_t m = ceil_div(n, SCAN_PER_BLOCK); m > 1; m = ceil_div(m, SCAN_PER_BLOCK))
        bytes += ((sizeof(T) * (size_t)m + 255) / 256) * 256;
    bytes += 1024;
    char *tmp = (char *)rs_ws(ctx, WS_SCAN_TMP, bytes);
    if (!tmp) return RS_ERR_OOM;
    return scan_rec<T>(ctx, data, n, total, tmp, bytes);
}

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int SORT_THREADS = 256;  // one thread per digit in the scatter's digit scan
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 8;
constexpr int64_t SORT_TILE = SORT_THREADS * SORT_ITEMS;
static_assert(SORT_TILE == RS_SORT_TILE, "tile size shared with the fixed-scratch entry point");
static_assert(SORT_THREADS == RADIX, "the scatter gives each digit one thread");

template <typename K>
__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist(const K *keys, int64_t n, int shift, uint32_t *hist,
                                                              int64_t ntiles)
{
    __shared__ uint32_t h[RADIX];
    for (int d = threadIdx.x; d < RADIX; d += SORT_THREADS) h[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * SORT_TILE;
#pragma unroll 4
    for (int j = 0; j < SORT_ITEMS; j++) {
        int64_t i = base + (int64_t)j * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & (RADIX - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += SORT_THREADS) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// One tile: stable ranks per warp (match_any), the tile's keys placed in
// shared memory in digit order, then written out in that order, so the
// items of one digit go to consecutive global slots (coalesced stores).
template <typename K>
__global__ void __launch_bounds__(SORT_THREADS, 4) k_sort_scatter(const K *kin, K *kout, const uint32_t *vin,
                                                                 uint32_t *vout, int64_t n, int shift,
                                                                 const uint32_t *hist, int64_t ntiles)
{
    __shared__ uint32_t wcnt[SORT_WARPS][RADIX];
    __shared__ uint32_t goff[RADIX];    // first global slot of each digit for this tile
    __shared__ uint32_t lstart[RADIX];  // first tile slot of each digit
    __shared__ uint32_t wsum[SORT_WARPS];
    __shared__ K skey[SORT_TILE];
    __shared__ uint32_t sval[SORT_TILE];
    const int lane = lane_id(), w = warp_id();
    for (int d = lane; d < RADIX; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const int64_t tbase = (int64_t)blockIdx.x * SORT_TILE;
    const int64_t wbase = tbase + (int64_t)w * 32 * SORT_ITEMS;
    const uint32_t lt = (1u << lane) - 1u;
    K key[SORT_ITEMS];
    uint32_t val[SORT_ITEMS];
    uint32_t rank[SORT_ITEMS];
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; j++) {
        int64_t i = wbase + j * 32 + lane;
        bool ok = i < n;
        key[j] = ok ? kin[i] : K(0);
        val[j] = ok ? vin[i] : 0u;
        uint32_t d = ok ? ((uint32_t)(key[j] >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (ok) before = wcnt[w][d];
        __syncwarp();
        if (ok && (peers & lt) == 0) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        rank[j] = before + __popc(peers & lt);
    }
    __syncthreads();
    // thread d: offsets of each warp within digit d, then the tile-local start
    // of digit d (an exclusive scan of the digit totals over the block)
    {
        const int d = threadIdx.x;
        uint32_t tot = 0;
#pragma unroll
        for (int ww = 0; ww < SORT_WARPS; ww++) {
            const uint32_t t = wcnt[ww][d];
            wcnt[ww][d] = tot;
            tot += t;
        }
        uint32_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        goff[d] = hist[(int64_t)d * ntiles + blockIdx.x];
        __syncthreads();
        uint32_t pre = 0;
        for (int ww = 0; ww < w; ww++) pre += wsum[ww];
        lstart[d] = pre + x - tot;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; j++) {
        if (wbase + j * 32 + lane < n) {
            const uint32_t d = (uint32_t)(key[j] >> shift) & (RADIX - 1);
            const uint32_t lp = lstart[d] + wcnt[w][d] + rank[j];
            skey[lp] = key[j];
            sval[lp] = val[j];
        }
    }
    __syncthreads();
    const int tn = (int)min((int64_t)SORT_TILE, n - tbase);
    for (int i = threadIdx.x; i < tn; i += SORT_THREADS) {
        const K k = skey[i];
        const uint32_t d = (uint32_t)(k >> shift) & (RADIX - 1);
        const uint32_t pos = goff[d] + ((uint32_t)i - lstart[d]);
        kout[pos] = k;
        vout[pos] = sval[i];
    }
}

template <typename K>
rs_status radix_sort(rs_ctx *ctx, K *k0, K *k1, uint32_t *v0, uint32_t *v1, int64_t n, int nbits, bool *alt,
                     const char *tag)
{
    const std::string hist_name = std::string(tag) + "_hist", scatter_name = std::string(tag) + "_scatter";
    *alt = false;
    if (n <= 1 || nbits <= 0) return RS_OK;
    if (n >= ((int64_t)1 << 32)) return rs_fail(ctx, RS_ERR_TOO_LARGE, "radix sort of 2^32 or more keys");
    int64_t ntiles = ceil_div(n, SORT_TILE);
    RS_WS(ctx, uint32_t, hist, WS_SORT_HIST, (int64_t)RADIX * ntiles);
    K *ki = k0, *ko = k1;
    uint32_t *vi = v0, *vo = v1;
    for (int shift = 0; shift < nbits; shift += RADIX_BITS) {
        RS_LAUNCH(ctx, hist_name.c_str(), k_sort_hist<K>, ntiles, SORT_THREADS, 0, (const K *)ki, n, shift, hist, ntiles);
        RS_TRY(scan_top<uint32_t>(ctx, hist, (int64_t)RADIX * ntiles, nullptr));
        RS_LAUNCH(ctx, scatter_name.c_str(), k_sort_scatter<K>, ntiles, SORT_THREADS, 0, (const K *)ki, ko,
                  (const uint32_t *)vi, vo, n, shift, (const uint32_t *)hist, ntiles);
        K *tk = ki;
        ki = ko;
        ko = tk;
        uint32_t *tv = vi;
        vi = vo;
        vo = tv;
        *alt = !*alt;
    }
    return RS_OK;
}

}  // namespace

rs_status rs_scan_u32(rs_ctx *ctx, uint32_t *data, int64_t n, uint32_t *total)
{
    return scan_top<uint32_t>(ctx, data, n, total);
}

rs_status rs_scan_i64(rs_ctx *ctx, int64_t *data, int64_t n, int64_t *total)
{
    return scan_top<long long>(ctx, (long long *)data, n, (long long *)total);
}

rs_status rs_radix_sort_u64(rs_ctx *ctx, uint64_t *k0, uint64_t *k1, uint32_t *v0, uint32_t *v1, int64_t n,
                            int nbits, bool *alt, const char *tag)
{
    return radix_sort<unsigned long long>(ctx, (unsigned long long *)k0, (unsigned long long *)k1, v0, v1, n,
                                          nbits, alt, tag);
}

rs_status rs_radix_sort_u32(rs_ctx *ctx, uint32_t *k0, uint32_t *k1, uint32_t *v0, uint32_t *v1, int64_t n,
                            int nbits, bool *alt, const char *tag)
{
    return radix_sort<uint32_t>(ctx, k0, k1, v0, v1, n, nbits, alt, tag);
}

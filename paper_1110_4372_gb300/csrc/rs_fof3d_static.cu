// rs_fof3d_static.cu -- 3D friends-of-friends without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// groups: a plugin running inside a host framework whose own pool allocator
// owns all device memory, a long-running service that fixes its device
// memory budget at start-up and forbids allocation afterwards, or a
// latency-critical loop that must not stall on an allocator or risk running
// out of memory mid-run.  rs_fof3d_static serves them: it computes exactly
// what rs_fof3d computes, but every temporary lives in one fixed scratch
// array that is part of the library image.
//
// The scratch is a file-scope __device__ array.  Every GPU that loads the
// library holds it (about 10 MB) until the process exits.  In host code its
// name is only a stand-in, not a device address, so the first call on each
// device looks its address up with cudaGetSymbolAddress (with that device
// current) and caches it; later calls on that device reuse the cached
// address.  All calls share the array and it keeps the contents of the last
// call; everything that must start at zero is cleared at the start of each
// call.  Two calls that overlap on the GPU (on different streams, or from
// several host threads) race on the array and give wrong results.
#include <cmath>
#include <cstring>
#include <mutex>

#include "rs_internal.cuh"

namespace {

constexpr int64_t STATIC_MAX_N = 65536;           // particles per call
constexpr int64_t STATIC_MAX_CELLS = 1 << 20;     // coarse cells of the neighbour table
constexpr int64_t STATIC_SORT_TILE = RS_SORT_TILE;  // keys per radix-sort tile
constexpr int64_t STATIC_SCAN_BYTES = 64 * 1024;

// byte size of each region, rounded to 256 so every region stays aligned
constexpr int64_t r256(int64_t b) { return (b + 255) / 256 * 256; }

constexpr int64_t SZ_STATUS = r256(sizeof(rs_dev_status));
constexpr int64_t SZ_K = r256(8 * STATIC_MAX_N);                       // sort keys (x2)
constexpr int64_t SZ_V = r256(4 * STATIC_MAX_N);                       // sort values (x2)
constexpr int64_t SZ_HIST = r256(4 * 256 * ((STATIC_MAX_N + STATIC_SORT_TILE - 1) / STATIC_SORT_TILE));
constexpr int64_t SZ_SCAN = r256(STATIC_SCAN_BYTES);
constexpr int64_t SZ_POS4 = r256(16 * STATIC_MAX_N);
constexpr int64_t SZ_MISC = r256(4 * (2 * STATIC_MAX_N + 8));
constexpr int64_t SZ_CELLOF = r256(4 * STATIC_MAX_N);
constexpr int64_t SZ_CELLSTART = r256(4 * (STATIC_MAX_N + 1));
constexpr int64_t SZ_CELLKEY = r256(8 * STATIC_MAX_N);
constexpr int64_t SZ_TABLE = r256(4 * STATIC_MAX_CELLS);
constexpr int64_t SZ_PARENT = r256(4 * STATIC_MAX_N);
constexpr int64_t SZ_ROOTMIN = r256(4 * STATIC_MAX_N);
constexpr int64_t SZ_OCC = r256(8 * STATIC_MAX_N);

constexpr int64_t STATIC_BYTES = SZ_STATUS + 2 * SZ_K + 2 * SZ_V + SZ_HIST + SZ_SCAN + SZ_POS4 + SZ_MISC +
                                 SZ_CELLOF + SZ_CELLSTART + SZ_CELLKEY + SZ_TABLE + SZ_PARENT + SZ_ROOTMIN +
                                 SZ_OCC;

// The fixed scratch of rs_fof3d_static (about 10 MB).
static __device__ __align__(256) unsigned char g_fof_scratch[STATIC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up
// once per device.
cudaError_t scratch_address(int device, void **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_fof_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

// Coarse cells of the grid rs_fof3d builds for (n, box, b), from the grid
// rule rs_fof3d itself uses, so the table size is checked before the call.
bool coarse_cells(int64_t n, double box, double b, int64_t *cells)
{
    const FofGridSize gs = fof_grid_size(n, box, b);
    if (!(gs.l > 0) || !(gs.gc < 2.0e6)) return false;
    *cells = (int64_t)gs.gc * (int64_t)gs.gc * (int64_t)gs.gc;
    return true;
}

}  // namespace

extern "C" rs_status rs_fof3d_static(const float *pos, int32_t stride, int64_t n, double box, double b,
                                     int32_t *labels, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!pos || !labels)) || (stride != 3 && stride != 4) || !(box > 0) || !(b > 0))
        return RS_ERR_INVALID_ARG;
    if (n > STATIC_MAX_N) return RS_ERR_TOO_LARGE;  // more particles than the fixed scratch holds
    if (n == 0) return RS_OK;
    int64_t cells = 0;
    if (!coarse_cells(n, box, b, &cells)) return RS_ERR_INVALID_ARG;
    if (cells > STATIC_MAX_CELLS) return RS_ERR_TOO_LARGE;  // the neighbour table would not fit

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= MAX_DEVICES) return RS_ERR_CUDA;
    void *base = nullptr;
    if (scratch_address(device, &base) != cudaSuccess) return RS_ERR_CUDA;

    // A host-side context whose workspace slots already point into the
    // scratch array at their full capacity, so rs_fof3d never has a reason to
    // allocate, and is marked fixed: should a slot ever be too small, the
    // call fails with RS_ERR_INTERNAL instead of allocating.  Its status words live in the scratch and on this stack.
    rs_ctx c;
    c.stream = (cudaStream_t)cuda_stream;
    c.device = device;
    c.fixed_ws = 1;  // a slot that would need more room fails instead of allocating
    if (cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return RS_ERR_CUDA;
    unsigned char *p = (unsigned char *)base;
    auto take = [&](int slot, int64_t bytes) {
        c.ws_ptr[slot] = p;
        c.ws_size[slot] = (size_t)bytes;
        p += bytes;
    };
    c.d_status = (rs_dev_status *)p;
    p += SZ_STATUS;
    take(WS_SORT_K0, SZ_K);
    take(WS_SORT_K1, SZ_K);
    take(WS_SORT_V0, SZ_V);
    take(WS_SORT_V1, SZ_V);
    take(WS_SORT_HIST, SZ_HIST);
    take(WS_SCAN_TMP, SZ_SCAN);
    take(WS_FOF_POS4, SZ_POS4);
    take(WS_FOF_MISC, SZ_MISC);
    take(WS_FOF_CELLOF, SZ_CELLOF);
    take(WS_FOF_CELLSTART, SZ_CELLSTART);
    take(WS_FOF_CELLKEY, SZ_CELLKEY);
    take(WS_FOF_TABLE, SZ_TABLE);
    take(WS_FOF_PARENT, SZ_PARENT);
    take(WS_FOF_ROOTMIN, SZ_ROOTMIN);
    take(WS_FOF_OCC, SZ_OCC);
    rs_dev_status h_status;
    int64_t h_scratch[64];
    c.h_status = &h_status;
    c.h_scratch = h_scratch;

    // the status word must start at zero; every other region is written
    // before it is read by rs_fof3d itself
    if (cudaMemsetAsync(c.d_status, 0, sizeof(rs_dev_status), c.stream) != cudaSuccess) return RS_ERR_CUDA;
    rs_status s = rs_fof3d(&c, pos, stride, n, box, b, labels, nullptr, nullptr);
    if (s != RS_OK) return s;
    // the device checks (out-of-range positions, bounded waits) report here
    return rs_sync_check(&c, "rs_fof3d_static");
}

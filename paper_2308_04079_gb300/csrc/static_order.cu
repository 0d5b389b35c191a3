// static_order.cu -- gs_depth_order_static: the depth ordering of the two-phase binning
// schedule (stable LSD radix sort of the Gaussians by fp32 depth bits, culled ones last) with
// every piece of scratch in one file-scope device array instead of the caller's workspace.
//
// Why it exists: some callers cannot allocate device memory at the point where they need the
// ordering.  A render loop that keeps several streams busy cannot call cudaMalloc / cudaFree
// there (cudaFree synchronises the device and cudaMalloc may), and a host that runs under a
// fixed device-memory budget, or without a caching allocator of its own, has no workspace to
// hand over for a one-off sort.  This entry point allocates nothing: the scratch below is
// part of the loaded module, its address is looked up once per device, and each call only
// clears the counters it needs and launches kernels.
//
// Limits and sharing: n <= GS_STATIC_ORDER_MAX_N.  The scratch is one per device and per
// process, so calls that overlap in time on the same device (two streams, two host threads)
// race on it and give undefined results; the caller must order them (same stream, or events).
//
// The paper has no counterpart: it sorts 64-bit (tile, depth) keys in one pass structure and
// has no separate depth ordering (App. C).
#include <mutex>

#include "gs_device.cuh"
#include "gs_kernels.h"

namespace gs {
namespace {

constexpr int kStaticMaxN = GS_STATIC_ORDER_MAX_N;
constexpr int kStaticRows = (kStaticMaxN + kSortTile - 1) / kSortTile;   // look-back rows per pass

// Scratch layout (each piece 256-byte aligned):
struct StaticScratch {
    uint32_t keys[2][kStaticMaxN];          // depth-key ping-pong
    uint32_t vals[2][kStaticMaxN];          // index ping-pong (the last pass writes the caller's order)
    uint32_t lookback[2][kStaticRows * 256];
    uint32_t hist[kDepthPasses][256];
    uint32_t counters[kDepthPasses];        // chunk-claim counters, one per pass
    uint32_t pad[64 - kDepthPasses];
};

static_assert(sizeof(StaticScratch) % 256 == 0, "scratch pieces stay 256-byte aligned");

// About 4.3 MB: 2 x 2 x 1 MB of keys and values, 2 x 64 KB of look-back rows, 4 KB of
// histograms and counters.
static __device__ __align__(256) unsigned char g_static_order_scratch[sizeof(StaticScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
StaticScratch* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.  The first
// lookup may load the module on that device, so the first call on each device must not be
// made while the stream is being captured.  The cache is keyed by device ordinal only: a
// cudaDeviceReset unloads the module and leaves the cached address stale (documented in gs.h:
// no further calls on a device after resetting it).
StaticScratch* scratch_address(int dev) {
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_order_scratch) != cudaSuccess) return nullptr;
        g_addr[dev] = static_cast<StaticScratch*>(p);
    }
    return g_addr[dev];
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_depth_order_static(int n, const float* depth, const int* radius, uint32_t* order,
                                           gs_device_status* status, cudaStream_t s) {
    if (n < 0 || n > kStaticMaxN || !status) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!depth || !radius || !order)) return GS_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GS_ERR_CUDA;
    StaticScratch* sc = scratch_address(dev);
    if (!sc) return GS_ERR_CUDA;
    // Start-at-zero state: the caller's status block (flags, visible count), the chunk-claim
    // counters and the digit histograms.  The first pass's look-back rows are zeroed by the
    // histogram kernel, every later pass's rows by the pass before it.
    if (cudaMemsetAsync(status, 0, sizeof(gs_device_status), s) != cudaSuccess) return GS_ERR_CUDA;
    if (n == 0) return GS_OK;
    if (cudaMemsetAsync(sc->hist, 0, sizeof(sc->hist) + sizeof(sc->counters), s) != cudaSuccess) return GS_ERR_CUDA;

    Multi<DepthHistArgs, 1> h;
    h.frames = 1;
    h.a[0] = DepthHistArgs{n, depth, radius, &sc->hist[0][0], sc->lookback[0], &status->num_visible};
    if (launch_depth_hist(h, s) != cudaSuccess) return GS_ERR_CUDA;
    const int chunks = (n + kSortTile - 1) / kSortTile;
    for (int p = 0; p < kDepthPasses; ++p) {
        const bool last = p + 1 == kDepthPasses;
        Multi<SortPassArgs<uint32_t>, 1> m;
        m.frames = 1;
        SortPassArgs<uint32_t>& a = m.a[0];
        a.keys_in = p == 0 ? nullptr : sc->keys[(p + 1) % 2];
        a.vals_in = p == 0 ? nullptr : sc->vals[(p + 1) % 2];
        a.depth_src = depth;
        a.radius_src = radius;
        a.keys_out = sc->keys[p % 2];
        a.vals_out = last ? order : sc->vals[p % 2];
        a.count_dev = nullptr;
        a.count_host = (uint32_t)n;
        a.shift = 8 * p;
        a.mask = 0xFFu;
        a.ballot_rank = 0;
        a.hist = sc->hist[p];
        a.lookback = sc->lookback[p % 2];
        a.lookback_next = last ? nullptr : sc->lookback[(p + 1) % 2];
        a.chunk_counter = &sc->counters[p];
        a.status = status;
        a.spin_limit = kSpinLimit;
        if (launch_onesweep(m, chunks, s) != cudaSuccess) return GS_ERR_CUDA;
    }
    return GS_OK;
}

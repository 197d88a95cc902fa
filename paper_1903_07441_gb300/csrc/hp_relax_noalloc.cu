// hp_relax_noalloc: the harmonic-field relaxation for callers that cannot
// allocate device memory.
//
// Some callers of this library may not call cudaMalloc at all: a real-time
// control loop that must not allocate after start-up (cudaMalloc can
// synchronise the device and its latency is unbounded), or a plug-in running
// inside a host application that owns every device allocation.  hp_relax needs
// a caller-provided workspace; this variant instead uses one file-scope device
// array, g_hp_noalloc_scratch, that lives as long as the library is loaded on
// each GPU that loads it.
//
// Set-up: the first call on a device (with that device current) asks the
// runtime for the array's device address once (cudaGetSymbolAddress) and
// caches it; host code never passes the array's name itself, which on the
// host is only a stand-in symbol.  Make that first call before any stream
// capture.  The kept address belongs to the device's context: after a
// cudaDeviceReset the caller must not use this entry point on that device
// again in the same process.
//
// The array is shared by every call on a device and keeps the previous call's
// contents; the solver clears everything that must start at zero (padding,
// reduction words) at the start of each call.  Calls whose GPU work overlaps
// (different streams, or different host threads) race on the array.
#include <mutex>

#include "common.cuh"

namespace tw {

constexpr size_t kNoAllocScratchBytes = HP_RELAX_NOALLOC_SCRATCH_BYTES;  // 9 MiB: up to 1024 x 1024 cells (870 x 870 with an error tolerance)
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_hp_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[kNoAllocMaxDevices];

// Device address of the scratch array on the current device (set-up on first use).
static int noalloc_scratch(void **out) {
    int dev = 0;
    TW_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return TW_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        TW_CUDA(cudaGetSymbolAddress(&p, g_hp_noalloc_scratch));
        if (!p || !ws_aligned(p)) return TW_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return TW_OK;
}

}  // namespace tw

using namespace tw;

extern "C" int hp_relax_noalloc(const tw_grid *g, const uint8_t *occ_dev, int gx, int gy, float *field_dev,
                                const hp_params *p, hp_stats *stats, void *stream) {
    if (!g || !p || (p->flags & HP_TIMING)) return TW_EINVAL;
    if (p->method != HP_RBSOR && p->method != HP_JACOBI) return TW_EINVAL;
    if (g->nx < 3 || g->ny < 3 || g->nx > 65535 || g->ny > 65535) return TW_EINVAL;
    const size_t need = hp_relax_workspace_size(g->nx, g->ny, p);
    if (need == 0 || need > kNoAllocScratchBytes) return TW_EWORKSPACE;  // grid too large for the array
    void *ws = nullptr;
    int e = noalloc_scratch(&ws);
    if (e) return e;
    // the host-driven convergence loop: instantiating the default CUDA graph could allocate
    hp_params q = *p;
    q.flags |= HP_HOST_LOOP;
    return hp_relax(g, occ_dev, gx, gy, field_dev, &q, stats, ws, kNoAllocScratchBytes, stream);
}

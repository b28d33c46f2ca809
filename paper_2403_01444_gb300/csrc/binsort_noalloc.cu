// gs_bin_sort_noalloc: tile binning + key sort for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// point where they bin: code running under an allocator that forbids new
// device allocations after start-up, real-time render loops that must not
// risk an allocation stall or an out-of-memory failure mid-frame, and
// plug-ins that only receive pre-sized buffers from a host application.
// For them this entry point uses a scratch buffer that the library itself
// declares at file scope in device memory, so the caller passes only inputs
// and outputs.
//
// The scratch is one static device array of kNoAllocScratchBytes (20 MiB);
// every GPU that loads this library holds it until the process exits.  It
// bounds the problem: n * V <= 131072 (view, Gaussian) entries and
// capacity <= 1048576 (Gaussian, tile) pairs, and in any case the scratch
// gs_bin_sort_workspace_size() reports for the call must fit in it.  Larger
// calls are rejected with GS_ERR_INVALID_ARG before anything is launched.
//
// All calls on a device share the one array and it keeps the last call's
// contents.  No part of it has to start at zero (every region is written
// before it is read within a call), so nothing is cleared.  Two calls whose
// work overlaps on the GPU (different streams without ordering, or different
// host threads) race on the array and give wrong results: serialise them.
//
// The first call on each device looks up the array's device address
// (cudaGetSymbolAddress, with that device current) and caches it; make that
// first call before any stream capture on the device.
#include <mutex>

#include "common.cuh"

namespace gs3 {

constexpr size_t kNoAllocScratchBytes = size_t(20) << 20;
constexpr int64_t kNoAllocMaxEntries = int64_t(1) << 17;
constexpr int64_t kNoAllocMaxPairs = int64_t(1) << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current.  In host code the array's name is only a
// host-side stand-in, never a device address.  The cached address is valid
// for the lifetime of the device's primary context: after cudaDeviceReset a
// process must not call gs_bin_sort_noalloc on that device again.
static void *scratch_address(int dev, gs_status &st)
{
    static std::mutex mu;
    static void *addr[kNoAllocMaxDevices] = {nullptr};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("gs_bin_sort_noalloc: device %d out of range", dev);
        st = GS_ERR_INVALID_ARG;
        return nullptr;
    }
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("gs_bin_sort_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                      cudaGetErrorString(e));
            st = GS_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = p;
    }
    st = GS_OK;
    return addr[dev];
}

}  // namespace gs3

using namespace gs3;

extern "C" gs_status gs_bin_sort_noalloc(const gs_projected *proj, int64_t n, int V, int W, int H,
                                         int bin, int64_t capacity, uint32_t *vals, uint32_t *ranges,
                                         uint64_t *keys, int64_t *d_count, int32_t *d_err,
                                         gs_stream stream)
{
    GS_REQUIRE(n >= 0 && V >= 1 && capacity >= 0, "gs_bin_sort_noalloc: bad n, V or capacity");
    // n is bounded before n * V is formed, so the product cannot wrap
    GS_REQUIRE(n <= kNoAllocMaxEntries / V,
               "gs_bin_sort_noalloc: n = %lld Gaussians x V = %d views exceeds the built-in limit "
               "of %lld entries", (long long)n, V, (long long)kNoAllocMaxEntries);
    GS_REQUIRE(capacity <= kNoAllocMaxPairs,
               "gs_bin_sort_noalloc: capacity %lld exceeds the built-in limit of %lld pairs",
               (long long)capacity, (long long)kNoAllocMaxPairs);
    size_t need = gs_bin_sort_workspace_size(n, V, W, H, capacity);
    GS_REQUIRE(need > 0 && need <= kNoAllocScratchBytes,
               "gs_bin_sort_noalloc: needs %zu bytes of scratch, the built-in buffer holds %zu",
               need, kNoAllocScratchBytes);
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("gs_bin_sort_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    gs_status st = GS_OK;
    void *ws = scratch_address(dev, st);
    if (st != GS_OK) return st;
    return gs_bin_sort(proj, n, V, W, H, bin, capacity, vals, ranges, keys, d_count, d_err, ws,
                       kNoAllocScratchBytes, stream);
}

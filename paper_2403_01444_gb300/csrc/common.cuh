// Shared device/host helpers of libgs3 (status handling, launch checks).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>

#include "../../include/gs3.h"

namespace gs3 {

// Thread-local message of the last failing call.
void set_error(const char *fmt, ...);

// Number of kernels this library has launched (all threads).
inline std::atomic<uint64_t> &launch_counter()
{
    static std::atomic<uint64_t> c{0};
    return c;
}
inline void note_launch() { launch_counter().fetch_add(1, std::memory_order_relaxed); }

inline gs_status launch_status(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return GS_ERR_CUDA;
    }
    return GS_OK;
}

#define GS_REQUIRE(cond, ...)                                                                     \
    do {                                                                                          \
        if (!(cond)) {                                                                            \
            ::gs3::set_error(__VA_ARGS__);                                                        \
            return GS_ERR_INVALID_ARG;                                                            \
        }                                                                                         \
    } while (0)

inline cudaStream_t as_stream(gs_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// Raise a kernel's dynamic shared-memory limit, except while the stream is
// being captured into a graph (the first, eager call has already done it).
inline void set_smem_limit(const void *kernel, int bytes, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cs == cudaStreamCaptureStatusNone)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline int tiles_x_of(int W) { return (W + GS_TILE - 1) / GS_TILE; }
inline int tiles_y_of(int H) { return (H + GS_TILE - 1) / GS_TILE; }
inline int bins_x_of(int W, int bin) { return (tiles_x_of(W) + bin - 1) / bin; }
inline int bins_y_of(int H, int bin) { return (tiles_y_of(H) + bin - 1) / bin; }

// Streaming multiprocessors of the current device (GB300: 2 dies x 76 = 152),
// queried once per device.  Grids are sized from it; workspaces that depend on
// a grid are sized for kMaxSMs so their size needs no device.
constexpr int kMaxSMs = 256;
inline int num_sms()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
        v = 152;
    v = v < kMaxSMs ? v : kMaxSMs;
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

// ------------------------------------------------------------------ device
// Tile rectangle of a footprint: x in [floor((u - r)/16), floor((u + r + 15)/16)),
// clamped to [0, tx].  floor(u - r) is taken exactly as floor of the
// round-down FP32 difference (exact while |floor(u - r)| < 2^24), so the
// result equals the real-number definition for any FP32 u.
__device__ __forceinline__ int floor_div16_of_sum(float u, float r_signed)
{
    float s = r_signed < 0.f ? __fsub_rd(u, -r_signed) : __fadd_rd(u, r_signed);
    s = fminf(fmaxf(s, -1.0e9f), 1.0e9f);
    int f = (int)floorf(s);
    return f >> 4;  // arithmetic shift: floor division by 16
}

__device__ __forceinline__ void tile_rect(float u, float v, int r, int tx, int ty, int &x0, int &y0,
                                          int &x1, int &y1)
{
    x0 = min(tx, max(0, floor_div16_of_sum(u, -(float)r)));
    x1 = min(tx, max(0, floor_div16_of_sum(u, (float)(r + GS_TILE - 1))));
    y0 = min(ty, max(0, floor_div16_of_sum(v, -(float)r)));
    y1 = min(ty, max(0, floor_div16_of_sum(v, (float)(r + GS_TILE - 1))));
}

// Bins of bin x bin tiles: the bin rectangle holding a footprint's tile
// rectangle (empty when the tile rectangle is empty).
__device__ __forceinline__ void bin_rect(float u, float v, int r, int tx, int ty, int bin, int &bx0,
                                         int &by0, int &bx1, int &by1)
{
    int x0, y0, x1, y1;
    tile_rect(u, v, r, tx, ty, x0, y0, x1, y1);
    if (x1 <= x0 || y1 <= y0) {
        bx0 = by0 = bx1 = by1 = 0;
        return;
    }
    bx0 = x0 / bin;
    by0 = y0 / bin;
    bx1 = (x1 - 1) / bin + 1;
    by1 = (y1 - 1) / bin + 1;
}

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

}  // namespace gs3

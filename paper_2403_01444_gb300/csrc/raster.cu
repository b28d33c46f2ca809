// Front-to-back alpha compositing (Section 3.2, Eq. 4) and its reverse.
// One 16x16 tile per block, one pixel per thread; the tile's depth-sorted
// records are staged through shared memory in batches.
#include "common.cuh"

namespace gs3 {

constexpr int RT = 256;        // threads = pixels per tile
constexpr int BWD_BATCH = 32;  // records per backward batch (one per lane)

struct RasterParams {
    const float2 *mean2d;
    const float4 *conic_op;
    const float *rgb;
    const uint32_t *vals;
    const uint2 *ranges;
    int64_t n;
    int V, W, H, tx, tiles;
    float bg0, bg1, bg2;
    float *img;
    float *T_final;
    int32_t *last;
    // backward
    const float *d_img;
    float *grads;
    float *d_opacity;
};

// power and alpha of one (pixel, Gaussian) pair.  Written with explicit
// roundings so the forward and the reverse pass take bit-identical decisions.
__device__ __forceinline__ float pair_power(float2 xy, float4 co, float px, float py, float &dx,
                                            float &dy)
{
    dx = __fsub_rn(px, xy.x);
    dy = __fsub_rn(py, xy.y);
    float q = fmaf(co.z, __fmul_rn(dy, dy), __fmul_rn(co.x, __fmul_rn(dx, dx)));
    return fmaf(-0.5f, q, -__fmul_rn(co.y, __fmul_rn(dx, dy)));
}

__device__ __forceinline__ float pair_alpha_raw(float4 co, float power)
{
    return __fmul_rn(co.w, __expf(power));
}

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaCap = 0.99f;
constexpr float kTEps = 1e-4f;

__global__ void __launch_bounds__(RT) raster_fwd_kernel(RasterParams p)
{
    __shared__ float2 s_xy[RT];
    __shared__ float4 s_co[RT];
    __shared__ float s_rgb[3][RT];
    const int tile = blockIdx.x, view = blockIdx.y;
    const int tid = threadIdx.x;
    const int px = (tile % p.tx) * 16 + (tid & 15);
    const int py = (tile / p.tx) * 16 + (tid >> 4);
    const bool inside = px < p.W && py < p.H;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const uint2 range = p.ranges[(int64_t)view * p.tiles + tile];
    const int total = (int)(range.y - range.x);
    const int64_t vb = (int64_t)view * p.n;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int last = 0;
    bool done = !inside;
    for (int base = 0; base < total; base += RT) {
        if (__syncthreads_count(done) == RT) break;
        int k = base + tid;
        if (k < total) {
            int64_t o = vb + p.vals[range.x + k];
            s_xy[tid] = p.mean2d[o];
            s_co[tid] = p.conic_op[o];
            s_rgb[0][tid] = p.rgb[3 * o];
            s_rgb[1][tid] = p.rgb[3 * o + 1];
            s_rgb[2][tid] = p.rgb[3 * o + 2];
        }
        __syncthreads();
        int cnt = min(RT, total - base);
        for (int j = 0; !done && j < cnt; ++j) {
            float dx, dy;
            float4 co = s_co[j];
            float power = pair_power(s_xy[j], co, pxf, pyf, dx, dy);
            if (power > 0.f) continue;
            float alpha = fminf(kAlphaCap, pair_alpha_raw(co, power));
            if (alpha < kAlphaMin) continue;
            float test_T = T * (1.f - alpha);
            if (test_T < kTEps) {
                done = true;
                break;
            }
            float w = alpha * T;
            C0 = fmaf(s_rgb[0][j], w, C0);
            C1 = fmaf(s_rgb[1][j], w, C1);
            C2 = fmaf(s_rgb[2][j], w, C2);
            T = test_T;
            last = base + j + 1;
        }
    }
    if (inside) {
        int64_t HW = (int64_t)p.H * p.W;
        int64_t pix = (int64_t)py * p.W + px;
        float *im = p.img + (int64_t)view * 3 * HW + pix;
        im[0] = fmaf(T, p.bg0, C0);
        im[HW] = fmaf(T, p.bg1, C1);
        im[2 * HW] = fmaf(T, p.bg2, C2);
        p.T_final[(int64_t)view * HW + pix] = T;
        p.last[(int64_t)view * HW + pix] = last;
    }
}

__global__ void __launch_bounds__(RT) raster_bwd_kernel(RasterParams p)
{
    __shared__ float2 s_xy[BWD_BATCH];
    __shared__ float4 s_co[BWD_BATCH];
    __shared__ float s_rgb[3][BWD_BATCH];
    __shared__ uint32_t s_g[BWD_BATCH];
    __shared__ float s_part[RT / 32][BWD_BATCH][9];
    __shared__ int s_max;
    const int tile = blockIdx.x, view = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int px = (tile % p.tx) * 16 + (tid & 15);
    const int py = (tile / p.tx) * 16 + (tid >> 4);
    const bool inside = px < p.W && py < p.H;
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const uint2 range = p.ranges[(int64_t)view * p.tiles + tile];
    const int64_t vb = (int64_t)view * p.n;
    const int64_t HW = (int64_t)p.H * p.W;
    const int64_t pix = (int64_t)py * p.W + px;
    int mylast = 0;
    float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
    if (inside) {
        mylast = p.last[(int64_t)view * HW + pix];
        T = p.T_final[(int64_t)view * HW + pix];
        const float *di = p.d_img + (int64_t)view * 3 * HW + pix;
        dC0 = di[0];
        dC1 = di[HW];
        dC2 = di[2 * HW];
    }
    float B0 = p.bg0, B1 = p.bg1, B2 = p.bg2;  // colour behind, normalised by T
    if (tid == 0) s_max = 0;
    __syncthreads();
    if (mylast > 0) atomicMax(&s_max, mylast);
    __syncthreads();
    const int maxlast = s_max;
    const bool want_op = p.d_opacity != nullptr;
    for (int hi = maxlast; hi > 0; hi -= BWD_BATCH) {
        const int lo = max(0, hi - BWD_BATCH);
        const int cnt = hi - lo;
        if (tid < cnt) {
            uint32_t g = p.vals[range.x + lo + tid];
            int64_t o = vb + g;
            s_g[tid] = g;
            s_xy[tid] = p.mean2d[o];
            s_co[tid] = p.conic_op[o];
            s_rgb[0][tid] = p.rgb[3 * o];
            s_rgb[1][tid] = p.rgb[3 * o + 1];
            s_rgb[2][tid] = p.rgb[3 * o + 2];
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            bool contrib = false;
            if (lo + j < mylast) {
                float dx, dy;
                float4 co = s_co[j];
                float power = pair_power(s_xy[j], co, pxf, pyf, dx, dy);
                if (power <= 0.f) {
                    float G = __expf(power);
                    float araw = __fmul_rn(co.w, G);
                    float alpha = fminf(kAlphaCap, araw);
                    if (alpha >= kAlphaMin) {
                        contrib = true;
                        T = T / (1.f - alpha);
                        float c0 = s_rgb[0][j], c1 = s_rgb[1][j], c2 = s_rgb[2][j];
                        float w = alpha * T;
                        v[5] = dC0 * w;
                        v[6] = dC1 * w;
                        v[7] = dC2 * w;
                        float dalpha = T * (dC0 * (c0 - B0) + dC1 * (c1 - B1) + dC2 * (c2 - B2));
                        B0 = fmaf(alpha, c0 - B0, B0);
                        B1 = fmaf(alpha, c1 - B1, B1);
                        B2 = fmaf(alpha, c2 - B2, B2);
                        if (araw < kAlphaCap) {
                            float dpow = dalpha * alpha;
                            v[0] = dpow * (co.x * dx + co.y * dy);
                            v[1] = dpow * (co.z * dy + co.y * dx);
                            v[2] = -0.5f * dpow * dx * dx;
                            v[3] = -dpow * dx * dy;
                            v[4] = -0.5f * dpow * dy * dy;
                            v[8] = dalpha * G;
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int k = 0; k < 9; ++k) v[k] = warp_sum(v[k]);
                if (lane == 0) {
#pragma unroll
                    for (int k = 0; k < 9; ++k) s_part[warp][j][k] = v[k];
                }
            } else if (lane == 0) {
#pragma unroll
                for (int k = 0; k < 9; ++k) s_part[warp][j][k] = 0.f;
            }
        }
        __syncthreads();
        // tile-wide sums: thread t -> (record t/2, half t%2), one float4 atomic
        if (tid < 2 * cnt) {
            int j = tid >> 1, h = (tid & 1) * 4;
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int w = 0; w < RT / 32; ++w) {
                s.x += s_part[w][j][h];
                s.y += s_part[w][j][h + 1];
                s.z += s_part[w][j][h + 2];
                s.w += s_part[w][j][h + 3];
            }
            if (s.x != 0.f || s.y != 0.f || s.z != 0.f || s.w != 0.f)
                atomicAdd(reinterpret_cast<float4 *>(p.grads + 8 * (vb + s_g[j]) + h), s);
        } else if (want_op && tid >= 64 && tid < 64 + cnt) {
            int j = tid - 64;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < RT / 32; ++w) s += s_part[w][j][8];
            if (s != 0.f) atomicAdd(p.d_opacity + vb + s_g[j], s);
        }
        __syncthreads();
    }
}

static gs_status fill(const gs_projected *proj, int64_t n, int V, int W, int H, const float *bg,
                      const uint32_t *vals, const uint32_t *ranges, RasterParams &p)
{
    GS_REQUIRE(proj && vals && ranges, "raster: null argument");
    GS_REQUIRE(n >= 0 && V >= 1 && V <= GS_MAX_VIEWS, "raster: bad n or V");
    GS_REQUIRE(W > 0 && H > 0 && W <= 16384 && H <= 16384, "raster: bad image size");
    GS_REQUIRE(aligned(proj->mean2d, 8) && aligned(proj->conic_opacity, 16) && aligned(ranges, 8),
               "raster: misaligned input");
    p.mean2d = reinterpret_cast<const float2 *>(proj->mean2d);
    p.conic_op = reinterpret_cast<const float4 *>(proj->conic_opacity);
    p.rgb = proj->rgb;
    p.vals = vals;
    p.ranges = reinterpret_cast<const uint2 *>(ranges);
    p.n = n;
    p.V = V;
    p.W = W;
    p.H = H;
    p.tx = tiles_x_of(W);
    p.tiles = p.tx * tiles_y_of(H);
    p.bg0 = bg ? bg[0] : 0.f;
    p.bg1 = bg ? bg[1] : 0.f;
    p.bg2 = bg ? bg[2] : 0.f;
    return GS_OK;
}

}  // namespace gs3

using namespace gs3;

extern "C" gs_status gs_raster_fwd(const gs_projected *proj, int64_t n, int V, int W, int H,
                                   const float *bg, const uint32_t *vals, const uint32_t *ranges,
                                   float *img, float *T_final, int32_t *last, gs_stream stream)
{
    RasterParams p{};
    gs_status st = fill(proj, n, V, W, H, bg, vals, ranges, p);
    if (st != GS_OK) return st;
    GS_REQUIRE(img && T_final && last, "gs_raster_fwd: null output");
    p.img = img;
    p.T_final = T_final;
    p.last = last;
    dim3 grid(p.tiles, V);
    note_launch();
    raster_fwd_kernel<<<grid, RT, 0, as_stream(stream)>>>(p);
    return launch_status("gs_raster_fwd");
}

extern "C" gs_status gs_raster_bwd(const gs_projected *proj, int64_t n, int V, int W, int H,
                                   const float *bg, const uint32_t *vals, const uint32_t *ranges,
                                   const float *T_final, const int32_t *last, const float *d_img,
                                   float *grads, float *d_opacity, gs_stream stream)
{
    RasterParams p{};
    gs_status st = fill(proj, n, V, W, H, bg, vals, ranges, p);
    if (st != GS_OK) return st;
    GS_REQUIRE(T_final && last && d_img && grads, "gs_raster_bwd: null argument");
    GS_REQUIRE(aligned(grads, 16), "gs_raster_bwd: grads must be 16-byte aligned");
    cudaStream_t s = as_stream(stream);
    cudaMemsetAsync(grads, 0, sizeof(float) * 8 * n * V, s);
    if (d_opacity) cudaMemsetAsync(d_opacity, 0, sizeof(float) * n * V, s);
    p.T_final = const_cast<float *>(T_final);
    p.last = const_cast<int32_t *>(last);
    p.d_img = d_img;
    p.grads = grads;
    p.d_opacity = d_opacity;
    dim3 grid(p.tiles, V);
    note_launch();
    raster_bwd_kernel<<<grid, RT, 0, s>>>(p);
    return launch_status("gs_raster_bwd");
}

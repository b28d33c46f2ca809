// Front-to-back alpha compositing (Section 3.2, Eq. 4) and its reverse.
// One 16x16 tile per block, one pixel per thread; the tile's depth-sorted
// records are staged through shared memory in batches.
#include "common.cuh"

namespace gs3 {

constexpr int RT = 128;         // threads per 16x16 tile: two pixels each, rows y and y + 8
constexpr int FWD_BATCH = 256;  // records staged per forward batch
constexpr int BWD_BATCH = 32;   // records per backward batch (one per lane)
constexpr int RWARPS = RT / 32;

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

// Front-to-back compositing state of one pixel.
struct PixFwd {
    float T, C0, C1, C2;
    int last;
    bool done;
};

__device__ __forceinline__ void blend_one(PixFwd &P, float2 xy, float4 co, const float *c, float pxf,
                                          float pyf, int pos)
{
    float dx, dy;
    float power = pair_power(xy, co, pxf, pyf, dx, dy);
    if (power > 0.f) return;
    float alpha = fminf(kAlphaCap, pair_alpha_raw(co, power));
    if (alpha < kAlphaMin) return;
    float test_T = P.T * (1.f - alpha);
    if (test_T < kTEps) {
        P.done = true;
        return;
    }
    float w = alpha * P.T;
    P.C0 = fmaf(c[0], w, P.C0);
    P.C1 = fmaf(c[1], w, P.C1);
    P.C2 = fmaf(c[2], w, P.C2);
    P.T = test_T;
    P.last = pos + 1;
}

__global__ void __launch_bounds__(RT) raster_fwd_kernel(RasterParams p)
{
    __shared__ float2 s_xy[FWD_BATCH];
    __shared__ float4 s_co[FWD_BATCH];
    __shared__ float s_rgb[FWD_BATCH][3];
    const int tile = blockIdx.x, view = blockIdx.y;
    const int tid = threadIdx.x;
    const int px = (tile % p.tx) * 16 + (tid & 15);
    const int py0 = (tile / p.tx) * 16 + (tid >> 4);
    const int py1 = py0 + 8;
    const float pxf = (float)px + 0.5f, pyf0 = (float)py0 + 0.5f, pyf1 = (float)py1 + 0.5f;
    const uint2 range = p.ranges[(int64_t)view * p.tiles + tile];
    const int total = (int)(range.y - range.x);
    const int64_t vb = (int64_t)view * p.n;
    PixFwd A{1.f, 0.f, 0.f, 0.f, 0, !(px < p.W && py0 < p.H)};
    PixFwd B{1.f, 0.f, 0.f, 0.f, 0, !(px < p.W && py1 < p.H)};
    for (int base = 0; base < total; base += FWD_BATCH) {
        if (__syncthreads_count(A.done && B.done) == RT) break;
#pragma unroll
        for (int h = 0; h < FWD_BATCH / RT; ++h) {
            int k = base + tid + h * RT;
            if (k < total) {
                int64_t o = vb + p.vals[range.x + k];
                int slot = tid + h * RT;
                s_xy[slot] = p.mean2d[o];
                s_co[slot] = p.conic_op[o];
                s_rgb[slot][0] = p.rgb[3 * o];
                s_rgb[slot][1] = p.rgb[3 * o + 1];
                s_rgb[slot][2] = p.rgb[3 * o + 2];
            }
        }
        __syncthreads();
        const int cnt = min(FWD_BATCH, total - base);
        for (int j = 0; j < cnt && !(A.done && B.done); ++j) {
            float2 xy = s_xy[j];
            float4 co = s_co[j];
            const float *c = s_rgb[j];
            if (!A.done) blend_one(A, xy, co, c, pxf, pyf0, base + j);
            if (!B.done) blend_one(B, xy, co, c, pxf, pyf1, base + j);
        }
    }
    const int64_t HW = (int64_t)p.H * p.W;
    if (px < p.W && py0 < p.H) {
        int64_t pix = (int64_t)py0 * p.W + px;
        float *im = p.img + (int64_t)view * 3 * HW + pix;
        im[0] = fmaf(A.T, p.bg0, A.C0);
        im[HW] = fmaf(A.T, p.bg1, A.C1);
        im[2 * HW] = fmaf(A.T, p.bg2, A.C2);
        p.T_final[(int64_t)view * HW + pix] = A.T;
        p.last[(int64_t)view * HW + pix] = A.last;
    }
    if (px < p.W && py1 < p.H) {
        int64_t pix = (int64_t)py1 * p.W + px;
        float *im = p.img + (int64_t)view * 3 * HW + pix;
        im[0] = fmaf(B.T, p.bg0, B.C0);
        im[HW] = fmaf(B.T, p.bg1, B.C1);
        im[2 * HW] = fmaf(B.T, p.bg2, B.C2);
        p.T_final[(int64_t)view * HW + pix] = B.T;
        p.last[(int64_t)view * HW + pix] = B.last;
    }
}

// Back-to-front state of one pixel.
struct PixBwd {
    int last;
    float T, dC0, dC1, dC2, B0, B1, B2;
};

template <bool WANT_OP>
__device__ __forceinline__ bool unblend_one(PixBwd &P, float2 xy, float4 co, const float *c,
                                            float pxf, float pyf, float *v)
{
    float dx, dy;
    float power = pair_power(xy, co, pxf, pyf, dx, dy);
    if (power > 0.f) return false;
    float G = __expf(power);
    float araw = __fmul_rn(co.w, G);
    float alpha = fminf(kAlphaCap, araw);
    if (alpha < kAlphaMin) return false;
    P.T = P.T / (1.f - alpha);
    float w = alpha * P.T;
    v[5] = fmaf(P.dC0, w, v[5]);
    v[6] = fmaf(P.dC1, w, v[6]);
    v[7] = fmaf(P.dC2, w, v[7]);
    float dalpha = P.T * (P.dC0 * (c[0] - P.B0) + P.dC1 * (c[1] - P.B1) + P.dC2 * (c[2] - P.B2));
    P.B0 = fmaf(alpha, c[0] - P.B0, P.B0);
    P.B1 = fmaf(alpha, c[1] - P.B1, P.B1);
    P.B2 = fmaf(alpha, c[2] - P.B2, P.B2);
    if (araw < kAlphaCap) {
        float dpow = dalpha * alpha;
        v[0] = fmaf(dpow, co.x * dx + co.y * dy, v[0]);
        v[1] = fmaf(dpow, co.z * dy + co.y * dx, v[1]);
        v[2] = fmaf(-0.5f * dpow, dx * dx, v[2]);
        v[3] = fmaf(-dpow, dx * dy, v[3]);
        v[4] = fmaf(-0.5f * dpow, dy * dy, v[4]);
        if (WANT_OP) v[8] = fmaf(dalpha, G, v[8]);
    }
    return true;
}

template <bool WANT_OP>
__global__ void __launch_bounds__(RT) raster_bwd_kernel(RasterParams p)
{
    constexpr int NV = WANT_OP ? 9 : 8;
    __shared__ float2 s_xy[BWD_BATCH];
    __shared__ float4 s_co[BWD_BATCH];
    __shared__ float s_rgb[BWD_BATCH][3];
    __shared__ uint32_t s_g[BWD_BATCH];
    __shared__ float s_part[RWARPS][BWD_BATCH][NV];
    __shared__ int s_max;
    const int tile = blockIdx.x, view = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int px = (tile % p.tx) * 16 + (tid & 15);
    const int py0 = (tile / p.tx) * 16 + (tid >> 4);
    const int py1 = py0 + 8;
    const float pxf = (float)px + 0.5f, pyf0 = (float)py0 + 0.5f, pyf1 = (float)py1 + 0.5f;
    const uint2 range = p.ranges[(int64_t)view * p.tiles + tile];
    const int64_t vb = (int64_t)view * p.n;
    const int64_t HW = (int64_t)p.H * p.W;
    PixBwd A{0, 1.f, 0.f, 0.f, 0.f, p.bg0, p.bg1, p.bg2};
    PixBwd B{0, 1.f, 0.f, 0.f, 0.f, p.bg0, p.bg1, p.bg2};
    if (px < p.W && py0 < p.H) {
        int64_t pix = (int64_t)view * HW + (int64_t)py0 * p.W + px;
        A.last = p.last[pix];
        A.T = p.T_final[pix];
        const float *di = p.d_img + (int64_t)view * 3 * HW + (int64_t)py0 * p.W + px;
        A.dC0 = di[0];
        A.dC1 = di[HW];
        A.dC2 = di[2 * HW];
    }
    if (px < p.W && py1 < p.H) {
        int64_t pix = (int64_t)view * HW + (int64_t)py1 * p.W + px;
        B.last = p.last[pix];
        B.T = p.T_final[pix];
        const float *di = p.d_img + (int64_t)view * 3 * HW + (int64_t)py1 * p.W + px;
        B.dC0 = di[0];
        B.dC1 = di[HW];
        B.dC2 = di[2 * HW];
    }
    if (tid == 0) s_max = 0;
    __syncthreads();
    const int mylast = max(A.last, B.last);
    if (mylast > 0) atomicMax(&s_max, mylast);
    __syncthreads();
    const int maxlast = s_max;
    for (int hi = maxlast; hi > 0; hi -= BWD_BATCH) {
        const int lo = max(0, hi - BWD_BATCH);
        const int cnt = hi - lo;
        if (tid < cnt) {
            uint32_t g = p.vals[range.x + lo + tid];
            int64_t o = vb + g;
            s_g[tid] = g;
            s_xy[tid] = p.mean2d[o];
            s_co[tid] = p.conic_op[o];
            s_rgb[tid][0] = p.rgb[3 * o];
            s_rgb[tid][1] = p.rgb[3 * o + 1];
            s_rgb[tid][2] = p.rgb[3 * o + 2];
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            float v[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] = 0.f;
            const int pos = lo + j;
            bool contrib = false;
            if (pos < mylast) {
                float2 xy = s_xy[j];
                float4 co = s_co[j];
                const float *c = s_rgb[j];
                if (pos < A.last) contrib |= unblend_one<WANT_OP>(A, xy, co, c, pxf, pyf0, v);
                if (pos < B.last) contrib |= unblend_one<WANT_OP>(B, xy, co, c, pxf, pyf1, v);
            }
            if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < NV; ++k) s_part[warp][j][k] = v[k];
            }
        }
        __syncthreads();
        // tile-wide sums: thread t -> (record t/2, half t%2), one float4 atomic
        if (tid < 2 * cnt) {
            int j = tid >> 1, h = (tid & 1) * 4;
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int w = 0; w < RWARPS; ++w) {
                s.x += s_part[w][j][h];
                s.y += s_part[w][j][h + 1];
                s.z += s_part[w][j][h + 2];
                s.w += s_part[w][j][h + 3];
            }
            if (s.x != 0.f || s.y != 0.f || s.z != 0.f || s.w != 0.f)
                atomicAdd(reinterpret_cast<float4 *>(p.grads + 8 * (vb + s_g[j]) + h), s);
        } else if (WANT_OP && tid >= 64 && tid < 64 + cnt) {
            int j = tid - 64;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < RWARPS; ++w) s += s_part[w][j][NV - 1];
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
    if (d_opacity)
        raster_bwd_kernel<true><<<grid, RT, 0, s>>>(p);
    else
        raster_bwd_kernel<false><<<grid, RT, 0, s>>>(p);
    return launch_status("gs_raster_bwd");
}

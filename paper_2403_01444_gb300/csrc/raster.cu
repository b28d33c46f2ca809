// Front-to-back alpha compositing (Section 3.2, Eq. 4) and its reverse.
// One 16x16 tile per 128-thread block, two vertically adjacent pixels per
// thread evaluated together in packed FP32; the tile's depth-sorted records
// are staged through shared memory in batches of 128.
#include "common.cuh"

namespace gs3 {

constexpr int NT = 128;          // threads per 16x16 tile: two pixels each
#ifndef BWD_CHUNK_RECORDS
#define BWD_CHUNK_RECORDS 32
#endif
constexpr int BWD_CHUNK = BWD_CHUNK_RECORDS;  // records per backward reduction chunk
#ifndef BWD_UNROLL
#define BWD_UNROLL 2
#endif
#ifndef FWD_UNROLL
#define FWD_UNROLL 8
#endif
constexpr int kBwdUnroll = BWD_UNROLL, kFwdUnroll = FWD_UNROLL;
// Optional minimum blocks per SM for the compositing kernels' launch bounds
// (0: none, the compiler's register choice).
#ifndef FWD_MIN_BLOCKS
#define FWD_MIN_BLOCKS 0
#endif
#ifndef BWD_MIN_BLOCKS
#define BWD_MIN_BLOCKS 0
#endif
#if FWD_MIN_BLOCKS > 0
#define FWD_BOUNDS __launch_bounds__(128, FWD_MIN_BLOCKS)
#else
#define FWD_BOUNDS __launch_bounds__(128)
#endif
#if BWD_MIN_BLOCKS > 0
#define BWD_BOUNDS __launch_bounds__(128, BWD_MIN_BLOCKS)
#else
#define BWD_BOUNDS __launch_bounds__(128)
#endif
#ifndef RASTER_WARP_BLOCKS
#define RASTER_WARP_BLOCKS 1     // 1: each warp owns a compact block of the tile; 0: rows
#endif

// Pixel of lane l in warp w, pixel k of the thread (k < ppt), for a 16x16
// tile split into 256 / (32 ppt) warps.  Blocks: a warp owns a compact
// rectangle (8x4 for one pixel per thread, 8x8 for two, 16x8 for four or
// more) whose pixels tend to share records and list ends; a thread's pixels
// are vertically adjacent.  Rows: thread t owns column t % 16 of rows
// t / 16 + k * (16 / ppt).
__device__ __forceinline__ void tile_pixel(int tid, int ppt, int k, int &x, int &y)
{
    if (RASTER_WARP_BLOCKS) {
        const int w = tid >> 5, l = tid & 31;
        const int rw = ppt >= 4 ? 16 : 8;         // warp rectangle width
        const int wpr = 16 / rw;                  // warps per tile row
        const int rows = (32 / rw) * ppt;         // warp rectangle height
        x = (w % wpr) * rw + l % rw;
        y = (w / wpr) * rows + (l / rw) * ppt + k;
    } else {
        x = tid & 15;
        y = (tid >> 4) + k * (16 / ppt);
    }
}

struct RasterParams {
    const float2 *mean2d;
    const float4 *conic_op;
    const float *rgb;
    const int32_t *radius;
    const uint32_t *vals;
    const uint2 *ranges;
    int64_t n;
    int V, W, H, tx, ty, bin, bins_x, bins;
    float bg0, bg1, bg2;
    float *img;
    float *T_final;
    int32_t *last;
    // backward
    const float *d_img;
    float *grads;
    float *d_opacity;
    unsigned long long *stats;  // optional: [tested, contributing] (pixel, Gaussian) pairs
    // optional per-tile lists of staged records (Gaussian, list position):
    // written by the forward, read by the reverse
    uint2 *tl_rec;
    int32_t *tl_cnt;
    int tl_cap;
};

// Add this thread's pair counts to the optional statistics words.
__device__ __forceinline__ void flush_stats(unsigned long long *stats, uint32_t tested,
                                            uint32_t contrib)
{
    if (!stats) return;
    unsigned long long a = tested, b = contrib;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(stats, a);
        atomicAdd(stats + 1, b);
    }
}

// power of one record at the two pixels (px, py.x) and (px, py.y) of a
// column, -0.5 (A dx^2 + C dy^2) - B dx dy, with explicit roundings so that
// the forward and the reverse pass take bit-identical decisions; the offset
// monomials dx^2, dx dy, dy^2 are returned for the reverse pass.  The
// row-dependent terms go two per packed instruction.
__device__ __forceinline__ float2 pair_power2(float2 xy, float4 co, float px, float2 py, float &dx,
                                              float2 &dy, float &dxx, float2 &dxy, float2 &dyy)
{
    dx = __fsub_rn(px, xy.x);
    dy = make_float2(__fsub_rn(py.x, xy.y), __fsub_rn(py.y, xy.y));
    dxx = __fmul_rn(dx, dx);
    dxy = __fmul2_rn(make_float2(dx, dx), dy);
    dyy = __fmul2_rn(dy, dy);
    const float axx = __fmul_rn(co.x, dxx);
    const float2 q = __ffma2_rn(make_float2(co.z, co.z), dyy, make_float2(axx, axx));
    const float2 nb = __fmul2_rn(make_float2(-co.y, -co.y), dxy);   // -(B dx dy), exact negation
    return __ffma2_rn(make_float2(-0.5f, -0.5f), q, nb);
}

#ifndef RASTER_LOG2_CONIC
#define RASTER_LOG2_CONIC 1
#endif
// With RASTER_LOG2_CONIC the staged conic is scaled by log2(e) (scale_conic),
// so pair_power yields the power in base-2 units and G = 2^power comes from
// one ex2.approx; G, alpha and dL/dpower keep their natural-unit meaning.
// moments_to_grads takes the unscaled conic (unscale_conic).
constexpr float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;

__device__ __forceinline__ float4 scale_conic(float4 co)
{
    return RASTER_LOG2_CONIC ? make_float4(co.x * kLog2e, co.y * kLog2e, co.z * kLog2e, co.w) : co;
}

__device__ __forceinline__ float4 unscale_conic(float4 co)
{
    return RASTER_LOG2_CONIC ? make_float4(co.x * kLn2, co.y * kLn2, co.z * kLn2, co.w) : co;
}

// G = exp(power) for a power from pair_power on a staged conic.
__device__ __forceinline__ float pair_gauss(float power)
{
#if RASTER_LOG2_CONIC
    float g;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(g) : "f"(power));
    return g;
#else
    return __expf(power);
#endif
}

// alpha >= 1/255 (Eq. 4's skip) is tested as power >= pmin on the base-2
// power, pmin = -log2(255 o) staged with the record: forward and reverse take
// the same decision, which differs from the test on alpha only within the
// rounding of the exponential
constexpr float kAlphaCap = 0.99f;
constexpr float kTEps = 1e-4f;

// Can record (m, co) reach alpha >= 1/255 at some pixel centre of tile
// (tx_t, ty_t)?  alpha = o exp(-q/2) with q = A dx^2 + 2B dx dy + C dy^2, so
// it needs q <= 2 ln(255 o) somewhere in the tile.  The minimum of the convex
// q over the tile's rectangle of pixel centres is 0 when the mean lies inside,
// else it is on an edge, where q is a 1-D quadratic minimised in closed form.
// A margin of 0.01 in q (far above FP32 rounding) keeps the test
// conservative: a dropped record is one every pixel of the tile would skip,
// so images, gradients and list positions are unchanged.
__device__ __forceinline__ bool ellipse_hits_tile(float2 m, float4 co, int tx_t, int ty_t)
{
    if (!(co.w * 255.f >= 1.f)) return false;
    const float tau = 2.f * __logf(255.f * co.w) + 0.01f;
    const float xa = (float)(tx_t * 16) + 0.5f - m.x, xb = xa + 15.f;
    const float ya = (float)(ty_t * 16) + 0.5f - m.y, yb = ya + 15.f;
    if (xa <= 0.f && xb >= 0.f && ya <= 0.f && yb >= 0.f) return true;
    const float A = co.x, B = co.y, C = co.z;
    // the 1-D minimisers need not be exact: q at any point of an edge bounds
    // its minimum from above, and a minimiser off by a rounding moves q by a
    // second-order amount, far inside the margin
    const float bA = B * __frcp_rn(A), bC = B * __frcp_rn(C);
    auto qx = [&](float dx) {  // min over dy in [ya, yb] at fixed dx
        float dy = fminf(fmaxf(-bC * dx, ya), yb);
        return A * dx * dx + 2.f * B * dx * dy + C * dy * dy;
    };
    auto qy = [&](float dy) {  // min over dx in [xa, xb] at fixed dy
        float dx = fminf(fmaxf(-bA * dy, xa), xb);
        return A * dx * dx + 2.f * B * dx * dy + C * dy * dy;
    };
    float q = fminf(fminf(qx(xa), qx(xb)), fminf(qy(ya), qy(yb)));
    return q <= tau;
}

// Does record o belong to tile (tx_t, ty_t)'s list (its tile rectangle holds
// the tile; implied when bins are single tiles) and can it contribute there?
template <bool BINNED>
__device__ __forceinline__ bool keep_record(const RasterParams &p, int64_t o, int tx_t, int ty_t,
                                            float2 &m, float4 &co)
{
    m = p.mean2d[o];
    co = p.conic_op[o];
    if (BINNED) {
        int r = p.radius[o];
        if (r <= 0) return false;
        int x0, y0, x1, y1;
        tile_rect(m.x, m.y, r, p.tx, p.ty, x0, y0, x1, y1);
        if (!(tx_t >= x0 && tx_t < x1 && ty_t >= y0 && ty_t < y1)) return false;
    }
    return ellipse_hits_tile(m, co, tx_t, ty_t);
}

// Block-wide stream compaction, order preserving: returns this thread's slot
// (or -1) and the number kept.
template <int THREADS>
__device__ __forceinline__ int compact_slot(bool keep, int *s_wcnt, int &count)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned b = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) s_wcnt[warp] = __popc(b);
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) {
        int c = s_wcnt[w];
        off += w < warp ? c : 0;
        tot += c;
    }
    count = tot;
    return keep ? off + __popc(b & ((1u << lane) - 1u)) : -1;
}

// Forward with two vertically adjacent pixels per thread (128 threads per
// tile): the record loads and the column offset are shared, and the pair of
// pixels is evaluated in packed FP32 (quadratic forms, alpha, transmittance,
// colour), two lanes of a register pair per instruction.  The arithmetic of an
// added pixel is the scalar one, rounding for rounding.
template <bool BINNED, bool STATS>
__global__ void FWD_BOUNDS raster_fwd2_kernel(RasterParams p)
{
    __shared__ float4 s_xy[NT];
    __shared__ float4 s_co[NT];
    __shared__ float4 s_rgbk[NT];  // colour and (bit pattern of) the list position
    __shared__ int s_wcnt[NT / 32];
    const int tile = blockIdx.x, view = blockIdx.y;
    const int tid = threadIdx.x;
    const int tx_t = tile % p.tx, ty_t = tile / p.tx;
    int px, py0;
    tile_pixel(tid, 2, 0, px, py0);
    px += tx_t * 16;
    py0 += ty_t * 16;
    const bool in0 = px < p.W && py0 < p.H, in1 = px < p.W && py0 + 1 < p.H;
    const float pxf = (float)px + 0.5f;
    const float2 pyf = make_float2((float)py0 + 0.5f, (float)py0 + 1.5f);
    const int binid = (ty_t / p.bin) * p.bins_x + tx_t / p.bin;
    const uint2 range = p.ranges[(int64_t)view * p.bins + binid];
    const int total = (int)(range.y - range.x);
    const int64_t vb = (int64_t)view * p.n;
    float T[2] = {1.f, 1.f}, C0[2] = {0.f, 0.f}, C1[2] = {0.f, 0.f}, C2[2] = {0.f, 0.f};
    int last[2] = {0, 0};
    bool done[2] = {!in0, !in1};
    uint32_t n_tested = 0, n_contrib = 0;
    const int64_t tg = (int64_t)view * gridDim.x + tile;  // the tile's list
    int staged = 0;
    // the last batch's first list index, and how far into it this thread's
    // pixels went (all of it unless both stopped)
    int staged_prev = 0, jlast = 0;
    __shared__ int s_jmax;
    if (tid == 0) s_jmax = 0;
    for (int base = 0; base < total; base += NT) {
        if (__syncthreads_count(done[0] && done[1]) == NT) break;
        const int k = base + tid;
        int64_t o = 0;
        uint32_t g = 0;
        bool keep = false;
        float2 m;
        float4 co;
        if (k < total) {
            g = p.vals[range.x + k];
            o = vb + g;
            keep = keep_record<BINNED>(p, o, tx_t, ty_t, m, co);
        }
        int cnt;
        const int slot = compact_slot<NT>(keep, s_wcnt, cnt);
        if (slot >= 0 && p.tl_rec && staged + slot < p.tl_cap)
            p.tl_rec[tg * p.tl_cap + staged + slot] = make_uint2(g, (uint32_t)k);
        staged_prev = staged;
        staged += cnt;
        jlast = done[0] && done[1] ? 0 : cnt;
        if (slot >= 0) {
            s_xy[slot] = make_float4(m.x, m.y, -__log2f(255.f * co.w), 0.f);
            s_co[slot] = scale_conic(co);
            s_rgbk[slot] = make_float4(p.rgb[3 * o], p.rgb[3 * o + 1], p.rgb[3 * o + 2],
                                       __int_as_float(k));
        }
        __syncthreads();
#pragma unroll kFwdUnroll
        for (int j = 0; !(done[0] && done[1]) && j < cnt; ++j) {
            const float4 cj = s_co[j];
            const float4 xyp = s_xy[j];
            float dx, dxx;
            float2 dy, dxy, dyy;
            const float2 pw = pair_power2(make_float2(xyp.x, xyp.y), cj, pxf, pyf, dx, dy, dxx, dxy, dyy);
            const bool t0 = !done[0] && pw.x <= 0.f && pw.x >= xyp.z;   // pixel takes part
            const bool t1 = !done[1] && pw.y <= 0.f && pw.y >= xyp.z;
            if (STATS) n_tested += !done[0] + !done[1];
            if (!(t0 || t1)) continue;
            // a pixel that does not take part has its power masked to -inf:
            // G = 0, alpha = 0 and its transmittance stays as it is (T * 1)
            const float g0 = pair_gauss(t0 ? pw.x : -INFINITY), g1 = pair_gauss(t1 ? pw.y : -INFINITY);
            const float2 araw = __fmul2_rn(make_float2(cj.w, cj.w), make_float2(g0, g1));
            float2 alpha = make_float2(fminf(kAlphaCap, araw.x), fminf(kAlphaCap, araw.y));
            const float2 om = __ffma2_rn(alpha, make_float2(-1.f, -1.f), make_float2(1.f, 1.f));
            const float2 Tv = make_float2(T[0], T[1]);
            float2 tT = __fmul2_rn(Tv, om);
            bool add0 = t0, add1 = t1;
            if (tT.x < kTEps || tT.y < kTEps) {
                // the pixel stops before this Gaussian (T stays >= 1e-4 otherwise,
                // so only a pixel that takes part can get here)
                const bool stop0 = tT.x < kTEps, stop1 = tT.y < kTEps;
                done[0] |= stop0;
                done[1] |= stop1;
                add0 = add0 && !stop0;
                add1 = add1 && !stop1;
                if (stop0) { alpha.x = 0.f; tT.x = Tv.x; }
                if (stop1) { alpha.y = 0.f; tT.y = Tv.y; }
                if (done[0] && done[1]) jlast = j + 1;
            }
            const float2 w = __fmul2_rn(alpha, Tv);
            const float4 ck = s_rgbk[j];
            const float2 c0 = __ffma2_rn(make_float2(ck.x, ck.x), w, make_float2(C0[0], C0[1]));
            const float2 c1 = __ffma2_rn(make_float2(ck.y, ck.y), w, make_float2(C1[0], C1[1]));
            const float2 c2 = __ffma2_rn(make_float2(ck.z, ck.z), w, make_float2(C2[0], C2[1]));
            C0[0] = c0.x; C0[1] = c0.y;
            C1[0] = c1.x; C1[1] = c1.y;
            C2[0] = c2.x; C2[1] = c2.y;
            T[0] = tT.x;
            T[1] = tT.y;
            const int kk = __float_as_int(ck.w) + 1;
            last[0] = add0 ? kk : last[0];
            last[1] = add1 ? kk : last[1];
            if (STATS) n_contrib += add0 + add1;
        }
    }
    if (STATS) flush_stats(p.stats, n_tested, n_contrib);
    if (p.tl_rec) {
        // records of the last batch past every thread's stop took part at no
        // pixel (their positions are at or past every pixel's last): the list
        // ends before them
        if (jlast > 0) atomicMax(&s_jmax, jlast);
        __syncthreads();
        if (tid == 0) {
            const int listed = staged_prev + s_jmax;
            p.tl_cnt[tg] = listed <= p.tl_cap ? listed : -1;
        }
    }
    const int64_t HW = (int64_t)p.H * p.W;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (!(q == 0 ? in0 : in1)) continue;
        const int64_t pix = (int64_t)(py0 + q) * p.W + px;
        float *im = p.img + (int64_t)view * 3 * HW + pix;
        im[0] = fmaf(T[q], p.bg0, C0[q]);
        im[HW] = fmaf(T[q], p.bg1, C1[q]);
        im[2 * HW] = fmaf(T[q], p.bg2, C2[q]);
        p.T_final[(int64_t)view * HW + pix] = T[q];
        p.last[(int64_t)view * HW + pix] = last[q];
    }
}

// Sum 8 per-lane values over the warp with 9 shuffles: each butterfly stage
// hands half of the remaining values to the partner lane.  Lane l returns the
// warp total of value index 4*bit4(l) + 2*bit3(l) + bit2(l) = l >> 2.  With
// FULL false the last two stages are left out (7 shuffles) and lane l returns
// the sum of that value over the 8 lanes that share l & 3: the warp total is
// the sum of lanes 4 (l >> 2) .. 4 (l >> 2) + 3.
template <bool FULL = true>
__device__ __forceinline__ float warp_reduce8(const float *v)
{
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float send = b4 ? v[i] : v[i + 4];
        float keep = b4 ? v[i + 4] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float send = b3 ? a[i] : a[i + 2];
        float keep = b3 ? a[i + 2] : a[i];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float send = b2 ? b[0] : b[1];
    float c = (b2 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
    if (FULL) {
        c += __shfl_xor_sync(0xffffffffu, c, 2);
        c += __shfl_xor_sync(0xffffffffu, c, 1);
    }
    return c;
}

// Record gradients from the tile sums of the moments: with power =
// -0.5 (A dx^2 + C dy^2) - B dx dy and dx = px - u,
//   dL/du = A S_x + B S_y,  dL/dv = C S_y + B S_x,
//   dL/dA = -S_xx / 2,  dL/dB = -S_xy,  dL/dC = -S_yy / 2,
// S_. = sum of dL/dpower times the offsets' monomials.  h = 0 holds
// (S_x, S_y, S_xx, S_xy), h = 1 holds (S_yy, r, g, b).
__device__ __forceinline__ float4 moments_to_grads(float4 s, float4 co, int h)
{
    if (h == 0)
        return make_float4(fmaf(co.x, s.x, co.y * s.y), fmaf(co.z, s.y, co.y * s.x), -0.5f * s.z, -s.w);
    return make_float4(-0.5f * s.x, s.y, s.z, s.w);
}

// Reverse with the thread's two vertically adjacent pixels evaluated together
// in packed FP32 (two lanes of a register pair per instruction).  A pixel
// that does not take part in a record (past its list end, or the record's
// power outside [pmin, 0]) gets alpha = 0, which leaves its transmittance,
// its colour-behind term and the sums exactly as they are.
struct PixBwd2 {
    int last0, last1;
    float2 T, dC0, dC1, dC2, S;
};

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

template <bool WANT_OP, bool STATS>
__device__ __forceinline__ bool unblend_pair(PixBwd2 &P, int pos, float4 co, float4 c, float2 pw, float pmin,
                                             float dx, float2 dy, float dxx, float2 dxy, float2 dyy,
                                             float *v, uint32_t &n_contrib)
{
    const bool in0 = pos < P.last0 && pw.x <= 0.f && pw.x >= pmin;
    const bool in1 = pos < P.last1 && pw.y <= 0.f && pw.y >= pmin;
    if (!(in0 || in1)) return false;
    if (STATS) n_contrib += (uint32_t)in0 + (uint32_t)in1;
    const float g0 = in0 ? pair_gauss(pw.x) : 0.f, g1 = in1 ? pair_gauss(pw.y) : 0.f;
    const float2 araw = __fmul2_rn(f2(co.w), make_float2(g0, g1));
    const float2 alpha = make_float2(fminf(kAlphaCap, araw.x), fminf(kAlphaCap, araw.y));
    const float2 om = __ffma2_rn(alpha, f2(-1.f), f2(1.f));   // 1 - alpha
    P.T = __fmul2_rn(P.T, make_float2(in0 ? rcp_approx(om.x) : 1.f, in1 ? rcp_approx(om.y) : 1.f));
    const float2 w = __fmul2_rn(alpha, P.T);
    const float2 c0 = __fmul2_rn(P.dC0, w), c1 = __fmul2_rn(P.dC1, w), c2 = __fmul2_rn(P.dC2, w);
    v[5] = c0.x + c0.y;
    v[6] = c1.x + c1.y;
    v[7] = c2.x + c2.y;
    float2 t = __fmul2_rn(P.dC0, f2(c.x));
    t = __ffma2_rn(P.dC1, f2(c.y), t);
    t = __ffma2_rn(P.dC2, f2(c.z), t);
    const float2 diff = __ffma2_rn(P.S, f2(-1.f), t);          // dC . c - S
    const float2 dalpha = __fmul2_rn(P.T, diff);
    P.S = __ffma2_rn(alpha, diff, P.S);
    // moments of dL/dpower over the pair offsets (no gradient through a capped alpha)
    float2 dpow = __fmul2_rn(dalpha, alpha);
    if (!(araw.x < kAlphaCap)) dpow.x = 0.f;
    if (!(araw.y < kAlphaCap)) dpow.y = 0.f;
    const float sd = dpow.x + dpow.y;
    v[0] = sd * dx;
    v[2] = sd * dxx;
    const float2 m1 = __fmul2_rn(dpow, dy), m3 = __fmul2_rn(dpow, dxy), m4 = __fmul2_rn(dpow, dyy);
    v[1] = m1.x + m1.y;
    v[3] = m3.x + m3.y;
    v[4] = m4.x + m4.y;
    if (WANT_OP) {
        const float2 gm = make_float2(araw.x < kAlphaCap ? g0 : 0.f, araw.y < kAlphaCap ? g1 : 0.f);
        const float2 op = __fmul2_rn(dalpha, gm);
        v[8] = op.x + op.y;
    }
    return true;
}

template <bool WANT_OP, bool BINNED, bool STATS>
__global__ void BWD_BOUNDS raster_bwd2_kernel(RasterParams p)
{
    constexpr int NW = NT / 32;
    constexpr int NV = WANT_OP ? 9 : 8;
    __shared__ float4 s_xy[NT];
    __shared__ float4 s_co[NT];
    __shared__ float4 s_rgbk[NT];  // colour and (bit pattern of) the list position
    __shared__ uint32_t s_g[NT];
    __shared__ int s_wcnt[NW];
    __shared__ float4 s_part[NW][BWD_CHUNK][8];
    __shared__ float s_pop[WANT_OP ? NW : 1][BWD_CHUNK];
    __shared__ int s_max;
    const int tile = blockIdx.x, view = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx_t = tile % p.tx, ty_t = tile / p.tx;
    int px, py0;
    tile_pixel(tid, 2, 0, px, py0);
    px += tx_t * 16;
    py0 += ty_t * 16;
    const float pxf = (float)px + 0.5f;
    const float2 pyf = make_float2((float)py0 + 0.5f, (float)py0 + 1.5f);
    const int binid = (ty_t / p.bin) * p.bins_x + tx_t / p.bin;
    const uint2 range = p.ranges[(int64_t)view * p.bins + binid];
    const int64_t vb = (int64_t)view * p.n;
    const int64_t HW = (int64_t)p.H * p.W;
    PixBwd2 P;
    P.last0 = P.last1 = 0;
    float Tq[2] = {1.f, 1.f}, d0[2] = {0.f, 0.f}, d1[2] = {0.f, 0.f}, d2[2] = {0.f, 0.f}, Sq[2] = {0.f, 0.f};
    int lq[2] = {0, 0};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int py = py0 + k;
        if (px < p.W && py < p.H) {
            int64_t pix = (int64_t)view * HW + (int64_t)py * p.W + px;
            lq[k] = p.last[pix];
            Tq[k] = p.T_final[pix];
            const float *di = p.d_img + (int64_t)view * 3 * HW + (int64_t)py * p.W + px;
            d0[k] = di[0];
            d1[k] = di[HW];
            d2[k] = di[2 * HW];
            Sq[k] = fmaf(d2[k], p.bg2, fmaf(d1[k], p.bg1, d0[k] * p.bg0));
        }
    }
    P.last0 = lq[0];
    P.last1 = lq[1];
    P.T = make_float2(Tq[0], Tq[1]);
    P.dC0 = make_float2(d0[0], d0[1]);
    P.dC1 = make_float2(d1[0], d1[1]);
    P.dC2 = make_float2(d2[0], d2[1]);
    P.S = make_float2(Sq[0], Sq[1]);
    const int mylast = max(lq[0], lq[1]);
    if (tid == 0) s_max = 0;
    __syncthreads();
    if (mylast > 0) atomicMax(&s_max, mylast);
    __syncthreads();
    const int maxlast = s_max;
    uint32_t n_tested = 0, n_contrib = 0;
    // with the forward's list of the tile, its records are staged straight
    // from it (list order is position order; the few past maxlast are
    // skipped by the position test); otherwise the bin's list is tested again
    const int64_t tg = (int64_t)view * gridDim.x + tile;
    const int listed = p.tl_rec ? p.tl_cnt[tg] : -1;
    for (int hi = listed >= 0 ? listed : maxlast; hi > 0; hi -= NT) {
        const int lo = max(0, hi - NT);
        int64_t o = 0;
        uint32_t g = 0;
        int k = 0;
        bool keep = false;
        float2 m;
        float4 co;
        int cnt, slot;
        if (listed >= 0) {
            if (lo + tid < hi) {
                const uint2 e = p.tl_rec[tg * p.tl_cap + lo + tid];
                g = e.x;
                k = (int)e.y;
                o = vb + g;
                m = p.mean2d[o];
                co = p.conic_op[o];
                keep = true;
            }
            cnt = hi - lo;
            slot = keep ? tid : -1;
        } else {
            k = lo + tid;
            if (k < hi) {
                g = p.vals[range.x + k];
                o = vb + g;
                keep = keep_record<BINNED>(p, o, tx_t, ty_t, m, co);
            }
            slot = compact_slot<NT>(keep, s_wcnt, cnt);
        }
        if (slot >= 0) {
            s_g[slot] = g;
            s_xy[slot] = make_float4(m.x, m.y, -__log2f(255.f * co.w), 0.f);
            s_co[slot] = scale_conic(co);
            s_rgbk[slot] = make_float4(p.rgb[3 * o], p.rgb[3 * o + 1], p.rgb[3 * o + 2],
                                       __int_as_float(k));
        }
        __syncthreads();
        for (int chi = cnt; chi > 0; chi -= BWD_CHUNK) {
            const int clo = max(0, chi - BWD_CHUNK);
#pragma unroll kBwdUnroll
            for (int j = chi - 1; j >= clo; --j) {
                float v[NV];
                const float4 c = s_rgbk[j];
                const int pos = __float_as_int(c.w);
                bool contrib = false;
                if (pos < mylast) {
                    const float4 xyp = s_xy[j];
                    const float4 cc = s_co[j];
                    float dx, dxx;
                    float2 dy, dxy, dyy;
                    const float2 pw = pair_power2(make_float2(xyp.x, xyp.y), cc, pxf, pyf, dx, dy, dxx, dxy, dyy);
                    if (STATS) n_tested += (pos < P.last0) + (pos < P.last1);
                    contrib = unblend_pair<WANT_OP, STATS>(P, pos, cc, c, pw, xyp.z, dx, dy, dxx, dxy,
                                                           dyy, v, n_contrib);
                }
                if (!contrib) {
#pragma unroll
                    for (int q = 0; q < NV; ++q) v[q] = 0.f;
                }
                float *part = reinterpret_cast<float *>(&s_part[warp][j - clo][0]);
                if (__any_sync(0xffffffffu, contrib)) {
                    part[lane] = warp_reduce8<false>(v);
                    if (WANT_OP) {
                        float ro = warp_sum(v[NV - 1]);
                        if (lane == 0) s_pop[warp][j - clo] = ro;
                    }
                } else {
                    part[lane] = 0.f;
                    if (WANT_OP && lane == 0) s_pop[warp][j - clo] = 0.f;
                }
            }
            __syncthreads();
            const int ccnt = chi - clo;
            if (tid < 4 * ccnt) {
                // four threads a record, two moments each
                const int j = tid >> 2, q = (tid & 3) * 2;
                float2 sum = make_float2(0.f, 0.f);
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const float4 a = s_part[w][j][q], b = s_part[w][j][q + 1];
                    sum.x += (a.x + a.y) + (a.z + a.w);
                    sum.y += (b.x + b.y) + (b.z + b.w);
                }
                if (sum.x != 0.f || sum.y != 0.f) {
                    float2 gq;
                    if (q == 0) {
                        const float4 co = unscale_conic(s_co[clo + j]);
                        gq = make_float2(fmaf(co.x, sum.x, co.y * sum.y), fmaf(co.z, sum.y, co.y * sum.x));
                    } else if (q == 2) {
                        gq = make_float2(-0.5f * sum.x, -sum.y);
                    } else if (q == 4) {
                        gq = make_float2(-0.5f * sum.x, sum.y);
                    } else {
                        gq = sum;
                    }
                    atomicAdd(reinterpret_cast<float2 *>(p.grads + 8 * (vb + s_g[clo + j]) + q), gq);
                }
            }
            if (WANT_OP) {
                for (int j = tid; j < ccnt; j += NT) {
                    float sum = 0.f;
#pragma unroll
                    for (int w = 0; w < NW; ++w) sum += s_pop[w][j];
                    if (sum != 0.f) atomicAdd(p.d_opacity + vb + s_g[clo + j], sum);
                }
            }
            __syncthreads();
        }
    }
    if (STATS) flush_stats(p.stats, n_tested, n_contrib);
}

static gs_status fill(const gs_projected *proj, int64_t n, int V, int W, int H, int bin,
                      const float *bg, const uint32_t *vals, const uint32_t *ranges,
                      const gs_tile_lists *lists, RasterParams &p)
{
    if (lists) {
        GS_REQUIRE(lists->rec && lists->count && lists->cap >= 1 && lists->cap <= (1 << 20),
                   "raster: tile lists need rec, count and 1 <= cap <= 2^20");
        GS_REQUIRE(aligned(lists->rec, 8) && aligned(lists->count, 4), "raster: misaligned tile lists");
        p.tl_rec = reinterpret_cast<uint2 *>(lists->rec);
        p.tl_cnt = lists->count;
        p.tl_cap = lists->cap;
    }
    GS_REQUIRE(proj && vals && ranges, "raster: null argument");
    GS_REQUIRE(n >= 0 && V >= 1 && V <= GS_MAX_VIEWS, "raster: bad n or V");
    GS_REQUIRE(W > 0 && H > 0 && W <= 16384 && H <= 16384, "raster: bad image size");
    GS_REQUIRE(aligned(proj->mean2d, 8) && aligned(proj->conic_opacity, 16) && aligned(ranges, 8),
               "raster: misaligned input");
    p.mean2d = reinterpret_cast<const float2 *>(proj->mean2d);
    p.conic_op = reinterpret_cast<const float4 *>(proj->conic_opacity);
    p.rgb = proj->rgb;
    p.radius = proj->radius;
    GS_REQUIRE(bin >= 1 && bin <= 64, "raster: bin must be 1..64 tiles");
    GS_REQUIRE(bin == 1 || n == 0 || proj->radius, "raster: binned lists need the radius array");
    p.vals = vals;
    p.ranges = reinterpret_cast<const uint2 *>(ranges);
    p.n = n;
    p.V = V;
    p.W = W;
    p.H = H;
    p.tx = tiles_x_of(W);
    p.ty = tiles_y_of(H);
    p.bin = bin;
    p.bins_x = bins_x_of(W, bin);
    p.bins = p.bins_x * bins_y_of(H, bin);
    p.bg0 = bg ? bg[0] : 0.f;
    p.bg1 = bg ? bg[1] : 0.f;
    p.bg2 = bg ? bg[2] : 0.f;
    return GS_OK;
}

template <bool WANT_OP, bool BINNED>
static void launch_bwd(const RasterParams &p, dim3 grid, cudaStream_t s)
{
    if (p.stats)
        raster_bwd2_kernel<WANT_OP, BINNED, true><<<grid, NT, 0, s>>>(p);
    else
        raster_bwd2_kernel<WANT_OP, BINNED, false><<<grid, NT, 0, s>>>(p);
}

}  // namespace gs3

using namespace gs3;

extern "C" gs_status gs_raster_fwd(const gs_projected *proj, int64_t n, int V, int W, int H,
                                   int bin, const float *bg, const uint32_t *vals,
                                   const uint32_t *ranges, float *img, float *T_final,
                                   int32_t *last, uint64_t *d_stats, const gs_tile_lists *lists,
                                   gs_stream stream)
{
    RasterParams p{};
    gs_status st = fill(proj, n, V, W, H, bin, bg, vals, ranges, lists, p);
    if (st != GS_OK) return st;
    GS_REQUIRE(img && T_final && last, "gs_raster_fwd: null output");
    p.img = img;
    p.T_final = T_final;
    p.last = last;
    p.stats = reinterpret_cast<unsigned long long *>(d_stats);
    dim3 grid(p.tx * p.ty, V);
    note_launch();
    cudaStream_t s = as_stream(stream);
    if (bin > 1 && p.stats)
        raster_fwd2_kernel<true, true><<<grid, NT, 0, s>>>(p);
    else if (bin > 1)
        raster_fwd2_kernel<true, false><<<grid, NT, 0, s>>>(p);
    else if (p.stats)
        raster_fwd2_kernel<false, true><<<grid, NT, 0, s>>>(p);
    else
        raster_fwd2_kernel<false, false><<<grid, NT, 0, s>>>(p);
    return launch_status("gs_raster_fwd");
}

extern "C" gs_status gs_raster_bwd(const gs_projected *proj, int64_t n, int V, int W, int H,
                                   int bin, const float *bg, const uint32_t *vals,
                                   const uint32_t *ranges, const float *T_final,
                                   const int32_t *last, const float *d_img, float *grads,
                                   float *d_opacity, uint64_t *d_stats, const gs_tile_lists *lists,
                                   gs_stream stream)
{
    RasterParams p{};
    gs_status st = fill(proj, n, V, W, H, bin, bg, vals, ranges, lists, p);
    if (st != GS_OK) return st;
    GS_REQUIRE(T_final && last && d_img && (grads || n == 0), "gs_raster_bwd: null argument");
    GS_REQUIRE(aligned(grads, 16), "gs_raster_bwd: grads must be 16-byte aligned");
    cudaStream_t s = as_stream(stream);
    if (n > 0) {
        cudaMemsetAsync(grads, 0, sizeof(float) * 8 * n * V, s);
        if (d_opacity) cudaMemsetAsync(d_opacity, 0, sizeof(float) * n * V, s);
    }
    p.T_final = const_cast<float *>(T_final);
    p.last = const_cast<int32_t *>(last);
    p.d_img = d_img;
    p.grads = grads;
    p.d_opacity = d_opacity;
    p.stats = reinterpret_cast<unsigned long long *>(d_stats);
    dim3 grid(p.tx * p.ty, V);
    note_launch();
    if (d_opacity && bin > 1)
        launch_bwd<true, true>(p, grid, s);
    else if (d_opacity)
        launch_bwd<true, false>(p, grid, s);
    else if (bin > 1)
        launch_bwd<false, true>(p, grid, s);
    else
        launch_bwd<false, false>(p, grid, s);
    return launch_status("gs_raster_bwd");
}

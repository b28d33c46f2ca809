// L1 + D-SSIM loss and its gradient (Section 4.1, Eq. 6).
// Pass 1 filters (x, y, x^2, y^2, xy) with the separable 11x11 Gaussian
// window, forms the SSIM map and the three per-pixel coefficients of its
// derivative wrt (mu_x, E[x^2], E[xy]); pass 2 filters those coefficients (the
// window is symmetric, so the adjoint is the same filter) and assembles
// dL/dI; pass 3 reduces the block partial sums (compensated FP32).
//
// Both filtering passes work on 32 x 48 output tiles.  The horizontal stage
// reads its inputs straight from global memory (through L1, as float4 where
// rows are 16-byte aligned; in pass 1 with such rows the tile's input window
// comes into shared memory by TMA instead) and leaves the row-filtered maps
// in shared memory; the vertical stage filters the columns from there.  The filters use
// the packed FP32 FMA of sm_100+ (both halves of an aligned register pair in
// one instruction): along a row a tap pair (w_t, w_t+1) multiplies an input
// pair (in_j, in_j+1) and the halves are added at the end; down a column the
// two maps of a pair (x and y, x^2 and y^2, two coefficient maps) share the
// weight.
#include <cuda.h>
#include <mutex>
#include <math.h>

#include "common.cuh"
#include "tc.cuh"

namespace gs3 {

constexpr int SX = 32;                 // output tile width
constexpr int SY = 48;                 // output tile height
constexpr int LH = 5;                  // window half-width
constexpr int SR = SY + 2 * LH;        // rows of the row-filtered maps (58)
constexpr int HSEG = 4;                // outputs of one horizontal item
constexpr int VSEG = 6;                // outputs of one thread in the vertical stage
constexpr int LTHREADS = 256;
constexpr int HITEMS = SR * (SX / HSEG);
static_assert(SX * (SY / VSEG) == LTHREADS, "vertical stage: one column segment per thread");
static_assert(SX % HSEG == 0 && HSEG == 4, "horizontal items hold four outputs");


// The window as tap pairs for the row filter: e[i] = (w_2i, w_2i+1) for
// outputs whose window starts on an even input, o[i] = (w_2i-1, w_2i) with
// w_-1 = 0 for the others.
struct RowTaps {
    float2 e[5], o[6];
    float w10;
};

__device__ __forceinline__ RowTaps row_taps(const float *w)
{
    RowTaps t;
#pragma unroll
    for (int i = 0; i < 5; ++i) t.e[i] = make_float2(w[2 * i], w[2 * i + 1]);
    t.o[0] = make_float2(0.f, w[0]);
#pragma unroll
    for (int i = 1; i < 6; ++i) t.o[i] = make_float2(w[2 * i - 1], w[2 * i]);
    t.w10 = w[10];
    return t;
}

// Inputs of one horizontal item as pairs: m[k] = (in_2k, in_2k+1), in_j the
// value at column B + j, B = x0 + c0 - 8 (a multiple of 4).  Output o of the
// item (column B + 8 + o) sums in_3+o .. in_13+o.
constexpr int NPAIR = 9;

__device__ __forceinline__ void load_pairs(const float *row, int W, int B, bool vec, float2 (&m)[NPAIR])
{
    m[0] = make_float2(0.f, 0.f);  // in_0, in_1: never used
    if (vec && B >= 0 && B + 16 <= W) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row + B);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = __ldg(r4 + q);
            m[2 * q] = make_float2(v.x, v.y);
            m[2 * q + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int k = 1; k < 8; ++k) {
            const int g0 = B + 2 * k, g1 = g0 + 1;
            m[k] = make_float2(g0 >= 0 && g0 < W ? __ldg(row + g0) : 0.f,
                               g1 >= 0 && g1 < W ? __ldg(row + g1) : 0.f);
        }
    }
    const int g16 = B + 16;
    m[8] = make_float2(g16 < W ? __ldg(row + g16) : 0.f, 0.f);
}

// Row filter of one map for the item's four outputs.
__device__ __forceinline__ void row_filter(const float2 (&m)[NPAIR], const RowTaps &t, float (&out)[HSEG])
{
#pragma unroll
    for (int o = 0; o < HSEG; o += 2) {
        // even output o: window in_3+o .. in_13+o, pairs from in_2+o with o[]
        float2 a = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 6; ++i) a = __ffma2_rn(t.o[i], m[1 + o / 2 + i], a);
        out[o] = a.x + a.y;
        // odd output o + 1: pairs from in_4+o with e[], last tap in_14+o
        float2 b = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 5; ++i) b = __ffma2_rn(t.e[i], m[2 + o / 2 + i], b);
        out[o + 1] = fmaf(t.w10, m[7 + o / 2].x, b.x + b.y);
    }
}

__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }

struct LossParams {
    float win[11];        // normalised 11-tap Gaussian window (sigma 1.5), set on the host
    const float *x, *y;
    int P, H, W;
    float lam;
    float invM;           // 1 / (planes H W), the mean's weight (set on the host)
    bool vec;             // rows of x, y and the coefficient maps are 16-byte aligned
    float *ca, *cb, *cc;  // per-pixel derivative coefficients
    float2 *partial;      // [blocks]: (sum of SSIM map, sum |x - y|)
    float *d_img;
    float *d_loss, *d_ssim;
    int nblocks;
};

#ifndef SSIM_FWD_MIN_BLOCKS
#define SSIM_FWD_MIN_BLOCKS 3  // 80 registers, no spills
#endif
// TMA staging of the forward's input window: columns x0 - 8 .. x0 + 39 (TW,
// a 16-byte aligned start) and rows y0 - LH .. y0 + SY + LH - 1 of one plane
// of each image, zero-filled outside the image by the copy itself.  Two
// stages of TH rows, each on its own mbarrier: the row filter works through
// the first half of the window while the second is still in flight.
constexpr int TW = 48;
constexpr int TH = SR / 2;   // 29 rows per stage
static_assert(SR % 2 == 0 && TH * (SX / HSEG) <= LTHREADS, "one round of items per stage");
constexpr uint32_t kTmaStageBytes = 2u * TH * TW * sizeof(float);   // x and y, one stage
// each (image, stage) buffer starts on a 128-byte boundary, as the copies require
constexpr int kTmaBufFloats = ((TH * TW * (int)sizeof(float) + 127) / 128) * 128 / (int)sizeof(float);
constexpr uint32_t kTmaSmem = 4u * kTmaBufFloats * sizeof(float) + 128;  // + alignment slack

template <bool TMA>
__global__ void __launch_bounds__(LTHREADS, SSIM_FWD_MIN_BLOCKS)
    ssim_fwd_kernel(LossParams p, const __grid_constant__ CUtensorMap tmx,
                    const __grid_constant__ CUtensorMap tmy)
{
    __shared__ float2 s_xy[SR][SX];   // row-filtered (x, y)
    __shared__ float2 s_sq[SR][SX];   // row-filtered (x^2, y^2)
    __shared__ float s_p[SR][SX];     // row-filtered x y
    __shared__ float red[2][LTHREADS / 32];
    __shared__ __align__(8) unsigned long long s_mbar[2];
    extern __shared__ __align__(128) unsigned char s_dyn[];   // TMA: [image][stage][TH][TW] floats
    float *s_in = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(s_dyn) + 127) & ~uintptr_t(127));
    const float *c_win = p.win;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * SX, y0 = blockIdx.y * SY, pl = blockIdx.z;
    const int64_t HW = (int64_t)p.H * p.W;
    const float *X = p.x + pl * HW, *Y = p.y + pl * HW;
    float lsum = 0.f;
    bool ok = true;
    if (TMA) {
        if (tid == 0) {
            tc::mbar_init(tc::smem_u32(&s_mbar[0]), 1);
            tc::mbar_init(tc::smem_u32(&s_mbar[1]), 1);
        }
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t mbar = tc::smem_u32(&s_mbar[h]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                             "r"(kTmaStageBytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(tc::smem_u32(s_in + h * kTmaBufFloats)),
                    "l"(reinterpret_cast<uint64_t>(&tmx)), "r"(x0 - 8), "r"(y0 - LH + h * TH), "r"(pl),
                    "r"(mbar)
                    : "memory");
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(tc::smem_u32(s_in + (2 + h) * kTmaBufFloats)),
                    "l"(reinterpret_cast<uint64_t>(&tmy)), "r"(x0 - 8), "r"(y0 - LH + h * TH), "r"(pl),
                    "r"(mbar)
                    : "memory");
            }
        }
    }
    {
        const RowTaps t = row_taps(c_win);
        for (int round = 0; round < (TMA ? 2 : (HITEMS + LTHREADS - 1) / LTHREADS); ++round) {
            int item;
            if (TMA) {
                // stage `round` holds rows TH round .. TH round + TH - 1; bounded
                // wait, and a block that gives up writes NaN outputs (the loss
                // and, through the gradient, the non-finite check report it)
                const bool got = tc::mbar_wait(tc::smem_u32(&s_mbar[round]), 0, tc::kWaitTries);
                ok = __syncthreads_and(ok && got);
                if (tid >= TH * (SX / HSEG)) continue;
                item = round * TH * (SX / HSEG) + tid;
            } else {
                item = round * LTHREADS + tid;
                if (item >= HITEMS) continue;
            }
            const int r = item / (SX / HSEG), c0 = (item % (SX / HSEG)) * HSEG;
            const int gy = y0 - LH + r;
            float fx[HSEG], fy[HSEG], fxx[HSEG], fyy[HSEG], fxy[HSEG];
            if (TMA || (gy >= 0 && gy < p.H)) {
                const int B = x0 + c0 - 8;
                float2 mx[NPAIR], my[NPAIR], mxx[NPAIR], myy[NPAIR], mxy[NPAIR];
                if (TMA) {
                    const int h = r / TH, rl = r - h * TH;   // stage and row within it
                    const float2 *rx =
                        reinterpret_cast<const float2 *>(s_in + h * kTmaBufFloats + rl * TW + c0);
                    const float2 *ry =
                        reinterpret_cast<const float2 *>(s_in + (2 + h) * kTmaBufFloats + rl * TW + c0);
                    mx[0] = my[0] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int k = 1; k < NPAIR; ++k) {
                        mx[k] = rx[k];
                        my[k] = ry[k];
                    }
                } else {
                    load_pairs(X + (int64_t)gy * p.W, p.W, B, p.vec, mx);
                    load_pairs(Y + (int64_t)gy * p.W, p.W, B, p.vec, my);
                }
#pragma unroll
                for (int k = 1; k < NPAIR; ++k) {
                    mxx[k] = __fmul2_rn(mx[k], mx[k]);
                    myy[k] = __fmul2_rn(my[k], my[k]);
                    mxy[k] = __fmul2_rn(mx[k], my[k]);
                }
                row_filter(mx, t, fx);
                row_filter(my, t, fy);
                row_filter(mxx, t, fxx);
                row_filter(myy, t, fyy);
                row_filter(mxy, t, fxy);
                // L1 term at the item's outputs in_8 .. in_11 (pairs 4 and 5)
                if (r >= LH && r < LH + SY && gy < p.H) {
#pragma unroll
                    for (int o = 0; o < HSEG; ++o) {
                        const float2 a = mx[4 + o / 2], b = my[4 + o / 2];
                        const float d = (o & 1) ? a.y - b.y : a.x - b.x;
                        if (x0 + c0 + o < p.W) lsum += fabsf(d);
                    }
                }
            } else {
#pragma unroll
                for (int o = 0; o < HSEG; ++o) fx[o] = fy[o] = fxx[o] = fyy[o] = fxy[o] = 0.f;
            }
#pragma unroll
            for (int o = 0; o < HSEG; ++o) {
                s_xy[r][c0 + o] = make_float2(fx[o], fy[o]);
                s_sq[r][c0 + o] = make_float2(fxx[o], fyy[o]);
                s_p[r][c0 + o] = fxy[o];
            }
        }
    }
    __syncthreads();
    // vertical: thread -> column c, rows r0 .. r0 + VSEG - 1 of the tile
    const int c = tid % SX, r0 = (tid / SX) * VSEG;
    float2 fxy2[VSEG], fsq2[VSEG];
    float fp[VSEG];
    {
        float2 wd[11];
#pragma unroll
        for (int k = 0; k < 11; ++k) wd[k] = dup(c_win[k]);
        float2 col[VSEG + 10];
#pragma unroll
        for (int k = 0; k < VSEG + 10; ++k) col[k] = s_xy[r0 + k][c];
#pragma unroll
        for (int o = 0; o < VSEG; ++o) {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 11; ++k) a = __ffma2_rn(wd[k], col[o + k], a);
            fxy2[o] = a;
        }
#pragma unroll
        for (int k = 0; k < VSEG + 10; ++k) col[k] = s_sq[r0 + k][c];
#pragma unroll
        for (int o = 0; o < VSEG; ++o) {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 11; ++k) a = __ffma2_rn(wd[k], col[o + k], a);
            fsq2[o] = a;
        }
        float cp[VSEG + 10];
#pragma unroll
        for (int k = 0; k < VSEG + 10; ++k) cp[k] = s_p[r0 + k][c];
#pragma unroll
        for (int o = 0; o < VSEG; ++o) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) a = fmaf(c_win[k], cp[o + k], a);
            fp[o] = a;
        }
    }
    // per-thread and per-warp sums in FP32 (at most VSEG * 32 terms), the
    // block's and the final reduction in FP64
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float ssum = 0.f;
    const int gx = x0 + c;
#pragma unroll
    for (int o = 0; o < VSEG; ++o) {
        const int gy = y0 + r0 + o;
        if (gy >= p.H || gx >= p.W) continue;
        const float mx = fxy2[o].x, my = fxy2[o].y, exx = fsq2[o].x, eyy = fsq2[o].y, exy = fp[o];
        const float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
        const float n1 = 2.f * mx * my + C1, n2 = 2.f * sxy + C2;
        const float d1 = mx * mx + my * my + C1, d2 = sxx + syy + C2;
        const float idd = 1.f / (d1 * d2);
        const float sv = n1 * n2 * idd;
        // 1 / d1 = d2 idd and 1 / d2 = d1 idd
        const float ds_dmx = 2.f * my * n2 * idd - sv * 2.f * mx * (d2 * idd);
        const float ds_dsxx = -sv * (d1 * idd);
        const float ds_dsxy = 2.f * n1 * idd;
        const int64_t oo = pl * HW + (int64_t)gy * p.W + gx;
        const float bad = ok ? 0.f : __int_as_float(0x7fc00000);   // NaN when the copy gave up
        p.ca[oo] = ds_dmx - 2.f * mx * ds_dsxx - my * ds_dsxy + bad;
        p.cb[oo] = ds_dsxx + bad;
        p.cc[oo] = ds_dsxy + bad;
        ssum += sv + bad;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = ssum;
        red[1][tid >> 5] = lsum;
    }
    __syncthreads();
    if (tid == 0) {
        float a = 0.f, b = 0.f;
        for (int ww = 0; ww < LTHREADS / 32; ++ww) {
            a += red[0][ww];
            b += red[1][ww];
        }
        int64_t bid = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        p.partial[bid] = make_float2(a, b);
    }
}

#ifndef SSIM_BWD_MIN_BLOCKS
#define SSIM_BWD_MIN_BLOCKS 4  // 62 registers, no spills
#endif
__global__ void __launch_bounds__(LTHREADS, SSIM_BWD_MIN_BLOCKS) ssim_bwd_kernel(LossParams p)
{
    __shared__ float2 s_ab[SR][SX];   // row-filtered (ca, cb)
    __shared__ float s_c[SR][SX];     // row-filtered cc
    const float *c_win = p.win;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * SX, y0 = blockIdx.y * SY, pl = blockIdx.z;
    const int64_t HW = (int64_t)p.H * p.W;
    {
        const RowTaps t = row_taps(c_win);
        const float *A = p.ca + pl * HW, *Bm = p.cb + pl * HW, *Cm = p.cc + pl * HW;
        for (int item = tid; item < HITEMS; item += LTHREADS) {
            const int r = item / (SX / HSEG), c0 = (item % (SX / HSEG)) * HSEG;
            const int gy = y0 - LH + r;
            float fa[HSEG], fb[HSEG], fc[HSEG];
            if (gy >= 0 && gy < p.H) {
                const int B = x0 + c0 - 8;
                const int64_t ro = (int64_t)gy * p.W;
                // all three rows in flight before any filtering
                float2 ma[NPAIR], mb[NPAIR], mc[NPAIR];
                load_pairs(A + ro, p.W, B, p.vec, ma);
                load_pairs(Bm + ro, p.W, B, p.vec, mb);
                load_pairs(Cm + ro, p.W, B, p.vec, mc);
                row_filter(ma, t, fa);
                row_filter(mb, t, fb);
                row_filter(mc, t, fc);
            } else {
#pragma unroll
                for (int o = 0; o < HSEG; ++o) fa[o] = fb[o] = fc[o] = 0.f;
            }
#pragma unroll
            for (int o = 0; o < HSEG; ++o) {
                s_ab[r][c0 + o] = make_float2(fa[o], fb[o]);
                s_c[r][c0 + o] = fc[o];
            }
        }
    }
    __syncthreads();
    const float invM = p.invM;
    const int c = tid % SX, r0 = (tid / SX) * VSEG;
    const int gx = x0 + c;
    // the images at this thread's outputs, loaded before the column filters
    float xv[VSEG], yv[VSEG];
#pragma unroll
    for (int o = 0; o < VSEG; ++o) {
        const int gy = y0 + r0 + o;
        const bool in = gy < p.H && gx < p.W;
        const int64_t oo = pl * HW + (int64_t)gy * p.W + gx;
        xv[o] = in ? __ldg(p.x + oo) : 0.f;
        yv[o] = in ? __ldg(p.y + oo) : 0.f;
    }
    float2 fab[VSEG];
    float fc[VSEG];
    {
        float2 wd[11];
#pragma unroll
        for (int k = 0; k < 11; ++k) wd[k] = dup(c_win[k]);
        float2 col[VSEG + 10];
#pragma unroll
        for (int k = 0; k < VSEG + 10; ++k) col[k] = s_ab[r0 + k][c];
#pragma unroll
        for (int o = 0; o < VSEG; ++o) {
            float2 a = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < 11; ++k) a = __ffma2_rn(wd[k], col[o + k], a);
            fab[o] = a;
        }
        float cp[VSEG + 10];
#pragma unroll
        for (int k = 0; k < VSEG + 10; ++k) cp[k] = s_c[r0 + k][c];
#pragma unroll
        for (int o = 0; o < VSEG; ++o) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) a = fmaf(c_win[k], cp[o + k], a);
            fc[o] = a;
        }
    }
#pragma unroll
    for (int o = 0; o < VSEG; ++o) {
        const int gy = y0 + r0 + o;
        if (gy >= p.H || gx >= p.W) continue;
        const int64_t oo = pl * HW + (int64_t)gy * p.W + gx;
        const float diff = xv[o] - yv[o];
        const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        const float dssim = fab[o].x + 2.f * xv[o] * fab[o].y + yv[o] * fc[o];
        p.d_img[oo] = ((1.f - p.lam) * sgn - p.lam * dssim) * invM;
    }
}

// Compensated (Kahan) accumulation: s + (-c) carries the sum to about one
// rounding, independent of the number of terms.
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Pass 3: the block partial sums in FP32, each thread's share compensated,
// the 1024 shares added in a tree (error about log2(1024) roundings).
__global__ void __launch_bounds__(1024) loss_final_kernel(LossParams p)
{
    __shared__ float red[2][32];
    float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
    for (int i = threadIdx.x; i < p.nblocks; i += blockDim.x) {
        const float2 v = p.partial[i];
        kahan_add(sa, ca, v.x);
        kahan_add(sb, cb, v.y);
    }
    float a = sa - ca, b = sb - cb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = (int)(blockDim.x >> 5);
        a = threadIdx.x < nw ? red[0][threadIdx.x] : 0.f;
        b = threadIdx.x < nw ? red[1][threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (threadIdx.x == 0) {
            const float ssim = a * p.invM;
            *p.d_loss = (1.f - p.lam) * (b * p.invM) + p.lam * (1.f - ssim);
            if (p.d_ssim) *p.d_ssim = ssim;
        }
    }
}

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

#ifndef SSIM_TMA
#define SSIM_TMA 1
#endif

// Tiled TMA map of a [planes][H][W] FP32 image stack with a TW x TH box.
// False (and the L1 path is used) when the driver entry point is missing or
// the rows are not 16-byte aligned.
static bool make_plane_map(CUtensorMap *m, const float *base, int planes, int H, int W)
{
    typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeTiled encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<EncodeTiled>(fn);
    }();
    if (!encode || W % 4 != 0 || !aligned(base, 16)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)W * sizeof(float), (cuuint64_t)H * W * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)TW, (cuuint32_t)TH, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace gs3

using namespace gs3;

extern "C" size_t gs_loss_workspace_size(int planes, int H, int W)
{
    if (planes <= 0 || H <= 0 || W <= 0) return 0;
    size_t px = (size_t)planes * H * W;
    size_t nb = (size_t)ceil_div(W, SX) * ceil_div(H, SY) * planes;
    return 3 * a256(4 * px) + a256(16 * nb);
}

extern "C" gs_status gs_loss_l1_dssim(const float *img, const float *target, int planes, int H,
                                      int W, float lambda, float *d_img, float *d_loss,
                                      float *d_ssim, void *ws, size_t ws_bytes, gs_stream stream)
{
    GS_REQUIRE(img && target && d_img && d_loss && ws, "gs_loss_l1_dssim: null argument");
    GS_REQUIRE(planes > 0 && H > 0 && W > 0 && planes <= 65535, "gs_loss_l1_dssim: bad shape");
    GS_REQUIRE(ws_bytes >= gs_loss_workspace_size(planes, H, W),
               "gs_loss_l1_dssim: workspace too small");
    GS_REQUIRE(aligned(ws, 256), "gs_loss_l1_dssim: workspace must be 256-byte aligned");
    LossParams p{};
    {
        double w[11], sum = 0.0;
        for (int i = 0; i < 11; ++i) sum += (w[i] = exp(-(double)((i - 5) * (i - 5)) / 4.5));
        for (int i = 0; i < 11; ++i) p.win[i] = (float)(w[i] / sum);
    }
    p.x = img;
    p.y = target;
    p.P = planes;
    p.H = H;
    p.W = W;
    p.lam = lambda;
    p.invM = (float)(1.0 / ((double)planes * (double)H * (double)W));
    size_t px = (size_t)planes * H * W;
    char *b = reinterpret_cast<char *>(ws);
    p.ca = reinterpret_cast<float *>(b);
    p.cb = reinterpret_cast<float *>(b + a256(4 * px));
    p.cc = reinterpret_cast<float *>(b + 2 * a256(4 * px));
    p.partial = reinterpret_cast<float2 *>(b + 3 * a256(4 * px));
    p.d_img = d_img;
    p.d_loss = d_loss;
    p.d_ssim = d_ssim;
    p.vec = (W % 4) == 0 && aligned(img, 16) && aligned(target, 16) && aligned(ws, 16);
    dim3 grid((unsigned)ceil_div(W, SX), (unsigned)ceil_div(H, SY), (unsigned)planes);
    p.nblocks = (int)(grid.x * grid.y * grid.z);
    cudaStream_t s = as_stream(stream);
    CUtensorMap tmx{}, tmy{};
    const bool tma = SSIM_TMA && p.vec && make_plane_map(&tmx, img, planes, H, W) &&
                     make_plane_map(&tmy, target, planes, H, W);
    note_launch();
    if (tma) {
        static std::once_flag once;
        std::call_once(once, [] {
            cudaFuncSetAttribute((const void *)ssim_fwd_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem);
        });
        ssim_fwd_kernel<true><<<grid, LTHREADS, kTmaSmem, s>>>(p, tmx, tmy);
    } else {
        ssim_fwd_kernel<false><<<grid, LTHREADS, 0, s>>>(p, tmx, tmy);
    }
    note_launch();
    ssim_bwd_kernel<<<grid, LTHREADS, 0, s>>>(p);
    note_launch();
    loss_final_kernel<<<1, 1024, 0, s>>>(p);
    return launch_status("gs_loss_l1_dssim");
}

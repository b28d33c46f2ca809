// Neural Transformation Cache (Section 4.1): multi-resolution hash encoding,
// the 32-64-64-7 MLP (FP32 SIMT path), the transformation of means and
// rotations, the warm-up loss (Eq. 7), and the optimiser kernels (Adam,
// non-finite check, loss-scale state).  The BF16 tensor-core MLP lives in
// mlp_tc.cu.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "ntc.cuh"
#include "sort.cuh"

namespace gs3 {

static thread_local char g_err[512];

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// ------------------------------------------------------------ hash grid
bool grid_params(const gs_hashgrid *g, GridParams &P, int64_t &total)
{
    if (!g || g->levels < 1 || g->levels > kMaxLevels || g->features != 2 || g->log2_table < 4 ||
        g->log2_table > 24 || g->n_min < 1 || g->n_max < g->n_min)
        return false;
    for (int k = 0; k < 3; ++k)
        if (!(g->aabb[3 + k] > g->aabb[k])) return false;
    const int L = g->levels;
    double b = L > 1 ? exp((log((double)g->n_max) - log((double)g->n_min)) / (double)(L - 1)) : 1.0;
    int64_t T = int64_t(1) << g->log2_table;
    int64_t off = 0;
    P.L = L;
    P.mask = (uint32_t)(T - 1);
    for (int k = 0; k < 3; ++k) {
        P.amin[k] = g->aabb[k];
        P.ext[k] = g->aabb[3 + k] - g->aabb[k];
    }
    for (int l = 0; l < L; ++l) {
        int res = (int)floor((double)g->n_min * pow(b, (double)l) + 1e-6);
        int64_t side = res + 1;
        bool dense = side * side * side <= T;
        P.res[l] = res;
        P.dense[l] = dense ? 1 : 0;
        P.offset[l] = (uint32_t)off;
        off += dense ? side * side * side : T;
    }
    total = off;
    return off < (int64_t(1) << 31);
}

template <typename T>
__device__ __forceinline__ float2 load_feat(const T *table, uint32_t row);
template <>
__device__ __forceinline__ float2 load_feat<__half>(const __half *table, uint32_t row)
{
    return __half22float2(reinterpret_cast<const __half2 *>(table)[row]);
}
template <>
__device__ __forceinline__ float2 load_feat<float>(const float *table, uint32_t row)
{
    return reinterpret_cast<const float2 *>(table)[row];
}

// The encoding kernels work on blocks of 32 Gaussians with one warp per level
// (ENC_THREADS = 32 x kMaxLevels threads; warps at l >= L idle): a warp's
// lanes gather the same level for 32 Gaussians, so when the Gaussians are in
// spatial order (ntc_spatial_order) the coarse levels' corners of a warp
// fall in a few table rows.  Block b takes the Gaussians order[32 b ..
// 32 b + 31] (the identity without an order); an order entry >= n is
// skipped.  Rows of the encoding and of its gradient pass through shared
// memory so that global accesses are whole rows.
constexpr int ENC_G = 32;
constexpr int ENC_THREADS = 32 * kMaxLevels;

__device__ __forceinline__ int64_t enc_row(const uint32_t *order, int64_t j, int64_t n)
{
    if (j >= n) return -1;
    const int64_t i = order ? (int64_t)order[j] : j;
    return i < n ? i : -1;
}

template <typename TT, typename ET>
__global__ void __launch_bounds__(ENC_THREADS) encode_fwd_kernel(const float *mean, int64_t n, GridParams g,
                                                                 const TT *table, ET *enc,
                                                                 const uint32_t *order)
{
    __shared__ float s_out[ENC_G][2 * kMaxLevels + 1];
    const int lane = threadIdx.x & 31, l = threadIdx.x >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * ENC_G;
    const int64_t i = enc_row(order, j0 + lane, n);
    if (i >= 0 && l < g.L) {
        const float3 m = make_float3(mean[3 * i], mean[3 * i + 1], mean[3 * i + 2]);
        uint32_t idx[8];
        float w[8];
        level_corners(g, l, m, idx, w);
        float2 t[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) t[c] = load_feat<TT>(table, idx[c]);
        float f0 = 0.f, f1 = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            f0 = fmaf(w[c], t[c].x, f0);
            f1 = fmaf(w[c], t[c].y, f1);
        }
        s_out[lane][2 * l] = f0;
        s_out[lane][2 * l + 1] = f1;
    }
    __syncthreads();
    // row r of the block: threads 16 r .. 16 r + 15 write its 2L values in pairs
    const int r = threadIdx.x >> 4, q = threadIdx.x & 15;
    const int64_t ir = enc_row(order, j0 + r, n);
    if (ir >= 0 && q < g.L) store2(enc + ir * (int64_t)(2 * g.L) + 2 * q, s_out[r][2 * q], s_out[r][2 * q + 1]);
}

// Reverse: one thread per (Gaussian, level), threadIdx.x the level and
// threadIdx.y the Gaussian (block b takes order[8 b ..], the identity
// without an order).  A Gaussian no view saw has a zero gradient and its
// threads return at once; the lanes of a warp scatter into different levels'
// tables.  (The level-major mapping with in-warp combining of the coarse
// levels' atomics was slower here, where most gradients are zero.)
constexpr int ENC_BWD_G = 8;

__global__ void __launch_bounds__(128) encode_bwd_kernel(const float *mean, int64_t n, GridParams g,
                                                         const float *d_enc, float *d_table,
                                                         const uint32_t *order, const int64_t *d_count)
{
    // with a count the grid is a fixed size that strides over the list
    const int64_t nj = d_count ? *d_count : n;
    const int l = threadIdx.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; j < nj; j += (int64_t)gridDim.x * blockDim.y) {
        const int64_t i = enc_row(order, j, n);
        if (i < 0 || l >= g.L) continue;
        const float2 gg = reinterpret_cast<const float2 *>(d_enc + i * (int64_t)(2 * g.L))[l];
        if (gg.x == 0.f && gg.y == 0.f) continue;
        const float3 m = make_float3(mean[3 * i], mean[3 * i + 1], mean[3 * i + 2]);
        uint32_t idx[8];
        float w[8];
        level_corners(g, l, m, idx, w);
#pragma unroll
        for (int c = 0; c < 8; ++c)
            atomicAdd(reinterpret_cast<float2 *>(d_table) + idx[c], make_float2(w[c] * gg.x, w[c] * gg.y));
    }
}

// The rows of d_raw7 with a nonzero (or non-finite) value, in no particular
// order: a warp's rows get consecutive slots from one atomic on the count.
__global__ void active_rows_kernel(const float *d_raw7, int64_t n, uint32_t *rows, unsigned long long *count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool act = false;
    if (i < n) {
        const float *r = d_raw7 + 7 * i;
#pragma unroll
        for (int q = 0; q < 7; ++q) act |= r[q] != 0.f;
    }
    const unsigned b = __ballot_sync(0xffffffffu, act);
    if (b == 0u) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(count, (unsigned long long)__popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (act) rows[base + __popc(b & ((1u << lane) - 1u))] = (uint32_t)i;
}

// Morton code (10 bits an axis) of every mean within the grid's box, and the
// identity as the values to sort.
__device__ __forceinline__ uint32_t spread10(uint32_t x)
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x30000ffu;
    x = (x | (x << 8)) & 0x300f00fu;
    x = (x | (x << 4)) & 0x30c30c3u;
    x = (x | (x << 2)) & 0x9249249u;
    return x;
}

__global__ void morton_kernel(const float *mean, int64_t n, GridParams g, uint32_t *code, uint32_t *idx)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float x = (mean[3 * i + k] - g.amin[k]) / g.ext[k];
        q[k] = (uint32_t)(fminf(fmaxf(x, 0.f), 1.f) * 1023.f);
    }
    code[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    idx[i] = (uint32_t)i;
}

// ------------------------------------------------------------ MLP (SIMT)
template <typename ET>
__global__ void __launch_bounds__(128) mlp_fwd_simt_kernel(const ET *enc, int64_t n, const float *W,
                                                           float *raw7)
{
    __shared__ float sW[GS_MLP_PARAMS];
    for (int k = threadIdx.x; k < GS_MLP_PARAMS; k += blockDim.x) sW[k] = W[k];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *W1 = sW, *W2 = sW + 64 * 32, *W3 = sW + 64 * 32 + 64 * 64;
    float x[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) x[k] = to_f32(enc[i * 32 + k]);
    float h1[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) s = fmaf(W1[j * 32 + k], x[k], s);
        h1[j] = fmaxf(s, 0.f);
    }
    float o[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j = 0; j < 64; ++j) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 64; ++k) s = fmaf(W2[j * 64 + k], h1[k], s);
        s = fmaxf(s, 0.f);
#pragma unroll
        for (int q = 0; q < 7; ++q) o[q] = fmaf(W3[q * 64 + j], s, o[q]);
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) raw7[i * 7 + q] = o[q];
}

// Backward: each block owns chunks of 128 rows; per chunk every thread forms
// its row's activations and gradients in shared memory, then every thread
// accumulates its share of the 6592 weight gradients over the 128 rows; one
// atomic per weight per block at the end.
constexpr int MB_ROWS = 128;
constexpr int MB_SX = 33, MB_SH = 65, MB_SO = 9;
constexpr int MB_PER_THREAD = (GS_MLP_PARAMS + MB_ROWS - 1) / MB_ROWS;  // 52
constexpr size_t MB_SMEM =
    sizeof(float) * (GS_MLP_PARAMS + MB_ROWS * (MB_SX + 4 * MB_SH + MB_SO));

template <typename ET>
__global__ void __launch_bounds__(MB_ROWS) mlp_bwd_simt_kernel(const ET *enc, int64_t n,
                                                               const float *W, const float *d_raw7,
                                                               const float *d_scale, float *dW,
                                                               float *d_enc, const uint32_t *rows,
                                                               const int64_t *d_rows)
{
    extern __shared__ float smem[];
    float *sW = smem;
    float *sX = sW + GS_MLP_PARAMS;
    float *sH1 = sX + MB_ROWS * MB_SX;
    float *sH2 = sH1 + MB_ROWS * MB_SH;
    float *sG2 = sH2 + MB_ROWS * MB_SH;
    float *sG1 = sG2 + MB_ROWS * MB_SH;
    float *sGO = sG1 + MB_ROWS * MB_SH;
    for (int k = threadIdx.x; k < GS_MLP_PARAMS; k += blockDim.x) sW[k] = W[k];
    const float *W1 = sW, *W2 = sW + 64 * 32, *W3 = sW + 64 * 32 + 64 * 64;
    const float scale = d_scale ? *d_scale : 1.f;
    const int t = threadIdx.x;
    float acc[MB_PER_THREAD];
#pragma unroll
    for (int r = 0; r < MB_PER_THREAD; ++r) acc[r] = 0.f;
    // with a row list, slot k of the work is row rows[k], k < *d_rows
    const int64_t nslots = d_rows ? *d_rows : n;
    const int64_t nchunks = (nslots + MB_ROWS - 1) / MB_ROWS;
    __syncthreads();
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t k = ch * MB_ROWS + t;
        int64_t i = k < nslots ? (rows ? (int64_t)rows[k] : k) : n;
        bool ok = i < n;
        float *x = sX + t * MB_SX, *h1 = sH1 + t * MB_SH, *h2 = sH2 + t * MB_SH;
        float *g2 = sG2 + t * MB_SH, *g1 = sG1 + t * MB_SH, *go = sGO + t * MB_SO;
        for (int k = 0; k < 32; ++k) x[k] = ok ? to_f32(enc[i * 32 + k]) : 0.f;
        for (int j = 0; j < 64; ++j) {
            float s = 0.f;
            for (int k = 0; k < 32; ++k) s = fmaf(W1[j * 32 + k], x[k], s);
            h1[j] = fmaxf(s, 0.f);
        }
        for (int j = 0; j < 64; ++j) {
            float s = 0.f;
            for (int k = 0; k < 64; ++k) s = fmaf(W2[j * 64 + k], h1[k], s);
            h2[j] = fmaxf(s, 0.f);
        }
        for (int q = 0; q < 7; ++q) go[q] = ok ? d_raw7[i * 7 + q] * scale : 0.f;
        for (int j = 0; j < 64; ++j) {
            float s = 0.f;
            for (int q = 0; q < 7; ++q) s = fmaf(W3[q * 64 + j], go[q], s);
            g2[j] = h2[j] > 0.f ? s : 0.f;
        }
        for (int k = 0; k < 64; ++k) {
            float s = 0.f;
            for (int j = 0; j < 64; ++j) s = fmaf(W2[j * 64 + k], g2[j], s);
            g1[k] = h1[k] > 0.f ? s : 0.f;
        }
        if (ok && d_enc) {
            for (int m = 0; m < 32; ++m) {
                float s = 0.f;
                for (int k = 0; k < 64; ++k) s = fmaf(W1[k * 32 + m], g1[k], s);
                d_enc[i * 32 + m] = s;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < MB_PER_THREAD; ++r) {
            int e = t + r * MB_ROWS;
            if (e < 64 * 32) {
                int k = e >> 5, m = e & 31;
                float s = 0.f;
                for (int q = 0; q < MB_ROWS; ++q) s = fmaf(sG1[q * MB_SH + k], sX[q * MB_SX + m], s);
                acc[r] += s;
            } else if (e < 64 * 32 + 64 * 64) {
                int e2 = e - 64 * 32, j = e2 >> 6, k = e2 & 63;
                float s = 0.f;
                for (int q = 0; q < MB_ROWS; ++q) s = fmaf(sG2[q * MB_SH + j], sH1[q * MB_SH + k], s);
                acc[r] += s;
            } else if (e < GS_MLP_PARAMS) {
                int e3 = e - 64 * 32 - 64 * 64, o = e3 >> 6, j = e3 & 63;
                float s = 0.f;
                for (int q = 0; q < MB_ROWS; ++q) s = fmaf(sGO[q * MB_SO + o], sH2[q * MB_SH + j], s);
                acc[r] += s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < MB_PER_THREAD; ++r) {
        int e = t + r * MB_ROWS;
        if (e < GS_MLP_PARAMS && acc[r] != 0.f) atomicAdd(dW + e, acc[r]);
    }
}

// ------------------------------------------------------- transformation
__global__ void apply_kernel(const float *mean, const float *quat, const float *raw7, int64_t n,
                             Box box, int order, float *mean_out, float *quat_out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 m = make_float3(mean[3 * i], mean[3 * i + 1], mean[3 * i + 2]);
    float4 q = reinterpret_cast<const float4 *>(quat)[i];
    const float *r = raw7 + 7 * i;
    float4 qn = qnormalize(q);
    if (!box.inside(m)) {
        mean_out[3 * i] = m.x;
        mean_out[3 * i + 1] = m.y;
        mean_out[3 * i + 2] = m.z;
        reinterpret_cast<float4 *>(quat_out)[i] = qn;
        return;
    }
    float4 dq = qnormalize(make_float4(r[3], r[4], r[5], r[6]));
    mean_out[3 * i] = m.x + r[0];
    mean_out[3 * i + 1] = m.y + r[1];
    mean_out[3 * i + 2] = m.z + r[2];
    reinterpret_cast<float4 *>(quat_out)[i] = order == 0 ? qmul(qn, dq) : qmul(dq, qn);
}

__global__ void apply_bwd_kernel(const float *mean, const float *quat, const float *raw7, int64_t n,
                                 Box box, int order, const float *d_mean_out,
                                 const float *d_quat_out, float *d_raw7)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float *o = d_raw7 + 7 * i;
    float3 m = make_float3(mean[3 * i], mean[3 * i + 1], mean[3 * i + 2]);
    if (!box.inside(m)) {
#pragma unroll
        for (int k = 0; k < 7; ++k) o[k] = 0.f;
        return;
    }
    o[0] = d_mean_out[3 * i];
    o[1] = d_mean_out[3 * i + 1];
    o[2] = d_mean_out[3 * i + 2];
    float4 qn = qnormalize(reinterpret_cast<const float4 *>(quat)[i]);
    const float *r = raw7 + 7 * i;
    float4 g = reinterpret_cast<const float4 *>(d_quat_out)[i];
    float4 gd = order == 0 ? qmul_left_T(qn, g) : qmul_right_T(qn, g);
    float4 dqraw = make_float4(r[3], r[4], r[5], r[6]);
    float4 d = qnormalize_bwd(dqraw, gd);
    o[3] = d.x;
    o[4] = d.y;
    o[5] = d.z;
    o[6] = d.w;
}

// ------------------------------------------------------------- warm-up
__global__ void __launch_bounds__(256) warmup_kernel(const float *raw7, int64_t n, float *d_raw7,
                                                     float *d_loss)
{
    __shared__ float red[8];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float L = 0.f;
    if (i < n) {
        const float *r = raw7 + 7 * i;
        float n2 = r[3] * r[3] + r[4] * r[4] + r[5] * r[5] + r[6] * r[6];
        float in = 1.f / (float)n;
        L = fabsf(r[0]) + fabsf(r[1]) + fabsf(r[2]) - r[3] * r[3] / n2;
        float *o = d_raw7 + 7 * i;
#pragma unroll
        for (int k = 0; k < 3; ++k) o[k] = (r[k] > 0.f ? 1.f : (r[k] < 0.f ? -1.f : 0.f)) * in;
        float w = r[3];
        float c = 2.f * w * w / (n2 * n2);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float v = c * r[3 + k];
            if (k == 0) v -= 2.f * w / n2;
            o[3 + k] = v * in;
        }
        L *= in;
    }
    L = warp_sum(L);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = L;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(d_loss, s);
    }
}

// ----------------------------------------------------------- optimiser
// Sixteen values per thread as four float4 loads, all in flight at once
// (g 16-byte aligned); block 0 also takes the scalar tail.
__global__ void __launch_bounds__(256) check_finite_kernel(const float *g, int64_t n, gs_train_state *st)
{
    const int64_t n4 = n / 4;
    const float4 *g4 = reinterpret_cast<const float4 *>(g);
    const int64_t q0 = (int64_t)blockIdx.x * blockDim.x * 4 + threadIdx.x;
    float4 q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = q0 + (int64_t)k * blockDim.x;
        q[k] = i < n4 ? g4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) bad |= !(isfinite(q[k].x) && isfinite(q[k].y) && isfinite(q[k].z) && isfinite(q[k].w));
    if (blockIdx.x == 0)
        for (int64_t i = 4 * n4 + threadIdx.x; i < n; i += blockDim.x) bad |= !isfinite(g[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) st->found_inf = 1;
}

template <int SHADOW>
__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, const gs_adam &hp,
                                         float lr, float bc1, float bc2, float inv)
{
    g *= inv;
    m = fmaf(hp.beta1, m, (1.f - hp.beta1) * g);
    v = fmaf(hp.beta2, v, (1.f - hp.beta2) * g * g);
    p = p - lr * (m / bc1) / (sqrtf(v / bc2) + hp.eps);
}

// The rate of the update with step number t (0-based): lr, or its
// exponential decay to lr * lr_final_ratio over decay_steps updates.
__device__ __forceinline__ float adam_rate(const gs_adam &hp, int t)
{
    if (hp.decay_steps <= 1) return hp.lr;
    const float last = (float)(hp.decay_steps - 1);
    const float f = fminf((float)t, last) / last;
    return hp.lr * exp2f(f * log2f(hp.lr_final_ratio));
}

// ADAM_GROUPS float4 groups of parameters per thread, strided by the block
// size so that every load is coalesced, all loaded before any is stored;
// block 0 also takes the scalar tail.  The arithmetic per parameter is
// adam_one's.  One group (4 parameters, 49 registers, many resident blocks)
// measured faster on the 3.3M-parameter table than four (130 registers).
#ifndef ADAM_GROUPS_N
#define ADAM_GROUPS_N 1  // one float4 per thread (49 registers) measured fastest after an L2 flush
#endif
#ifndef ADAM_MIN_BLOCKS
#define ADAM_MIN_BLOCKS 0
#endif
#if ADAM_MIN_BLOCKS > 0
#define ADAM_BOUNDS __launch_bounds__(256, ADAM_MIN_BLOCKS)
#else
#define ADAM_BOUNDS __launch_bounds__(256)
#endif
constexpr int ADAM_GROUPS = ADAM_GROUPS_N;

template <int SHADOW>
__global__ void ADAM_BOUNDS adam_kernel(float *__restrict__ p, float *__restrict__ g,
                                                   float *__restrict__ m, float *__restrict__ v,
                                                   int64_t n, gs_adam hp,
                                                   const gs_train_state *__restrict__ st,
                                                   void *__restrict__ shadow)
{
    const bool skip = st->found_inf != 0;
    // bias corrections 1 - b^t as -expm1(t log b): no cancellation when b is close to 1
    const int t = st->step + 1;
    const float bc1 = -expm1f((float)t * logf(hp.beta1));
    const float bc2 = -expm1f((float)t * logf(hp.beta2));
    const float inv = 1.f / st->loss_scale;
    const float lr = adam_rate(hp, st->step);
    const int64_t n4 = n / 4;
    float4 *p4 = reinterpret_cast<float4 *>(p), *g4 = reinterpret_cast<float4 *>(g);
    float4 *m4 = reinterpret_cast<float4 *>(m), *v4 = reinterpret_cast<float4 *>(v);
    const int64_t q0 = (int64_t)blockIdx.x * blockDim.x * ADAM_GROUPS + threadIdx.x;
    float4 gq[ADAM_GROUPS], mq[ADAM_GROUPS], vq[ADAM_GROUPS], pq[ADAM_GROUPS];
#pragma unroll
    for (int k = 0; k < ADAM_GROUPS; ++k) {
        const int64_t q = q0 + (int64_t)k * blockDim.x;
        if (q < n4) {
            gq[k] = g4[q];
            mq[k] = m4[q];
            vq[k] = v4[q];
            pq[k] = p4[q];
        }
    }
#pragma unroll
    for (int k = 0; k < ADAM_GROUPS; ++k) {
        const int64_t q = q0 + (int64_t)k * blockDim.x;
        if (q >= n4) continue;
        g4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (skip) continue;
        adam_one<SHADOW>(pq[k].x, gq[k].x, mq[k].x, vq[k].x, hp, lr, bc1, bc2, inv);
        adam_one<SHADOW>(pq[k].y, gq[k].y, mq[k].y, vq[k].y, hp, lr, bc1, bc2, inv);
        adam_one<SHADOW>(pq[k].z, gq[k].z, mq[k].z, vq[k].z, hp, lr, bc1, bc2, inv);
        adam_one<SHADOW>(pq[k].w, gq[k].w, mq[k].w, vq[k].w, hp, lr, bc1, bc2, inv);
        m4[q] = mq[k];
        v4[q] = vq[k];
        p4[q] = pq[k];
        if (SHADOW == GS_F16) {
            __half2 *h = reinterpret_cast<__half2 *>(shadow) + 2 * q;
            h[0] = __floats2half2_rn(pq[k].x, pq[k].y);
            h[1] = __floats2half2_rn(pq[k].z, pq[k].w);
        }
        if (SHADOW == GS_BF16) {
            __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(shadow) + 2 * q;
            h[0] = __floats2bfloat162_rn(pq[k].x, pq[k].y);
            h[1] = __floats2bfloat162_rn(pq[k].z, pq[k].w);
        }
    }
    if (blockIdx.x != 0) return;
    for (int64_t i = 4 * n4 + threadIdx.x; i < n; i += blockDim.x) {
        float gi = g[i], mi = m[i], vi = v[i], pi = p[i];
        g[i] = 0.f;
        if (skip) continue;
        adam_one<SHADOW>(pi, gi, mi, vi, hp, lr, bc1, bc2, inv);
        m[i] = mi;
        v[i] = vi;
        p[i] = pi;
        if (SHADOW == GS_F16) reinterpret_cast<__half *>(shadow)[i] = __float2half_rn(pi);
        if (SHADOW == GS_BF16) reinterpret_cast<__nv_bfloat16 *>(shadow)[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void state_advance_kernel(gs_train_state *st, int growth)
{
    if (st->found_inf) {
        st->loss_scale *= 0.5f;
        st->clean_steps = 0;
        st->found_inf = 0;
        return;
    }
    st->step += 1;
    st->clean_steps += 1;
    if (growth > 0 && st->clean_steps >= growth) {
        st->loss_scale *= 2.f;
        st->clean_steps = 0;
    }
}

}  // namespace gs3

using namespace gs3;

extern "C" const char *gs_last_error(void) { return g_err; }
extern "C" uint64_t gs_launch_count(void) { return gs3::launch_counter().load(); }
extern "C" int gs_version(void) { return (0 << 16) | 1; }

extern "C" int64_t ntc_hashgrid_entries(const gs_hashgrid *grid)
{
    GridParams P;
    int64_t total = 0;
    if (!grid_params(grid, P, total)) return -1;
    return total;
}

extern "C" gs_status ntc_encode_fwd(const float *mean, int64_t n, const gs_hashgrid *grid,
                                   const void *table, int table_dtype, void *enc, int enc_dtype,
                                   const uint32_t *order, gs_stream stream)
{
    GridParams g;
    int64_t total;
    GS_REQUIRE(grid_params(grid, g, total), "ntc_encode_fwd: invalid hash grid");
    GS_REQUIRE(table_dtype == GS_F16 || table_dtype == GS_F32, "ntc_encode_fwd: table dtype");
    GS_REQUIRE(enc_dtype == GS_F32 || enc_dtype == GS_BF16, "ntc_encode_fwd: enc dtype");
    GS_REQUIRE(n >= 0, "ntc_encode_fwd: negative n");
    if (n == 0) return GS_OK;
    GS_REQUIRE(mean && table && enc, "ntc_encode_fwd: null argument");
    const unsigned blocks = (unsigned)ceil_div(n, ENC_G);
    cudaStream_t s = as_stream(stream);
    note_launch();
    if (table_dtype == GS_F16 && enc_dtype == GS_F32)
        encode_fwd_kernel<__half, float><<<blocks, ENC_THREADS, 0, s>>>(mean, n, g, (const __half *)table,
                                                                        (float *)enc, order);
    else if (table_dtype == GS_F16)
        encode_fwd_kernel<__half, __nv_bfloat16><<<blocks, ENC_THREADS, 0, s>>>(
            mean, n, g, (const __half *)table, (__nv_bfloat16 *)enc, order);
    else if (enc_dtype == GS_F32)
        encode_fwd_kernel<float, float><<<blocks, ENC_THREADS, 0, s>>>(mean, n, g, (const float *)table,
                                                                      (float *)enc, order);
    else
        encode_fwd_kernel<float, __nv_bfloat16><<<blocks, ENC_THREADS, 0, s>>>(
            mean, n, g, (const float *)table, (__nv_bfloat16 *)enc, order);
    return launch_status("ntc_encode_fwd");
}

extern "C" gs_status ntc_encode_bwd(const float *mean, int64_t n, const gs_hashgrid *grid,
                                   const float *d_enc, float *d_table, const uint32_t *order,
                                   const int64_t *d_count, gs_stream stream)
{
    GridParams g;
    int64_t total;
    GS_REQUIRE(grid_params(grid, g, total), "ntc_encode_bwd: invalid hash grid");
    GS_REQUIRE(n >= 0, "ntc_encode_bwd: negative n");
    if (n == 0) return GS_OK;
    GS_REQUIRE(mean && d_enc && d_table, "ntc_encode_bwd: null argument");
    GS_REQUIRE(aligned(d_table, 8) && aligned(d_enc, 8), "ntc_encode_bwd: misaligned");
    GS_REQUIRE(d_count == nullptr || order, "ntc_encode_bwd: a count needs its row list (order)");
    note_launch();
    const dim3 blk(g.L, ENC_BWD_G);
    // over a list of unknown length: 16 blocks an SM stride over it
    const int64_t blocks = d_count ? std::min<int64_t>(ceil_div(n, ENC_BWD_G), (int64_t)num_sms() * 16)
                                   : ceil_div(n, ENC_BWD_G);
    encode_bwd_kernel<<<(unsigned)blocks, blk, 0, as_stream(stream)>>>(mean, n, g, d_enc, d_table, order, d_count);
    return launch_status("ntc_encode_bwd");
}

extern "C" gs_status ntc_active_rows(const float *d_raw7, int64_t n, uint32_t *rows, int64_t *d_count,
                                    gs_stream stream)
{
    GS_REQUIRE(n >= 0 && n <= (int64_t(1) << 32) - 1, "ntc_active_rows: n out of range");
    GS_REQUIRE(d_count, "ntc_active_rows: null count");
    GS_REQUIRE(n == 0 || (d_raw7 && rows), "ntc_active_rows: null argument");
    cudaStream_t s = as_stream(stream);
    cudaMemsetAsync(d_count, 0, sizeof(int64_t), s);
    if (n == 0) return launch_status("ntc_active_rows");
    note_launch();
    active_rows_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(d_raw7, n, rows,
                                                                 reinterpret_cast<unsigned long long *>(d_count));
    return launch_status("ntc_active_rows");
}

extern "C" size_t ntc_spatial_order_workspace_size(int64_t n)
{
    if (n < 0 || n > (int64_t(1) << 32) - 1) return 0;
    const size_t a = ((size_t)4 * std::max<int64_t>(n, 1) + 255) & ~size_t(255);
    return 3 * a + ((radix_sort_hist_words() * 4 + 255) & ~size_t(255));
}

extern "C" gs_status ntc_spatial_order(const float *mean, int64_t n, const gs_hashgrid *grid,
                                      uint32_t *order, void *ws, size_t ws_bytes, gs_stream stream)
{
    GridParams g;
    int64_t total;
    GS_REQUIRE(grid_params(grid, g, total), "ntc_spatial_order: invalid hash grid");
    GS_REQUIRE(n >= 0 && n <= (int64_t(1) << 32) - 1, "ntc_spatial_order: n out of range");
    if (n == 0) return GS_OK;
    GS_REQUIRE(mean && order && ws, "ntc_spatial_order: null argument");
    GS_REQUIRE(aligned(ws, 256), "ntc_spatial_order: workspace must be 256-byte aligned");
    const size_t need = ntc_spatial_order_workspace_size(n);
    GS_REQUIRE(ws_bytes >= need, "ntc_spatial_order: workspace too small (%zu < %zu)", ws_bytes, need);
    const size_t a = ((size_t)4 * n + 255) & ~size_t(255);
    char *w = reinterpret_cast<char *>(ws);
    // the values start in `order` and end there: 30 key bits take four passes
    uint32_t *k[2] = {reinterpret_cast<uint32_t *>(w), reinterpret_cast<uint32_t *>(w + a)};
    uint32_t *v[2] = {order, reinterpret_cast<uint32_t *>(w + 2 * a)};
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + 3 * a);
    cudaStream_t s = as_stream(stream);
    note_launch();
    morton_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(mean, n, g, k[0], v[0]);
    int cur = 0;
    gs_status e = radix_sort_pairs(k, v, n, 30, hist, cur, s);
    if (e != GS_OK) return e;
    if (cur != 0) cudaMemcpyAsync(order, v[cur], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    return launch_status("ntc_spatial_order");
}

extern "C" gs_status ntc_mlp_fwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w,
                                float *raw7, gs_stream stream)
{
    GS_REQUIRE(w && n >= 0, "ntc_mlp_fwd: null weights or negative n");
    GS_REQUIRE(enc_dtype == GS_F32 || enc_dtype == GS_BF16, "ntc_mlp_fwd: enc dtype");
    if (n == 0) return GS_OK;
    GS_REQUIRE(enc && raw7, "ntc_mlp_fwd: null argument");
    if (w->precision == GS_MLP_BF16) return mlp_tc_fwd(enc, enc_dtype, n, w, raw7, as_stream(stream));
    GS_REQUIRE(w->precision == GS_MLP_FP32 && w->w_f32, "ntc_mlp_fwd: bad precision / weights");
    int blocks = (int)ceil_div(n, 128);
    cudaStream_t s = as_stream(stream);
    note_launch();
    if (enc_dtype == GS_F32)
        mlp_fwd_simt_kernel<float><<<blocks, 128, 0, s>>>((const float *)enc, n, w->w_f32, raw7);
    else
        mlp_fwd_simt_kernel<__nv_bfloat16><<<blocks, 128, 0, s>>>((const __nv_bfloat16 *)enc, n, w->w_f32,
                                                                  raw7);
    return launch_status("ntc_mlp_fwd");
}

extern "C" gs_status ntc_mlp_bwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w,
                                const float *d_raw7, const float *d_scale, float *dW, float *d_enc,
                                const uint32_t *rows, const int64_t *d_rows, gs_stream stream)
{
    GS_REQUIRE(w && dW && n >= 0, "ntc_mlp_bwd: null weights or negative n");
    GS_REQUIRE(enc_dtype == GS_F32 || enc_dtype == GS_BF16, "ntc_mlp_bwd: enc dtype");
    GS_REQUIRE((rows == nullptr) == (d_rows == nullptr), "ntc_mlp_bwd: rows and d_rows go together");
    if (n == 0) return GS_OK;
    GS_REQUIRE(enc && d_raw7, "ntc_mlp_bwd: null argument");
    if (w->precision == GS_MLP_BF16)
        return mlp_tc_bwd(enc, enc_dtype, n, w, d_raw7, d_scale, dW, d_enc, rows, d_rows, as_stream(stream));
    GS_REQUIRE(w->precision == GS_MLP_FP32 && w->w_f32, "ntc_mlp_bwd: bad precision / weights");
    cudaStream_t s = as_stream(stream);
    int blocks = (int)std::min<int64_t>(ceil_div(n, MB_ROWS), 2 * num_sms());
    if (enc_dtype == GS_F32) {
        set_smem_limit((const void *)mlp_bwd_simt_kernel<float>, (int)MB_SMEM, s);
        note_launch();
        mlp_bwd_simt_kernel<float><<<blocks, MB_ROWS, MB_SMEM, s>>>((const float *)enc, n, w->w_f32,
                                                                    d_raw7, d_scale, dW, d_enc, rows, d_rows);
    } else {
        set_smem_limit((const void *)mlp_bwd_simt_kernel<__nv_bfloat16>, (int)MB_SMEM, s);
        note_launch();
        mlp_bwd_simt_kernel<__nv_bfloat16><<<blocks, MB_ROWS, MB_SMEM, s>>>(
            (const __nv_bfloat16 *)enc, n, w->w_f32, d_raw7, d_scale, dW, d_enc, rows, d_rows);
    }
    return launch_status("ntc_mlp_bwd");
}

extern "C" gs_status ntc_apply(const float *mean, const float *quat, const float *raw7, int64_t n,
                              const float *aabb, int order, float *mean_out, float *quat_out,
                              gs_stream stream)
{
    GS_REQUIRE(order == 0 || order == 1, "ntc_apply: order must be 0 or 1");
    GS_REQUIRE(n >= 0, "ntc_apply: negative n");
    if (n == 0) return GS_OK;
    GS_REQUIRE(mean && quat && raw7 && aabb && mean_out && quat_out, "ntc_apply: null argument");
    GS_REQUIRE(aligned(quat, 16) && aligned(quat_out, 16), "ntc_apply: quaternions misaligned");
    Box b = Box::from(aabb);
    note_launch();
    apply_kernel<<<(int)ceil_div(n, 256), 256, 0, as_stream(stream)>>>(mean, quat, raw7, n, b, order,
                                                                       mean_out, quat_out);
    return launch_status("ntc_apply");
}

extern "C" gs_status ntc_apply_bwd(const float *mean, const float *quat, const float *raw7,
                                  int64_t n, const float *aabb, int order, const float *d_mean_out,
                                  const float *d_quat_out, float *d_raw7, gs_stream stream)
{
    GS_REQUIRE(order == 0 || order == 1, "ntc_apply_bwd: order must be 0 or 1");
    GS_REQUIRE(n >= 0, "ntc_apply_bwd: negative n");
    if (n == 0) return GS_OK;
    GS_REQUIRE(mean && quat && raw7 && aabb && d_mean_out && d_quat_out && d_raw7,
               "ntc_apply_bwd: null argument");
    GS_REQUIRE(aligned(quat, 16) && aligned(d_quat_out, 16), "ntc_apply_bwd: misaligned");
    Box b = Box::from(aabb);
    note_launch();
    apply_bwd_kernel<<<(int)ceil_div(n, 256), 256, 0, as_stream(stream)>>>(
        mean, quat, raw7, n, b, order, d_mean_out, d_quat_out, d_raw7);
    return launch_status("ntc_apply_bwd");
}

extern "C" gs_status ntc_warmup_loss(const float *raw7, int64_t n, float *d_raw7, float *d_loss,
                                    gs_stream stream)
{
    GS_REQUIRE(raw7 && d_raw7 && d_loss && n > 0, "ntc_warmup_loss: bad argument");
    cudaStream_t s = as_stream(stream);
    cudaMemsetAsync(d_loss, 0, sizeof(float), s);
    note_launch();
    warmup_kernel<<<(int)ceil_div(n, 256), 256, 0, s>>>(raw7, n, d_raw7, d_loss);
    return launch_status("ntc_warmup_loss");
}

extern "C" gs_status gs_check_finite(const float *g, int64_t n, gs_train_state *d_state,
                                     gs_stream stream)
{
    GS_REQUIRE(d_state && n >= 0, "gs_check_finite: null state or negative n");
    if (n == 0) return GS_OK;
    GS_REQUIRE(g, "gs_check_finite: null argument");
    GS_REQUIRE(aligned(g, 16), "gs_check_finite: g must be 16-byte aligned");
    const int blocks = (int)std::max<int64_t>(ceil_div(n / 4, 256 * 4), 1);
    note_launch();
    check_finite_kernel<<<blocks, 256, 0, as_stream(stream)>>>(g, n, d_state);
    return launch_status("gs_check_finite");
}

extern "C" gs_status adam_step(float *p, float *g, float *m, float *v, int64_t n, const gs_adam *hp,
                               const gs_train_state *d_state, void *shadow, int shadow_dtype,
                               gs_stream stream)
{
    GS_REQUIRE(hp && d_state && n >= 0, "adam_step: null hyper-parameters / state or negative n");
    GS_REQUIRE(shadow == nullptr || shadow_dtype == GS_F16 || shadow_dtype == GS_BF16,
               "adam_step: shadow dtype must be GS_F16 or GS_BF16");
    GS_REQUIRE(hp->decay_steps <= 1 || hp->lr_final_ratio > 0.f,
               "adam_step: lr_final_ratio must be positive when the rate decays");
    if (n == 0) return GS_OK;
    GS_REQUIRE(p && g && m && v, "adam_step: null argument");
    GS_REQUIRE(aligned(p, 16) && aligned(g, 16) && aligned(m, 16) && aligned(v, 16) &&
                   (shadow == nullptr || aligned(shadow, 8)),
               "adam_step: arrays must be 16-byte aligned (shadow 8)");
    const int blocks = (int)std::max<int64_t>(ceil_div(n / 4, 256 * ADAM_GROUPS), 1);
    cudaStream_t s = as_stream(stream);
    note_launch();
    if (!shadow)
        adam_kernel<GS_NONE><<<blocks, 256, 0, s>>>(p, g, m, v, n, *hp, d_state, nullptr);
    else if (shadow_dtype == GS_F16)
        adam_kernel<GS_F16><<<blocks, 256, 0, s>>>(p, g, m, v, n, *hp, d_state, shadow);
    else
        adam_kernel<GS_BF16><<<blocks, 256, 0, s>>>(p, g, m, v, n, *hp, d_state, shadow);
    return launch_status("adam_step");
}

extern "C" gs_status gs_train_state_advance(gs_train_state *d_state, int growth_interval,
                                            gs_stream stream)
{
    GS_REQUIRE(d_state, "gs_train_state_advance: null state");
    note_launch();
    state_advance_kernel<<<1, 1, 0, as_stream(stream)>>>(d_state, growth_interval);
    return launch_status("gs_train_state_advance");
}

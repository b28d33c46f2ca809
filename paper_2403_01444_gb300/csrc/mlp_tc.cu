// BF16 tensor-core MLP of the transformation cache (Section 4.1, Eq. 5):
// 32 -> 64 -> 64 -> 7 with ReLU, no biases, BF16 x BF16 -> FP32 on tcgen05.
//
// One CTA of 128 threads owns a tile of 128 Gaussians (the M = 128 rows of
// every MMA); thread t holds row t, which is TMEM lane t.  Operands are staged
// in shared memory in the K-major no-swizzle layout, the accumulator lives in
// TMEM, thread 0 issues the MMAs and an mbarrier tracks their completion
// (bounded waits).  Forward: two chained MMAs with ReLU epilogues; the 64 -> 7
// output layer runs in FP32 in the second epilogue (448 FMAs per row), so
// the translation and rotation carry no BF16 rounding of the last layer.
// Backward (recomputing the forward from the encoding):
//   dH2 = (G W3) . relu'(H2),  dH1 = (dH2 W2) . relu'(H1),  d_enc = dH1 W1
//   dW2 = dH2^T H1, dW1 = dH1^T enc, dW3 = G^T H2
// The three weight gradients are contractions over the Gaussians; they are
// stacked into two M = 128 MMAs over K = 128 rows of the tile and accumulate
// in TMEM across all tiles a CTA owns, then one FP32 atomic per weight per CTA.
#include "ntc.cuh"
#include "tc.cuh"

#include <atomic>

namespace gs3 {
using namespace tc;
typedef __nv_bfloat16 bf16;

__device__ int g_tc_timeouts;

constexpr int TM = 128;

struct FwdSmem {
    bf16 a1[TM * 32];   // encoding tile, K = 32
    bf16 a2[TM * 64];   // hidden activations, K = 64
    bf16 w1[64 * 32];   // B operands [N][K]: W1 as stored [out][in]
    bf16 w2[64 * 64];
    float w3f[7 * 64];  // output layer, FP32 (applied in the epilogue)
    unsigned long long mbar;
    uint32_t tmem;
};

// The backward's buffers are shared between the stages of a tile where
// their lives do not overlap, so that two CTAs fit on an SM (about 110 KB
// each): a1 holds the encoding (stage 1) then the output gradient G
// (stage 2); hbuf holds H1, dH2 and dH1 in turn; AT holds [H2^T; dH2^T]
// until the stage-3 MMAs (dW3 among them) have read it, then [dH1^T; dH2^T].
struct BwdSmem {
    bf16 AT[128 * TM];  // A of the weight-gradient MMAs; K = tile rows
    bf16 BT[112 * TM];  // rows: H1^T (0..63), enc^T (64..95), G^T (96..111)
    bf16 a1[TM * 32];   // enc (K = 32), then G (K = 16)
    bf16 hbuf[TM * 64]; // H1, dH2, dH1 (K = 64)
    bf16 w1[64 * 32];   // [out][in]
    bf16 w2[64 * 64];
    bf16 w3t[64 * 16];  // [hidden][out], out padded to 16
    bf16 w2t[64 * 64];  // [in][out]
    bf16 w1t[32 * 64];  // [in][hidden]
    unsigned long long mbar;
    uint32_t tmem;
};
// two CTAs an SM: 228 KB of shared memory, 1 KB reserved per CTA, 1 KB of alignment slack
static_assert(2 * (sizeof(BwdSmem) + 1024 + 1024) <= 228 * 1024, "backward tile buffers too large");

// Arguments of the MLP kernels.  The standalone MLP reads encodings and
// writes raw outputs; the fused cache kernels (FUSED = true) also encode the
// means from the FP16 hash table and apply the transformation (forward), or
// take the transformation's backward and scatter into the table (backward).
struct TcParams {
    const void *enc;
    int64_t n;
    const bf16 *w;
    const float *w3f;   // FP32 output-layer weights (forward)
    float *raw7;
    const float *d_raw7, *d_scale;
    float *dW, *d_enc;
    // fused cache path
    const float *mean, *quat;
    GridParams grid;
    const __half *table;
    bf16 *enc_save;
    const float *raw7_in;
    float *mean_out, *quat_out;
    const float *d_mean_out, *d_quat_out;
    float *d_table;
    Box box;
    int order;
    uint32_t wait_tries;  // polls of an MMA-completion wait before giving up
    // reverse over a row list: slot k of the work is row rows[k], k < *d_rows
    const uint32_t *rows;
    const int64_t *d_rows;
};

template <typename T>
__device__ __forceinline__ T *aligned_smem(unsigned char *raw)
{
    uintptr_t p = reinterpret_cast<uintptr_t>(raw);
    p = (p + 1023) & ~uintptr_t(1023);
    return reinterpret_cast<T *>(p);
}

__device__ __forceinline__ void load_row32(const float *enc, int64_t row, int64_t n, float *v)
{
    if (row < n) {
        const float4 *p = reinterpret_cast<const float4 *>(enc + row * 32);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float4 q = p[c];
            v[4 * c] = q.x;
            v[4 * c + 1] = q.y;
            v[4 * c + 2] = q.z;
            v[4 * c + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 0.f;
    }
}
__device__ __forceinline__ void load_row32(const bf16 *enc, int64_t row, int64_t n, float *v)
{
    if (row < n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(enc + row * 32);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint4 q = p[c];
            const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 f = __bfloat1622float2(h[j]);
                v[8 * c + 2 * j] = f.x;
                v[8 * c + 2 * j + 1] = f.y;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 0.f;
    }
}

// Hash encoding of one mean (Section 4.1), FP16 features, FP32 sums: the
// arithmetic of encode_fwd_kernel, so the values are the same.
__device__ __forceinline__ void encode_row(const TcParams &p, int64_t row, float *v)
{
    if (row >= p.n) {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = 0.f;
        return;
    }
    float3 m = make_float3(p.mean[3 * row], p.mean[3 * row + 1], p.mean[3 * row + 2]);
    const __half2 *tab = reinterpret_cast<const __half2 *>(p.table);
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        float f0 = 0.f, f1 = 0.f;
        if (l < p.grid.L) {
            uint32_t idx[8];
            float w8[8];
            level_corners(p.grid, l, m, idx, w8);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float2 t = __half22float2(tab[idx[c]]);
                f0 = fmaf(w8[c], t.x, f0);
                f1 = fmaf(w8[c], t.y, f1);
            }
        }
        v[2 * l] = f0;
        v[2 * l + 1] = f1;
    }
}

// Trilinear-weighted scatter of one row's encoding gradient into the table.
__device__ __forceinline__ void scatter_row(const TcParams &p, int64_t row, const float *g)
{
    float3 m = make_float3(p.mean[3 * row], p.mean[3 * row + 1], p.mean[3 * row + 2]);
    float2 *dt = reinterpret_cast<float2 *>(p.d_table);
#pragma unroll
    for (int l = 0; l < 16; ++l) {
        if (l >= p.grid.L) break;
        float gx = g[2 * l], gy = g[2 * l + 1];
        if (gx == 0.f && gy == 0.f) continue;
        uint32_t idx[8];
        float w8[8];
        level_corners(p.grid, l, m, idx, w8);
#pragma unroll
        for (int c = 0; c < 8; ++c) atomicAdd(dt + idx[c], make_float2(w8[c] * gx, w8[c] * gy));
    }
}

// Transformation of one Gaussian (Section 4.1): the arithmetic of apply_kernel.
__device__ __forceinline__ void apply_row(const TcParams &p, int64_t row, const float *r)
{
    float3 m = make_float3(p.mean[3 * row], p.mean[3 * row + 1], p.mean[3 * row + 2]);
    float4 qn = qnormalize(reinterpret_cast<const float4 *>(p.quat)[row]);
    if (!p.box.inside(m)) {
        p.mean_out[3 * row] = m.x;
        p.mean_out[3 * row + 1] = m.y;
        p.mean_out[3 * row + 2] = m.z;
        reinterpret_cast<float4 *>(p.quat_out)[row] = qn;
        return;
    }
    float4 dq = qnormalize(make_float4(r[3], r[4], r[5], r[6]));
    p.mean_out[3 * row] = m.x + r[0];
    p.mean_out[3 * row + 1] = m.y + r[1];
    p.mean_out[3 * row + 2] = m.z + r[2];
    reinterpret_cast<float4 *>(p.quat_out)[row] = p.order == 0 ? qmul(qn, dq) : qmul(dq, qn);
}

// Reverse of apply_row wrt the raw outputs (the arithmetic of apply_bwd_kernel).
__device__ __forceinline__ void apply_bwd_row(const TcParams &p, int64_t row, float *g)
{
    float3 m = make_float3(p.mean[3 * row], p.mean[3 * row + 1], p.mean[3 * row + 2]);
    if (!p.box.inside(m)) {
#pragma unroll
        for (int k = 0; k < 7; ++k) g[k] = 0.f;
        return;
    }
    g[0] = p.d_mean_out[3 * row];
    g[1] = p.d_mean_out[3 * row + 1];
    g[2] = p.d_mean_out[3 * row + 2];
    float4 qn = qnormalize(reinterpret_cast<const float4 *>(p.quat)[row]);
    const float *r = p.raw7_in + 7 * row;
    float4 gq = reinterpret_cast<const float4 *>(p.d_quat_out)[row];
    float4 gd = p.order == 0 ? qmul_left_T(qn, gq) : qmul_right_T(qn, gq);
    float4 d = qnormalize_bwd(make_float4(r[3], r[4], r[5], r[6]), gd);
    g[3] = d.x;
    g[4] = d.y;
    g[5] = d.z;
    g[6] = d.w;
}

// W1 | W2 | W3 (bf16, [out][in] row-major) into K-major B operands.
// The BF16 weights (W1 [64][32], W2 [64][64], W3 [7][64] as stored, 6592
// values) staged in shared memory 16 bytes a load, every load of a thread
// issued before its stores: K-major W1 and W2 (the B operands of the forward
// products) and, for the backward, K-major W1^T, W2^T and W3^T (outputs
// padded to 16 with zeros).
template <bool BWD>
__device__ __forceinline__ void stage_weights(const bf16 *w, bf16 *w1, bf16 *w2, bf16 *w3t, bf16 *w2t,
                                              bf16 *w1t)
{
    constexpr int NQ = 6592 / 8;
    constexpr int PER = (NQ + TM - 1) / TM;
    const uint4 *src = reinterpret_cast<const uint4 *>(w);
    uint4 q[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int k = threadIdx.x + i * TM;
        q[i] = k < NQ ? src[k] : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int k = threadIdx.x + i * TM;
        if (k >= NQ) continue;
        const int e0 = 8 * k;
        const bf16 *h = reinterpret_cast<const bf16 *>(&q[i]);
        if (e0 < 2048) {
            const int j = e0 >> 5, i0 = e0 & 31;  // W1[j][i0 .. i0 + 7]
            *reinterpret_cast<uint4 *>(w1 + kmajor_off(j, i0, 32)) = q[i];
            if (BWD) {
#pragma unroll
                for (int c = 0; c < 8; ++c) w1t[kmajor_off(i0 + c, j, 64)] = h[c];
            }
        } else if (e0 < 6144) {
            const int f = e0 - 2048, j = f >> 6, k0 = f & 63;  // W2[j][k0 .. k0 + 7]
            *reinterpret_cast<uint4 *>(w2 + kmajor_off(j, k0, 64)) = q[i];
            if (BWD) {
#pragma unroll
                for (int c = 0; c < 8; ++c) w2t[kmajor_off(k0 + c, j, 64)] = h[c];
            }
        } else if (BWD) {
            const int f = e0 - 6144, o = f >> 6, j0 = f & 63;  // W3[o][j0 .. j0 + 7]
#pragma unroll
            for (int c = 0; c < 8; ++c) w3t[kmajor_off(j0 + c, o, 16)] = h[c];
        }
    }
    if (BWD) {
        for (int e = threadIdx.x; e < 64 * 9; e += TM) w3t[kmajor_off(e / 9, 7 + e % 9, 16)] = __float2bfloat16(0.f);
    }
}

// All threads wait for the MMA batch; returns false (block-uniformly) on timeout.
__device__ __forceinline__ bool wait_mma(uint32_t mbar, uint32_t &phase, uint32_t tries)
{
    bool ok = mbar_wait(mbar, phase, tries);
    phase ^= 1u;
    ok = __syncthreads_and(ok);
    fence_after_sync();
    return ok;
}

// Staged operands written by all threads -> visible to the tensor core.
__device__ __forceinline__ void publish_smem()
{
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
}

template <typename ET, bool FUSED>
__global__ void __launch_bounds__(TM, 4) mlp_tc_fwd_kernel(TcParams p)
{
    extern __shared__ unsigned char smem_raw[];
    FwdSmem &S = *aligned_smem<FwdSmem>(smem_raw);
    const ET *enc = reinterpret_cast<const ET *>(p.enc);
    const int64_t n = p.n;
    const bf16 *w = p.w;
    float *raw7 = p.raw7;
    const int t = threadIdx.x, warp = t >> 5;
    stage_weights<false>(w, S.w1, S.w2, nullptr, nullptr, nullptr);
    if ((reinterpret_cast<uintptr_t>(p.w3f) & 15) == 0) {
        if (t < 7 * 64 / 4) reinterpret_cast<float4 *>(S.w3f)[t] = reinterpret_cast<const float4 *>(p.w3f)[t];
    } else {
        for (int e = t; e < 7 * 64; e += TM) S.w3f[e] = p.w3f[e];
    }
    const uint32_t mbar = smem_u32(&S.mbar);
    if (t == 0) mbar_init(mbar, 1);
    if (warp == 0) {
        tmem_alloc(smem_u32(&S.tmem), 64);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tm = S.tmem;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    const uint32_t id64 = idesc_bf16_f32(128, 64);
    const uint32_t a1 = smem_u32(S.a1), a2 = smem_u32(S.a2);
    const uint32_t w1 = smem_u32(S.w1), w2 = smem_u32(S.w2);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (n + TM - 1) / TM;
    int64_t tile = blockIdx.x;
    for (; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t row = tile * TM + t;
        float v[64];
        if (FUSED) {
            encode_row(p, row, v);
            if (row < n) {
                uint4 *dst = reinterpret_cast<uint4 *>(p.enc_save + row * 32);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    dst[c] = make_uint4(pack_bf16x2(v[8 * c], v[8 * c + 1]), pack_bf16x2(v[8 * c + 2], v[8 * c + 3]),
                                        pack_bf16x2(v[8 * c + 4], v[8 * c + 5]), pack_bf16x2(v[8 * c + 6], v[8 * c + 7]));
            }
        } else {
            load_row32(enc, row, n, v);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) st_chunk8(S.a1, t, 8 * c, 32, v + 8 * c);
        publish_smem();
        if (t == 0) {
            fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                mma_bf16(tm, desc_kmajor(a1 + 256 * ks, 128, 512), desc_kmajor(w1 + 256 * ks, 128, 512),
                         id64, ks > 0);
            mma_commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase, p.wait_tries))) break;
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16(tm + lane + 16 * c, v + 16 * c);
#pragma unroll
        for (int k = 0; k < 64; ++k) v[k] = fmaxf(v[k], 0.f);
#pragma unroll
        for (int c = 0; c < 8; ++c) st_chunk8(S.a2, t, 8 * c, 64, v + 8 * c);
        publish_smem();
        if (t == 0) {
            fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(tm, desc_kmajor(a2 + 256 * ks, 128, 1024), desc_kmajor(w2 + 256 * ks, 128, 1024),
                         id64, ks > 0);
            mma_commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase, p.wait_tries))) break;
        // output layer (64 -> 7) in FP32 on the FP32 accumulator, 16 columns
        // of H2 at a time: the raw translation and rotation carry no BF16
        // rounding of the last layer
        float o7[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            tmem_ld16(tm + lane + 16 * c, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float h = fmaxf(v[k], 0.f);
#pragma unroll
                for (int q = 0; q < 7; ++q) o7[q] = fmaf(S.w3f[q * 64 + 16 * c + k], h, o7[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 7; ++q) v[q] = o7[q];
        if (row < n) {
#pragma unroll
            for (int q = 0; q < 7; ++q) raw7[row * 7 + q] = v[q];
            if (FUSED) apply_row(p, row, v);
        }
        fence_before_sync();
        __syncthreads();
    }
    if (!ok) {
        // A wait gave up.  The MMA batch it waited for may still be running:
        // wait for it (bounded) before the TMEM is released.  Every row this
        // block did not finish is then written non-finite, so the Gaussian is
        // culled by the projection and the step's non-finite gradient check
        // skips the update, as for an overflow.
        mbar_wait(mbar, phase ^ 1u, kWaitTries);
        const float nan = __int_as_float(0x7fc00000);
        for (; tile < ntiles; tile += gridDim.x) {
            const int64_t row = tile * TM + t;
            if (row >= n) continue;
#pragma unroll
            for (int q = 0; q < 7; ++q) raw7[row * 7 + q] = nan;
            if (FUSED) {
#pragma unroll
                for (int q = 0; q < 3; ++q) p.mean_out[row * 3 + q] = nan;
#pragma unroll
                for (int q = 0; q < 4; ++q) p.quat_out[row * 4 + q] = nan;
            }
        }
        if (t == 0) atomicAdd(&g_tc_timeouts, 1);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tm, 64);
}

template <typename ET, bool FUSED>
__global__ void __launch_bounds__(TM, 2) mlp_tc_bwd_kernel(TcParams p)
{
    extern __shared__ unsigned char smem_raw[];
    BwdSmem &S = *aligned_smem<BwdSmem>(smem_raw);
    const ET *enc = reinterpret_cast<const ET *>(p.enc);
    const int64_t n = p.n;
    const bf16 *w = p.w;
    const float *d_raw7 = p.d_raw7, *d_scale = p.d_scale;
    float *dW = p.dW, *d_enc = p.d_enc;
    const int t = threadIdx.x, warp = t >> 5;
    stage_weights<true>(w, S.w1, S.w2, S.w3t, S.w2t, S.w1t);
    const uint32_t mbar = smem_u32(&S.mbar);
    if (t == 0) mbar_init(mbar, 1);
    if (warp == 0) {
        tmem_alloc(smem_u32(&S.tmem), 256);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tm = S.tmem;
    const uint32_t D0 = tm, D1 = tm + 64, DW = tm + 128, DW3 = tm + 224;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    const uint32_t id64 = idesc_bf16_f32(128, 64), id32 = idesc_bf16_f32(128, 32);
    const uint32_t id96 = idesc_bf16_f32(128, 96), id16 = idesc_bf16_f32(128, 16);
    const uint32_t sAT = smem_u32(S.AT), sBT = smem_u32(S.BT);
    const uint32_t sa1 = smem_u32(S.a1), sga = sa1;
    const uint32_t sh1 = smem_u32(S.hbuf), sg2 = sh1, sg1 = sh1;
    const uint32_t sw1 = smem_u32(S.w1), sw2 = smem_u32(S.w2), sw3t = smem_u32(S.w3t);
    const uint32_t sw2t = smem_u32(S.w2t), sw1t = smem_u32(S.w1t);
    const float scale = d_scale ? *d_scale : 1.f;
    uint32_t phase = 0;
    bool ok = true;
    int done_tiles = 0;
    const int64_t nslots = p.d_rows ? *p.d_rows : n;
    const int64_t ntiles = (nslots + TM - 1) / TM;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        // a slot past the list is row n: every use below checks row < n
        const int64_t slot = tile * TM + t;
        const int64_t row = slot < nslots ? (p.rows ? (int64_t)p.rows[slot] : slot) : n;
        float v[64];
        // ---- stage the encoding and the scaled output gradient
        load_row32(enc, row, n, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) st_chunk8(S.a1, t, 8 * c, 32, v + 8 * c);
#pragma unroll
        for (int i = 0; i < 32; ++i) S.BT[kmajor_off(64 + i, t, TM)] = __float2bfloat16_rn(v[i]);
        float g[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) g[q] = 0.f;
        if (row < n) {
            if (FUSED) {
                apply_bwd_row(p, row, g);
            } else {
#pragma unroll
                for (int q = 0; q < 7; ++q) g[q] = d_raw7[row * 7 + q];
            }
#pragma unroll
            for (int q = 0; q < 7; ++q) g[q] *= scale;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) S.BT[kmajor_off(96 + q, t, TM)] = __float2bfloat16_rn(g[q]);
        publish_smem();
        if (t == 0) {
            fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
                mma_bf16(D0, desc_kmajor(sa1 + 256 * ks, 128, 512), desc_kmajor(sw1 + 256 * ks, 128, 512),
                         id64, ks > 0);
            mma_commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase, p.wait_tries))) break;
        // ---- H1 = relu(enc W1^T)
        uint32_t m1lo = 0, m1hi = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16(D0 + lane + 16 * c, v + 16 * c);
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            bool pos = v[k] > 0.f;
            v[k] = pos ? v[k] : 0.f;
            if (k < 32) m1lo |= (uint32_t)pos << k;
            else m1hi |= (uint32_t)pos << (k - 32);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) st_chunk8(S.hbuf, t, 8 * c, 64, v + 8 * c);
        // G over the encoding, which stage 1 has read
        st_chunk8(S.a1, t, 0, 16, g);
        st_chunk8(S.a1, t, 8, 16, g + 8);
#pragma unroll
        for (int j = 0; j < 64; ++j) S.BT[kmajor_off(j, t, TM)] = __float2bfloat16_rn(v[j]);
        publish_smem();
        if (t == 0) {
            fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(D0, desc_kmajor(sh1 + 256 * ks, 128, 1024), desc_kmajor(sw2 + 256 * ks, 128, 1024),
                         id64, ks > 0);
            mma_bf16(D1, desc_kmajor(sga, 128, 256), desc_kmajor(sw3t, 128, 256), id64, 0);
            mma_commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase, p.wait_tries))) break;
        // ---- H2 = relu(H1 W2^T); dH2 = (G W3) . relu'(H2)
        uint32_t m2lo = 0, m2hi = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16(D0 + lane + 16 * c, v + 16 * c);
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            bool pos = v[k] > 0.f;
            v[k] = pos ? v[k] : 0.f;
            if (k < 32) m2lo |= (uint32_t)pos << k;
            else m2hi |= (uint32_t)pos << (k - 32);
        }
#pragma unroll
        for (int j = 0; j < 64; ++j) S.AT[kmajor_off(j, t, TM)] = __float2bfloat16_rn(v[j]);
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16(D1 + lane + 16 * c, v + 16 * c);
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            bool pos = k < 32 ? ((m2lo >> k) & 1u) : ((m2hi >> (k - 32)) & 1u);
            v[k] = pos ? v[k] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) st_chunk8(S.hbuf, t, 8 * c, 64, v + 8 * c);
#pragma unroll
        for (int j = 0; j < 64; ++j) S.AT[kmajor_off(64 + j, t, TM)] = __float2bfloat16_rn(v[j]);
        publish_smem();
        if (t == 0) {
            fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(D0, desc_kmajor(sg2 + 256 * ks, 128, 1024), desc_kmajor(sw2t + 256 * ks, 128, 1024),
                         id64, ks > 0);
            // dW3^T += H2^T G (rows 64..127 of this product are unused)
            const uint32_t acc0 = done_tiles > 0 ? 1u : 0u;
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
                mma_bf16(DW3, desc_kmajor(sAT + 256 * ks, 128, 2048),
                         desc_kmajor(sBT + 12 * 2048 + 256 * ks, 128, 2048), id16, ks > 0 ? 1u : acc0);
            mma_commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase, p.wait_tries))) break;
        // ---- dH1 = (dH2 W2) . relu'(H1)
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16(D0 + lane + 16 * c, v + 16 * c);
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            bool pos = k < 32 ? ((m1lo >> k) & 1u) : ((m1hi >> (k - 32)) & 1u);
            v[k] = pos ? v[k] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) st_chunk8(S.hbuf, t, 8 * c, 64, v + 8 * c);
        // dH1^T over H2^T, which the stage-3 MMAs have read
#pragma unroll
        for (int j = 0; j < 64; ++j) S.AT[kmajor_off(j, t, TM)] = __float2bfloat16_rn(v[j]);
        publish_smem();
        if (t == 0) {
            fence_after_sync();
            // d_enc = dH1 W1
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(D0, desc_kmajor(sg1 + 256 * ks, 128, 1024), desc_kmajor(sw1t + 256 * ks, 128, 1024),
                         id32, ks > 0);
            // [. | dW1 ; dW2 | .] += [dH1^T ; dH2^T] [H1 | enc], K = the tile's rows
            const uint32_t acc0 = done_tiles > 0 ? 1u : 0u;
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
                mma_bf16(DW, desc_kmajor(sAT + 256 * ks, 128, 2048), desc_kmajor(sBT + 256 * ks, 128, 2048),
                         id96, ks > 0 ? 1u : acc0);
            mma_commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase, p.wait_tries))) break;
        if (FUSED) {
            tmem_ld16(D0 + lane, v);
            tmem_ld16(D0 + lane + 16, v + 16);
            if (row < n) scatter_row(p, row, v);
        } else if (d_enc) {
            tmem_ld16(D0 + lane, v);
            tmem_ld16(D0 + lane + 16, v + 16);
            if (row < n) {
                float4 *o = reinterpret_cast<float4 *>(d_enc + row * 32);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    o[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
            }
        }
        ++done_tiles;
        fence_before_sync();
        __syncthreads();
    }
    if (ok && done_tiles > 0) {
        // one FP32 atomic per weight per CTA, four at a time where dW is
        // 16-byte aligned (the rows of dW1 and dW2 are contiguous)
        const bool v4 = (reinterpret_cast<uintptr_t>(dW) & 15) == 0;
        auto add16 = [&](float *dst, const float *v) {
            if (v4) {
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    atomicAdd(reinterpret_cast<float4 *>(dst + i), make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]));
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(dst + i, v[i]);
            }
        };
        float v[16];
        if (warp < 2) {
            const int j = t;  // dW1 row (hidden unit) j, dW3 column j
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                tmem_ld16(DW + lane + 64 + 16 * c, v);
                add16(dW + j * 32 + 16 * c, v);
            }
            tmem_ld16(DW3 + lane, v);
#pragma unroll
            for (int o = 0; o < 7; ++o) atomicAdd(dW + 6144 + o * 64 + j, v[o]);
        } else {
            const int j = t - 64;  // dW2 row (output unit) j
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                tmem_ld16(DW + lane + 16 * c, v);
                add16(dW + 2048 + j * 64 + 16 * c, v);
            }
        }
    }
    if (!ok) {
        // A wait gave up: wait (bounded) for the MMA batch still in flight
        // before the TMEM is released, and make the weight gradient
        // non-finite so that the step's non-finite check skips the update
        // (the rows not finished have no gradient).
        mbar_wait(mbar, phase ^ 1u, kWaitTries);
        if (t == 0) {
            atomicAdd(dW, __int_as_float(0x7fc00000));
            atomicAdd(&g_tc_timeouts, 1);
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tm, 256);
}

static gs_status check_common(const void *enc, int enc_dtype, const gs_mlp *w)
{
    GS_REQUIRE(w->w_bf16, "BF16 MLP: w_bf16 (the BF16 weight copy) is required");
    GS_REQUIRE(aligned(w->w_bf16, 16) && aligned(enc, 16), "BF16 MLP: misaligned enc or weights");
    GS_REQUIRE(enc_dtype == GS_F32 || enc_dtype == GS_BF16, "BF16 MLP: enc dtype");
    return GS_OK;
}

// Polls of an MMA-completion wait before a kernel gives up (set by
// gs_tc_set_wait_limit; read when a kernel is launched or captured).
static std::atomic<uint32_t> s_wait_tries{kWaitTries};

template <typename ET, bool FUSED>
static gs_status launch_fwd(TcParams p, cudaStream_t s)
{
    p.wait_tries = s_wait_tries.load();
    const size_t smem = sizeof(FwdSmem) + 1024;
    const int grid = (int)std::min<int64_t>(ceil_div(p.n, TM), num_sms() * 4);
    set_smem_limit((const void *)mlp_tc_fwd_kernel<ET, FUSED>, (int)smem, s);
    note_launch();
    mlp_tc_fwd_kernel<ET, FUSED><<<grid, TM, smem, s>>>(p);
    return launch_status(FUSED ? "ntc_fused_fwd" : "ntc_mlp_fwd (tcgen05)");
}

template <typename ET, bool FUSED>
static gs_status launch_bwd(TcParams p, cudaStream_t s)
{
    p.wait_tries = s_wait_tries.load();
    const size_t smem = sizeof(BwdSmem) + 1024;
    const int grid = (int)std::min<int64_t>(ceil_div(p.n, TM), num_sms() * 2);
    set_smem_limit((const void *)mlp_tc_bwd_kernel<ET, FUSED>, (int)smem, s);
    note_launch();
    mlp_tc_bwd_kernel<ET, FUSED><<<grid, TM, smem, s>>>(p);
    return launch_status(FUSED ? "ntc_fused_bwd" : "ntc_mlp_bwd (tcgen05)");
}

gs_status mlp_tc_fwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w, float *raw7,
                     cudaStream_t s)
{
    gs_status st = check_common(enc, enc_dtype, w);
    if (st != GS_OK) return st;
    GS_REQUIRE(w->w_f32, "BF16 MLP: w_f32 (the FP32 weights) is required for the output layer");
    TcParams p{};
    p.enc = enc;
    p.n = n;
    p.w = reinterpret_cast<const bf16 *>(w->w_bf16);
    p.w3f = w->w_f32 + 6144;
    p.raw7 = raw7;
    return enc_dtype == GS_BF16 ? launch_fwd<bf16, false>(p, s) : launch_fwd<float, false>(p, s);
}

gs_status mlp_tc_bwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w,
                     const float *d_raw7, const float *d_scale, float *dW, float *d_enc,
                     const uint32_t *rows, const int64_t *d_rows, cudaStream_t s)
{
    gs_status st = check_common(enc, enc_dtype, w);
    if (st != GS_OK) return st;
    GS_REQUIRE(d_enc == nullptr || aligned(d_enc, 16), "BF16 MLP: d_enc misaligned");
    TcParams p{};
    p.enc = enc;
    p.n = n;
    p.w = reinterpret_cast<const bf16 *>(w->w_bf16);
    p.d_raw7 = d_raw7;
    p.d_scale = d_scale;
    p.dW = dW;
    p.d_enc = d_enc;
    p.rows = rows;
    p.d_rows = d_rows;
    return enc_dtype == GS_BF16 ? launch_bwd<bf16, false>(p, s) : launch_bwd<float, false>(p, s);
}

}  // namespace gs3

using namespace gs3;

extern "C" gs_status ntc_fused_fwd(const float *mean, const float *quat, int64_t n,
                                   const gs_hashgrid *grid, const void *table_f16, const gs_mlp *w,
                                   int order, float *mean_out, float *quat_out, float *raw7,
                                   void *enc_save, gs_stream stream)
{
    GS_REQUIRE(grid && table_f16 && w && n >= 0, "ntc_fused_fwd: null grid, table or weights");
    GS_REQUIRE(n == 0 || (mean && quat && mean_out && quat_out && raw7 && enc_save),
               "ntc_fused_fwd: null argument");
    GS_REQUIRE(w->precision == GS_MLP_BF16 && w->w_bf16, "ntc_fused_fwd: needs BF16 MLP weights");
    GS_REQUIRE(order == 0 || order == 1, "ntc_fused_fwd: order must be 0 or 1");
    GS_REQUIRE(aligned(quat, 16) && aligned(quat_out, 16) && aligned(enc_save, 16) &&
                   aligned(w->w_bf16, 16) && aligned(table_f16, 4),
               "ntc_fused_fwd: misaligned argument");
    TcParams p{};
    int64_t total;
    GS_REQUIRE(grid_params(grid, p.grid, total), "ntc_fused_fwd: invalid hash grid");
    GS_REQUIRE(w->w_f32, "ntc_fused_fwd: w_f32 (the FP32 weights) is required");
    if (n == 0) return GS_OK;
    p.n = n;
    p.w = reinterpret_cast<const bf16 *>(w->w_bf16);
    p.w3f = w->w_f32 + 6144;
    p.raw7 = raw7;
    p.mean = mean;
    p.quat = quat;
    p.table = reinterpret_cast<const __half *>(table_f16);
    p.enc_save = reinterpret_cast<bf16 *>(enc_save);
    p.mean_out = mean_out;
    p.quat_out = quat_out;
    p.box = Box::from(grid->aabb);
    p.order = order;
    return launch_fwd<bf16, true>(p, as_stream(stream));
}

extern "C" gs_status ntc_fused_bwd(const float *mean, const float *quat, const float *raw7,
                                   const void *enc_save, int64_t n, const gs_hashgrid *grid,
                                   const gs_mlp *w, int order, const float *d_mean_out,
                                   const float *d_quat_out, const float *d_scale, float *dW,
                                   float *d_table, gs_stream stream)
{
    GS_REQUIRE(grid && w && dW && d_table && n >= 0, "ntc_fused_bwd: null grid, weights or gradients");
    GS_REQUIRE(n == 0 || (mean && quat && raw7 && enc_save && d_mean_out && d_quat_out),
               "ntc_fused_bwd: null argument");
    GS_REQUIRE(w->precision == GS_MLP_BF16 && w->w_bf16, "ntc_fused_bwd: needs BF16 MLP weights");
    GS_REQUIRE(order == 0 || order == 1, "ntc_fused_bwd: order must be 0 or 1");
    GS_REQUIRE(aligned(quat, 16) && aligned(d_quat_out, 16) && aligned(enc_save, 16) &&
                   aligned(w->w_bf16, 16) && aligned(d_table, 8),
               "ntc_fused_bwd: misaligned argument");
    TcParams p{};
    int64_t total;
    GS_REQUIRE(grid_params(grid, p.grid, total), "ntc_fused_bwd: invalid hash grid");
    if (n == 0) return GS_OK;
    p.enc = enc_save;
    p.n = n;
    p.w = reinterpret_cast<const bf16 *>(w->w_bf16);
    p.d_scale = d_scale;
    p.dW = dW;
    p.mean = mean;
    p.quat = quat;
    p.raw7_in = raw7;
    p.d_mean_out = d_mean_out;
    p.d_quat_out = d_quat_out;
    p.d_table = d_table;
    p.box = Box::from(grid->aabb);
    p.order = order;
    return launch_bwd<bf16, true>(p, as_stream(stream));
}

// Self-test of the bounded wait: one block initialises an mbarrier that
// nothing arrives on and waits for it with the MLP kernels' wait helper.
__global__ void tc_wait_selftest_kernel(uint32_t tries, int32_t *status)
{
    __shared__ __align__(8) unsigned long long mbar;
    const uint32_t m = gs3::tc::smem_u32(&mbar);
    if (threadIdx.x == 0) gs3::tc::mbar_init(m, 1);
    __syncthreads();
    const bool ok = __syncthreads_and(gs3::tc::mbar_wait(m, 0u, tries));
    if (threadIdx.x == 0) *status = ok ? GS_OK : GS_ERR_TIMEOUT;
}

extern "C" gs_status gs_tc_wait_selftest(uint32_t tries, int32_t *d_status, gs_stream stream)
{
    GS_REQUIRE(d_status && tries > 0 && tries <= (1u << 20), "gs_tc_wait_selftest: bad arguments");
    note_launch();
    tc_wait_selftest_kernel<<<1, 128, 0, as_stream(stream)>>>(tries, d_status);
    return launch_status("gs_tc_wait_selftest");
}

extern "C" gs_status gs_tc_set_wait_limit(uint32_t tries)
{
    gs3::s_wait_tries.store(tries);
    return GS_OK;
}

extern "C" int gs_tc_timeouts(void)
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, gs3::g_tc_timeouts, sizeof(int)) != cudaSuccess) return -1;
    return v;
}

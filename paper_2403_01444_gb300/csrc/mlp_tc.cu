// BF16 tensor-core MLP of the transformation cache (Section 4.1, Eq. 5):
// 32 -> 64 -> 64 -> 7 with ReLU, no biases, BF16 x BF16 -> FP32 on tcgen05.
//
// One CTA of 128 threads owns a tile of 128 Gaussians (the M = 128 rows of
// every MMA); thread t holds row t, which is TMEM lane t.  Operands are staged
// in shared memory in the K-major no-swizzle layout, the accumulator lives in
// TMEM, thread 0 issues the MMAs and an mbarrier tracks their completion
// (bounded waits).  Forward: three chained MMAs with ReLU epilogues.
// Backward (recomputing the forward from the encoding):
//   dH2 = (G W3) . relu'(H2),  dH1 = (dH2 W2) . relu'(H1),  d_enc = dH1 W1
//   dW2 = dH2^T H1, dW1 = dH1^T enc, dW3 = G^T H2
// The three weight gradients are contractions over the Gaussians; they are
// stacked into two M = 128 MMAs over K = 128 rows of the tile and accumulate
// in TMEM across all tiles a CTA owns, then one FP32 atomic per weight per CTA.
#include "ntc.cuh"
#include "tc.cuh"

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
    bf16 w3[16 * 64];   // rows 7..15 zero (N padded to 16)
    unsigned long long mbar;
    uint32_t tmem;
};

struct BwdSmem {
    bf16 AT[192 * TM];  // rows: H2^T (0..63), dH2^T (64..127), dH1^T (128..191); K = tile rows
    bf16 BT[112 * TM];  // rows: H1^T (0..63), enc^T (64..95), G^T (96..111)
    bf16 a1[TM * 32];
    bf16 h1a[TM * 64];
    bf16 g2a[TM * 64];
    bf16 g1a[TM * 64];
    bf16 ga[TM * 16];
    bf16 w1[64 * 32];   // [out][in]
    bf16 w2[64 * 64];
    bf16 w3t[64 * 16];  // [hidden][out], out padded to 16
    bf16 w2t[64 * 64];  // [in][out]
    bf16 w1t[32 * 64];  // [in][hidden]
    unsigned long long mbar;
    uint32_t tmem;
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

// W1 | W2 | W3 (bf16, [out][in] row-major) into K-major B operands.
__device__ __forceinline__ void load_weights_fwd(const bf16 *w, bf16 *w1, bf16 *w2, bf16 *w3)
{
    for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) w1[kmajor_off(e >> 5, e & 31, 32)] = w[e];
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x)
        w2[kmajor_off(e >> 6, e & 63, 64)] = w[2048 + e];
    for (int e = threadIdx.x; e < 16 * 64; e += blockDim.x) {
        int o = e >> 6, j = e & 63;
        w3[kmajor_off(o, j, 64)] = o < 7 ? w[6144 + o * 64 + j] : __float2bfloat16(0.f);
    }
}

// All threads wait for the MMA batch; returns false (block-uniformly) on timeout.
__device__ __forceinline__ bool wait_mma(uint32_t mbar, uint32_t &phase)
{
    bool ok = mbar_wait(mbar, phase, kWaitTries);
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

template <typename ET>
__global__ void __launch_bounds__(TM) mlp_tc_fwd_kernel(const ET *enc, int64_t n, const bf16 *w,
                                                        float *raw7)
{
    extern __shared__ unsigned char smem_raw[];
    FwdSmem &S = *aligned_smem<FwdSmem>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5;
    load_weights_fwd(w, S.w1, S.w2, S.w3);
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
    const uint32_t id64 = idesc_bf16_f32(128, 64), id16 = idesc_bf16_f32(128, 16);
    const uint32_t a1 = smem_u32(S.a1), a2 = smem_u32(S.a2);
    const uint32_t w1 = smem_u32(S.w1), w2 = smem_u32(S.w2), w3 = smem_u32(S.w3);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (n + TM - 1) / TM;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t row = tile * TM + t;
        float v[64];
        load_row32(enc, row, n, v);
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
        if (!(ok = wait_mma(mbar, phase))) break;
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
        if (!(ok = wait_mma(mbar, phase))) break;
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
                mma_bf16(tm, desc_kmajor(a2 + 256 * ks, 128, 1024), desc_kmajor(w3 + 256 * ks, 128, 1024),
                         id16, ks > 0);
            mma_commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase))) break;
        tmem_ld16(tm + lane, v);
        if (row < n) {
#pragma unroll
            for (int q = 0; q < 7; ++q) raw7[row * 7 + q] = v[q];
        }
        fence_before_sync();
        __syncthreads();
    }
    if (!ok && t == 0) atomicAdd(&g_tc_timeouts, 1);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tm, 64);
}

template <typename ET>
__global__ void __launch_bounds__(TM) mlp_tc_bwd_kernel(const ET *enc, int64_t n, const bf16 *w,
                                                        const float *d_raw7, const float *d_scale,
                                                        float *dW, float *d_enc)
{
    extern __shared__ unsigned char smem_raw[];
    BwdSmem &S = *aligned_smem<BwdSmem>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5;
    load_weights_fwd(w, S.w1, S.w2, S.w3t);  // w3t slot reused below; rewritten transposed
    __syncthreads();
    for (int e = t; e < 64 * 16; e += TM) {
        int j = e >> 4, o = e & 15;
        S.w3t[kmajor_off(j, o, 16)] = o < 7 ? w[6144 + o * 64 + j] : __float2bfloat16(0.f);
    }
    for (int e = t; e < 64 * 64; e += TM) {
        int j = e >> 6, k = e & 63;  // W2[j][k] -> w2t[k][j]
        S.w2t[kmajor_off(k, j, 64)] = w[2048 + e];
    }
    for (int e = t; e < 64 * 32; e += TM) {
        int j = e >> 5, i = e & 31;  // W1[j][i] -> w1t[i][j]
        S.w1t[kmajor_off(i, j, 64)] = w[e];
    }
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
    const uint32_t sa1 = smem_u32(S.a1), sh1 = smem_u32(S.h1a), sg2 = smem_u32(S.g2a);
    const uint32_t sg1 = smem_u32(S.g1a), sga = smem_u32(S.ga);
    const uint32_t sw1 = smem_u32(S.w1), sw2 = smem_u32(S.w2), sw3t = smem_u32(S.w3t);
    const uint32_t sw2t = smem_u32(S.w2t), sw1t = smem_u32(S.w1t);
    const float scale = d_scale ? *d_scale : 1.f;
    uint32_t phase = 0;
    bool ok = true;
    int done_tiles = 0;
    const int64_t ntiles = (n + TM - 1) / TM;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t row = tile * TM + t;
        float v[64];
        // ---- stage the encoding and the scaled output gradient
        load_row32(enc, row, n, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) st_chunk8(S.a1, t, 8 * c, 32, v + 8 * c);
#pragma unroll
        for (int i = 0; i < 32; ++i) S.BT[kmajor_off(64 + i, t, TM)] = __float2bfloat16_rn(v[i]);
        float g[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) g[q] = (q < 7 && row < n) ? d_raw7[row * 7 + q] * scale : 0.f;
        st_chunk8(S.ga, t, 0, 16, g);
        st_chunk8(S.ga, t, 8, 16, g + 8);
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
        if (!(ok = wait_mma(mbar, phase))) break;
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
        for (int c = 0; c < 8; ++c) st_chunk8(S.h1a, t, 8 * c, 64, v + 8 * c);
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
        if (!(ok = wait_mma(mbar, phase))) break;
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
        for (int c = 0; c < 8; ++c) st_chunk8(S.g2a, t, 8 * c, 64, v + 8 * c);
#pragma unroll
        for (int j = 0; j < 64; ++j) S.AT[kmajor_off(64 + j, t, TM)] = __float2bfloat16_rn(v[j]);
        publish_smem();
        if (t == 0) {
            fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(D0, desc_kmajor(sg2 + 256 * ks, 128, 1024), desc_kmajor(sw2t + 256 * ks, 128, 1024),
                         id64, ks > 0);
            mma_commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase))) break;
        // ---- dH1 = (dH2 W2) . relu'(H1)
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld16(D0 + lane + 16 * c, v + 16 * c);
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            bool pos = k < 32 ? ((m1lo >> k) & 1u) : ((m1hi >> (k - 32)) & 1u);
            v[k] = pos ? v[k] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) st_chunk8(S.g1a, t, 8 * c, 64, v + 8 * c);
#pragma unroll
        for (int j = 0; j < 64; ++j) S.AT[kmajor_off(128 + j, t, TM)] = __float2bfloat16_rn(v[j]);
        publish_smem();
        if (t == 0) {
            fence_after_sync();
            // d_enc = dH1 W1
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                mma_bf16(D0, desc_kmajor(sg1 + 256 * ks, 128, 1024), desc_kmajor(sw1t + 256 * ks, 128, 1024),
                         id32, ks > 0);
            // [dW2 | . ; . | dW1] += [dH2^T ; dH1^T] [H1 | enc], K = the tile's rows
            const uint32_t acc0 = done_tiles > 0 ? 1u : 0u;
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
                mma_bf16(DW, desc_kmajor(sAT + 8 * 2048 + 256 * ks, 128, 2048),
                         desc_kmajor(sBT + 256 * ks, 128, 2048), id96, ks > 0 ? 1u : acc0);
            // dW3^T += H2^T G (rows 64..127 of this product are unused)
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
                mma_bf16(DW3, desc_kmajor(sAT + 256 * ks, 128, 2048),
                         desc_kmajor(sBT + 12 * 2048 + 256 * ks, 128, 2048), id16, ks > 0 ? 1u : acc0);
            mma_commit(mbar);
        }
        if (!(ok = wait_mma(mbar, phase))) break;
        if (d_enc) {
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
        float v[16];
        if (warp < 2) {
            const int j = t;  // dW2 row (output unit) j, dW3 column j
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                tmem_ld16(DW + lane + 16 * c, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(dW + 2048 + j * 64 + 16 * c + i, v[i]);
            }
            tmem_ld16(DW3 + lane, v);
#pragma unroll
            for (int o = 0; o < 7; ++o) atomicAdd(dW + 6144 + o * 64 + j, v[o]);
        } else {
            const int j = t - 64;  // dW1 row j
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                tmem_ld16(DW + lane + 64 + 16 * c, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(dW + j * 32 + 16 * c + i, v[i]);
            }
        }
    }
    if (!ok && t == 0) atomicAdd(&g_tc_timeouts, 1);
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

gs_status mlp_tc_fwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w, float *raw7,
                     cudaStream_t s)
{
    gs_status st = check_common(enc, enc_dtype, w);
    if (st != GS_OK) return st;
    const size_t smem = sizeof(FwdSmem) + 1024;
    const int64_t ntiles = ceil_div(n, TM);
    const int grid = (int)std::min<int64_t>(ntiles, kNumSMs * 4);
    const bf16 *wb = reinterpret_cast<const bf16 *>(w->w_bf16);
    note_launch();
    if (enc_dtype == GS_BF16) {
        set_smem_limit((const void *)mlp_tc_fwd_kernel<bf16>, (int)smem, s);
        mlp_tc_fwd_kernel<bf16><<<grid, TM, smem, s>>>((const bf16 *)enc, n, wb, raw7);
    } else {
        set_smem_limit((const void *)mlp_tc_fwd_kernel<float>, (int)smem, s);
        mlp_tc_fwd_kernel<float><<<grid, TM, smem, s>>>((const float *)enc, n, wb, raw7);
    }
    return launch_status("ntc_mlp_fwd (tcgen05)");
}

gs_status mlp_tc_bwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w,
                     const float *d_raw7, const float *d_scale, float *dW, float *d_enc,
                     cudaStream_t s)
{
    gs_status st = check_common(enc, enc_dtype, w);
    if (st != GS_OK) return st;
    GS_REQUIRE(d_enc == nullptr || aligned(d_enc, 16), "BF16 MLP: d_enc misaligned");
    const size_t smem = sizeof(BwdSmem) + 1024;
    const int64_t ntiles = ceil_div(n, TM);
    const int grid = (int)std::min<int64_t>(ntiles, kNumSMs);
    const bf16 *wb = reinterpret_cast<const bf16 *>(w->w_bf16);
    note_launch();
    if (enc_dtype == GS_BF16) {
        set_smem_limit((const void *)mlp_tc_bwd_kernel<bf16>, (int)smem, s);
        mlp_tc_bwd_kernel<bf16><<<grid, TM, smem, s>>>((const bf16 *)enc, n, wb, d_raw7, d_scale, dW, d_enc);
    } else {
        set_smem_limit((const void *)mlp_tc_bwd_kernel<float>, (int)smem, s);
        mlp_tc_bwd_kernel<float><<<grid, TM, smem, s>>>((const float *)enc, n, wb, d_raw7, d_scale, dW, d_enc);
    }
    return launch_status("ntc_mlp_bwd (tcgen05)");
}

}  // namespace gs3

extern "C" int gs_tc_timeouts(void)
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, gs3::g_tc_timeouts, sizeof(int)) != cudaSuccess) return -1;
    return v;
}

// Device helpers of the Neural Transformation Cache kernels (Section 4.1).
#pragma once

#include "common.cuh"

namespace gs3 {

constexpr int kMaxLevels = 16;

struct GridParams {
    int L;
    uint32_t mask;
    float amin[3], ext[3];
    int res[kMaxLevels];
    int dense[kMaxLevels];
    uint32_t offset[kMaxLevels];
};

bool grid_params(const gs_hashgrid *g, GridParams &P, int64_t &total);

// The 8 corners of the cell holding m at level l and their trilinear weights.
// Dense levels index x + y s + z s^2 (s = N + 1); hashed levels use the
// I-NGP spatial hash (x * 1 ^ y * 2654435761 ^ z * 805459861) mod T.
__device__ __forceinline__ void level_corners(const GridParams &g, int l, float3 m, uint32_t *idx,
                                              float *w)
{
    const int N = g.res[l];
    float pos[3] = {m.x, m.y, m.z};
    uint32_t c[3];
    float f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float x = (pos[k] - g.amin[k]) / g.ext[k];
        x = fminf(fmaxf(x, 0.f), 1.f);
        float p = x * (float)N;
        float fl = fminf(floorf(p), (float)(N - 1));
        c[k] = (uint32_t)fl;
        f[k] = p - fl;
    }
    const uint32_t s = (uint32_t)N + 1u;
    const bool dense = g.dense[l] != 0;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        uint32_t bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
        uint32_t x = c[0] + bx, y = c[1] + by, z = c[2] + bz;
        uint32_t h = dense ? (x + y * s + z * s * s)
                           : ((x * 1u) ^ (y * 2654435761u) ^ (z * 805459861u)) & g.mask;
        idx[corner] = g.offset[l] + h;
        w[corner] = (bx ? f[0] : 1.f - f[0]) * (by ? f[1] : 1.f - f[1]) * (bz ? f[2] : 1.f - f[2]);
    }
}

__device__ __forceinline__ void store2(float *p, float a, float b)
{
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}
__device__ __forceinline__ void store2(__nv_bfloat16 *p, float a, float b)
{
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }

// ------------------------------------------------------------ quaternions
// Hamilton product, (w, x, y, z) stored in (x, y, z, w) of a float4.
__device__ __forceinline__ float4 qmul(float4 a, float4 b)
{
    return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w,
                       a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                       a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y,
                       a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}
__device__ __forceinline__ float4 qconj(float4 a) { return make_float4(a.x, -a.y, -a.z, -a.w); }
// Transposes of d -> a (x) d and d -> d (x) a applied to g.
__device__ __forceinline__ float4 qmul_left_T(float4 a, float4 g) { return qmul(qconj(a), g); }
__device__ __forceinline__ float4 qmul_right_T(float4 a, float4 g) { return qmul(g, qconj(a)); }

__device__ __forceinline__ float4 qnormalize(float4 q)
{
    float len = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float d = 1.f / fmaxf(len, 1e-12f);
    return make_float4(q.x * d, q.y * d, q.z * d, q.w * d);
}
// d/dq of q / max(|q|, 1e-12) applied to g.
__device__ __forceinline__ float4 qnormalize_bwd(float4 q, float4 g)
{
    float len = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    if (!(len > 1e-12f)) return make_float4(g.x * 1e12f, g.y * 1e12f, g.z * 1e12f, g.w * 1e12f);
    float il = 1.f / len;
    float4 n = make_float4(q.x * il, q.y * il, q.z * il, q.w * il);
    float dot = n.x * g.x + n.y * g.y + n.z * g.z + n.w * g.w;
    return make_float4((g.x - n.x * dot) * il, (g.y - n.y * dot) * il, (g.z - n.z * dot) * il,
                       (g.w - n.w * dot) * il);
}

struct Box {
    float lo[3], hi[3];
    static Box from(const float *a)
    {
        Box b;
        for (int k = 0; k < 3; ++k) {
            b.lo[k] = a[k];
            b.hi[k] = a[3 + k];
        }
        return b;
    }
    __device__ __forceinline__ bool inside(float3 m) const
    {
        return m.x >= lo[0] && m.x <= hi[0] && m.y >= lo[1] && m.y <= hi[1] && m.z >= lo[2] &&
               m.z <= hi[2];
    }
};

// BF16 tensor-core MLP (mlp_tc.cu)
gs_status mlp_tc_fwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w, float *raw7,
                     cudaStream_t s);
gs_status mlp_tc_bwd(const void *enc, int enc_dtype, int64_t n, const gs_mlp *w,
                     const float *d_raw7, const float *d_scale, float *dW, float *d_enc,
                     const uint32_t *rows, const int64_t *d_rows, cudaStream_t s);

}  // namespace gs3

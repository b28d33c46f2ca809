// EWA projection + SH colour (Section 3.2, Eq. 2-3) and its reverse.
// One thread per Gaussian handles all V views of a launch, so each Gaussian's
// parameters (up to 236 bytes with SH degree 3) are read from HBM once.
#include <type_traits>

#include "common.cuh"
#include "sh.cuh"

namespace gs3 {

struct ProjectParams {
    const float *mean, *quat, *scale, *opl, *sh;
    bool sh_vec4;  // sh is 16-byte aligned
    int64_t n;
    int deg, K;
    const gs_camera *cams;
    int V, W, H, tx, ty;
    // forward outputs
    float2 *mean2d;
    float4 *conic_op;
    float *rgb;
    float *depth;
    int32_t *radius;
    int32_t *tiles;
    int32_t *d_err;  // GS_ERR_NONFINITE on a non-finite Gaussian (nullable)
    // backward
    const float *grads;
    float *d_mean, *d_quat;
    // full backward (every parameter of Gaussians [first, first + count))
    const float *d_opacity;
    int64_t first, count;
    float *d_scale, *d_ologit, *d_sh;
};

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float *Y)
{
    sh_basis_t<float>(deg, x, y, z, Y);
}

// sum_k w[k] * grad Y_k(x, y, z)
__device__ __forceinline__ float3 sh_basis_grad_dot(int deg, float x, float y, float z,
                                                    const float *w)
{
    float3 g = make_float3(0.f, 0.f, 0.f);
    if (deg < 1) return g;
    g.y += -float(SH_C1) * w[1];
    g.z += float(SH_C1) * w[2];
    g.x += -float(SH_C1) * w[3];
    if (deg < 2) return g;
    float xx = x * x, yy = y * y, zz = z * z;
    g.x += float(SH_C2A) * y * w[4];
    g.y += float(SH_C2A) * x * w[4];
    g.y += -float(SH_C2A) * z * w[5];
    g.z += -float(SH_C2A) * y * w[5];
    g.x += -2.f * float(SH_C2B) * x * w[6];
    g.y += -2.f * float(SH_C2B) * y * w[6];
    g.z += 4.f * float(SH_C2B) * z * w[6];
    g.x += -float(SH_C2A) * z * w[7];
    g.z += -float(SH_C2A) * x * w[7];
    g.x += 2.f * float(SH_C2C) * x * w[8];
    g.y += -2.f * float(SH_C2C) * y * w[8];
    if (deg < 3) return g;
    g.x += -6.f * float(SH_C3A) * x * y * w[9];
    g.y += -float(SH_C3A) * (3.f * xx - 3.f * yy) * w[9];
    g.x += float(SH_C3B) * y * z * w[10];
    g.y += float(SH_C3B) * x * z * w[10];
    g.z += float(SH_C3B) * x * y * w[10];
    g.x += 2.f * float(SH_C3C) * x * y * w[11];
    g.y += -float(SH_C3C) * (4.f * zz - xx - 3.f * yy) * w[11];
    g.z += -8.f * float(SH_C3C) * y * z * w[11];
    g.x += -6.f * float(SH_C3D) * x * z * w[12];
    g.y += -6.f * float(SH_C3D) * y * z * w[12];
    g.z += float(SH_C3D) * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
    g.x += -float(SH_C3C) * (4.f * zz - 3.f * xx - yy) * w[13];
    g.y += 2.f * float(SH_C3C) * x * y * w[13];
    g.z += -8.f * float(SH_C3C) * x * z * w[13];
    g.x += 2.f * float(SH_C3E) * x * z * w[14];
    g.y += -2.f * float(SH_C3E) * y * z * w[14];
    g.z += float(SH_C3E) * (xx - yy) * w[14];
    g.x += -float(SH_C3A) * (3.f * xx - 3.f * yy) * w[15];
    g.y += 6.f * float(SH_C3A) * x * y * w[15];
    return g;
}

// Per-Gaussian, view-independent quantities.
struct GaussLocal {
    float3 mu;
    float qn[4];
    float qlen;
    float R[9];
    float s[3];
    float Sig[6];  // s00 s01 s02 s11 s12 s22
    float op;
};

__device__ __forceinline__ void load_gauss(const ProjectParams &p, int64_t i, GaussLocal &G)
{
    G.mu = make_float3(p.mean[3 * i], p.mean[3 * i + 1], p.mean[3 * i + 2]);
    float4 q = reinterpret_cast<const float4 *>(p.quat)[i];
    float ql = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    G.qlen = ql;
    float inv = 1.f / ql;
    float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    G.qn[0] = w; G.qn[1] = x; G.qn[2] = y; G.qn[3] = z;
    G.R[0] = 1.f - 2.f * (y * y + z * z); G.R[1] = 2.f * (x * y - w * z); G.R[2] = 2.f * (x * z + w * y);
    G.R[3] = 2.f * (x * y + w * z); G.R[4] = 1.f - 2.f * (x * x + z * z); G.R[5] = 2.f * (y * z - w * x);
    G.R[6] = 2.f * (x * z - w * y); G.R[7] = 2.f * (y * z + w * x); G.R[8] = 1.f - 2.f * (x * x + y * y);
    G.s[0] = p.scale[3 * i]; G.s[1] = p.scale[3 * i + 1]; G.s[2] = p.scale[3 * i + 2];
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[3 * r + c] = G.R[3 * r + c] * G.s[c];
    G.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    G.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    G.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    G.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    G.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    G.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    G.op = 1.f / (1.f + expf(-p.opl[i]));
}

// Per-(Gaussian, view) forward state reused by the reverse pass.
struct ViewLocal {
    bool valid;
    float t[3];
    float txz, tyz, limx, limy;
    bool clx, cly;
    float T[6];  // J W (2x3)
    float a, b, c;
    float det;
    float conic[3];
    int radius;
    float u, v;
    int tiles;
    float3 dir;
    float dlen;
    float rgb_raw[3];
};

template <int DEG>
__device__ __forceinline__ void project_view(const ProjectParams &p, const GaussLocal &G,
                                             const float *sh, const gs_camera &c, ViewLocal &L)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    L.valid = false;
    L.radius = 0;
    L.tiles = 0;
    const float *Wm = c.viewmat;
    L.t[0] = fmaf(Wm[0], G.mu.x, fmaf(Wm[1], G.mu.y, fmaf(Wm[2], G.mu.z, Wm[3])));
    L.t[1] = fmaf(Wm[4], G.mu.x, fmaf(Wm[5], G.mu.y, fmaf(Wm[6], G.mu.z, Wm[7])));
    L.t[2] = fmaf(Wm[8], G.mu.x, fmaf(Wm[9], G.mu.y, fmaf(Wm[10], G.mu.z, Wm[11])));
    float tz = L.t[2];
    if (!(tz > 0.2f)) return;
    float itz = 1.f / tz;
    L.limx = 1.3f * (0.5f * (float)c.width / c.fx);
    L.limy = 1.3f * (0.5f * (float)c.height / c.fy);
    L.txz = L.t[0] * itz;
    L.tyz = L.t[1] * itz;
    float txc = fminf(L.limx, fmaxf(-L.limx, L.txz));
    float tyc = fminf(L.limy, fmaxf(-L.limy, L.tyz));
    L.clx = (L.txz < -L.limx) || (L.txz > L.limx);
    L.cly = (L.tyz < -L.limy) || (L.tyz > L.limy);
    float j00 = c.fx * itz, j02 = -c.fx * txc * itz;
    float j11 = c.fy * itz, j12 = -c.fy * tyc * itz;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        L.T[j] = j00 * Wm[j] + j02 * Wm[8 + j];
        L.T[3 + j] = j11 * Wm[4 + j] + j12 * Wm[8 + j];
    }
    // 2D covariance T Sigma T^T + 0.3 I through P = T R diag(s) (2x3), so
    // that T Sigma T^T = P P^T.  Its determinant by the Cauchy-Binet formula,
    //   det(P P^T + 0.3 I) = sum of the squared 2x2 minors of P
    //                        + 0.3 (|P_0|^2 + |P_1|^2) + 0.09,
    // is a sum of non-negative terms: no cancellation, even for a needle
    // whose a c - b^2 would cancel to nothing in FP32.
    float P[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float m0 = G.R[k] * G.s[k], m1 = G.R[3 + k] * G.s[k], m2 = G.R[6 + k] * G.s[k];
        P[k] = L.T[0] * m0 + L.T[1] * m1 + L.T[2] * m2;
        P[3 + k] = L.T[3] * m0 + L.T[4] * m1 + L.T[5] * m2;
    }
    const float pa = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    const float pc = P[3] * P[3] + P[4] * P[4] + P[5] * P[5];
    L.a = pa + 0.3f;
    L.b = P[0] * P[3] + P[1] * P[4] + P[2] * P[5];
    L.c = pc + 0.3f;
    const float m01 = P[0] * P[4] - P[1] * P[3];
    const float m02 = P[0] * P[5] - P[2] * P[3];
    const float m12 = P[1] * P[5] - P[2] * P[4];
    const float det = m01 * m01 + m02 * m02 + m12 * m12 + 0.3f * (pa + pc) + 0.09f;
    const float tr = L.a + L.c;
    if (!(det > 0.f)) return;   // only for non-finite inputs
    L.det = det;
    const float id = 1.f / det;
    L.conic[0] = L.c * id;
    L.conic[1] = -L.b * id;
    L.conic[2] = L.a * id;
    float mid = 0.5f * tr;
    float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - L.det));
    L.radius = (int)ceilf(3.f * sqrtf(lam));
    L.u = c.fx * L.t[0] * itz + c.cx;
    L.v = c.fy * L.t[1] * itz + c.cy;
    int x0, y0, x1, y1;
    tile_rect(L.u, L.v, L.radius, p.tx, p.ty, x0, y0, x1, y1);
    L.tiles = (x1 - x0) * (y1 - y0);
    if (L.tiles == 0) {
        L.radius = 0;
        return;
    }
    float3 d = make_float3(G.mu.x - c.campos[0], G.mu.y - c.campos[1], G.mu.z - c.campos[2]);
    L.dlen = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
    float il = 1.f / L.dlen;
    L.dir = make_float3(d.x * il, d.y * il, d.z * il);
    float Y[16];
    sh_basis(DEG, L.dir.x, L.dir.y, L.dir.z, Y);
    float r0 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        r0 = fmaf(Y[k], sh[3 * k], r0);
        r1 = fmaf(Y[k], sh[3 * k + 1], r1);
        r2 = fmaf(Y[k], sh[3 * k + 2], r2);
    }
    L.rgb_raw[0] = r0 + 0.5f;
    L.rgb_raw[1] = r1 + 0.5f;
    L.rgb_raw[2] = r2 + 0.5f;
    L.valid = true;
}

// Gaussian i's SH coefficients into registers (float4 loads when each
// Gaussian's 3K floats keep 16-byte alignment).
template <int DEG>
__device__ __forceinline__ void load_sh(const ProjectParams &p, int64_t i, float (&sh)[3 * (DEG + 1) * (DEG + 1)])
{
    constexpr int N = 3 * (DEG + 1) * (DEG + 1);
    const float *shg = p.sh + (int64_t)N * i;
    if (N % 4 == 0 && p.sh_vec4) {
        const float4 *s4 = reinterpret_cast<const float4 *>(shg);
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 t = __ldg(s4 + q);
            sh[4 * q] = t.x;
            sh[4 * q + 1] = t.y;
            sh[4 * q + 2] = t.z;
            sh[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) sh[q] = __ldg(shg + q);
    }
}

#ifndef PROJ_FWD_MIN_BLOCKS
#define PROJ_FWD_MIN_BLOCKS 1
#endif
template <int DEG>
__global__ void __launch_bounds__(256, PROJ_FWD_MIN_BLOCKS) project_fwd_kernel(ProjectParams p)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    extern __shared__ gs_camera s_cams[];
    for (int k = threadIdx.x; k < p.V; k += blockDim.x) s_cams[k] = p.cams[k];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    GaussLocal G;
    load_gauss(p, i, G);
    // the Gaussian's SH coefficients once, for every view
    float sh[3 * K];
    load_sh<DEG>(p, i, sh);
    // a Gaussian with a non-finite mean, rotation, scale or opacity, or whose
    // projected record comes out non-finite, is culled in every view and
    // reported in the error word
    bool bad = !isfinite(G.mu.x + G.mu.y + G.mu.z + G.qlen + G.s[0] + G.s[1] + G.s[2] + G.op);
    for (int v = 0; v < p.V; ++v) {
        ViewLocal L;
        L.valid = false;
        if (!bad) project_view<DEG>(p, G, sh, s_cams[v], L);
        if (L.valid && !isfinite(L.u + L.v + L.conic[0] + L.conic[1] + L.conic[2] + L.rgb_raw[0] +
                                 L.rgb_raw[1] + L.rgb_raw[2])) {
            L.valid = false;
            bad = true;
        }
        int64_t o = (int64_t)v * p.n + i;
        if (L.valid) {
            p.mean2d[o] = make_float2(L.u, L.v);
            p.conic_op[o] = make_float4(L.conic[0], L.conic[1], L.conic[2], G.op);
            p.rgb[3 * o] = fmaxf(L.rgb_raw[0], 0.f);
            p.rgb[3 * o + 1] = fmaxf(L.rgb_raw[1], 0.f);
            p.rgb[3 * o + 2] = fmaxf(L.rgb_raw[2], 0.f);
            p.depth[o] = L.t[2];
            p.radius[o] = L.radius;
            p.tiles[o] = L.tiles;
        } else {
            p.mean2d[o] = make_float2(0.f, 0.f);
            p.conic_op[o] = make_float4(0.f, 0.f, 0.f, 0.f);
            p.rgb[3 * o] = 0.f;
            p.rgb[3 * o + 1] = 0.f;
            p.rgb[3 * o + 2] = 0.f;
            p.depth[o] = 0.f;
            p.radius[o] = 0;
            p.tiles[o] = 0;
        }
    }
    if (bad && p.d_err) atomicCAS(p.d_err, 0, (int32_t)GS_ERR_NONFINITE);
}

// One view's contribution to dL/dmu and dL/dSigma (everything but the
// SH-coefficient and opacity terms) from that view's record gradient.
template <int DEG>
__device__ __forceinline__ void bwd_view(const GaussLocal &G, const float *sh, const gs_camera &c,
                                         const ViewLocal &L, float4 g0, float4 g1, float *dmu,
                                         float *dS)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    float du = g0.x, dv = g0.y, dA = g0.z, dB = g0.w, dC = g1.x;
    float drgb[3] = {g1.y, g1.z, g1.w};
    // colour -> direction -> mean
    float wk[16];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
            if (L.rgb_raw[ch] > 0.f) acc = fmaf(drgb[ch], sh[3 * k + ch], acc);
        wk[k] = acc;
    }
    float3 gd = sh_basis_grad_dot(DEG, L.dir.x, L.dir.y, L.dir.z, wk);
    float dd = L.dir.x * gd.x + L.dir.y * gd.y + L.dir.z * gd.z;
    float il = 1.f / L.dlen;
    dmu[0] += (gd.x - L.dir.x * dd) * il;
    dmu[1] += (gd.y - L.dir.y * dd) * il;
    dmu[2] += (gd.z - L.dir.z * dd) * il;
    // 2D mean
    float tz = L.t[2], itz = 1.f / tz, itz2 = itz * itz;
    float dt0 = du * c.fx * itz;
    float dt1 = dv * c.fy * itz;
    float dt2 = -(du * c.fx * L.t[0] + dv * c.fy * L.t[1]) * itz2;
    // conic -> 2D covariance
    float a = L.a, b = L.b, cc = L.c;
    float id2 = 1.f / (L.det * L.det);
    float ga = (-cc * cc * dA + b * cc * dB - b * b * dC) * id2;
    float gb = (2.f * b * cc * dA - (a * cc + b * b) * dB + 2.f * a * b * dC) * id2;
    float gc = (-b * b * dA + a * b * dB - a * a * dC) * id2;
    float G00 = ga, G01 = 0.5f * gb, G11 = gc;
    // GT = G * T (2x3)
    float GT[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        GT[j] = G00 * L.T[j] + G01 * L.T[3 + j];
        GT[3 + j] = G01 * L.T[j] + G11 * L.T[3 + j];
    }
    // dSigma += T^T GT
    dS[0] += L.T[0] * GT[0] + L.T[3] * GT[3];
    dS[1] += L.T[0] * GT[1] + L.T[3] * GT[4];
    dS[2] += L.T[0] * GT[2] + L.T[3] * GT[5];
    dS[3] += L.T[1] * GT[1] + L.T[4] * GT[4];
    dS[4] += L.T[1] * GT[2] + L.T[4] * GT[5];
    dS[5] += L.T[2] * GT[2] + L.T[5] * GT[5];
    // dT = 2 GT Sigma (2x3)
    const float *S = G.Sig;
    float dT[6];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float *q = GT + 3 * r;
        dT[3 * r + 0] = 2.f * (q[0] * S[0] + q[1] * S[1] + q[2] * S[2]);
        dT[3 * r + 1] = 2.f * (q[0] * S[1] + q[1] * S[3] + q[2] * S[4]);
        dT[3 * r + 2] = 2.f * (q[0] * S[2] + q[1] * S[4] + q[2] * S[5]);
    }
    // T = J W  ->  dJ = dT W^T (only the four non-zero entries of J)
    const float *Wm = c.viewmat;
    float dJ00 = dT[0] * Wm[0] + dT[1] * Wm[1] + dT[2] * Wm[2];
    float dJ02 = dT[0] * Wm[8] + dT[1] * Wm[9] + dT[2] * Wm[10];
    float dJ11 = dT[3] * Wm[4] + dT[4] * Wm[5] + dT[5] * Wm[6];
    float dJ12 = dT[3] * Wm[8] + dT[4] * Wm[9] + dT[5] * Wm[10];
    dt2 += -c.fx * itz2 * dJ00 - c.fy * itz2 * dJ11;
    if (L.clx) {
        float ls = L.txz < 0.f ? -L.limx : L.limx;  // J02 = -fx ls / tz
        dt2 += c.fx * ls * itz2 * dJ02;
    } else {  // J02 = -fx tx / tz^2
        dt0 += -c.fx * itz2 * dJ02;
        dt2 += 2.f * c.fx * L.t[0] * itz2 * itz * dJ02;
    }
    if (L.cly) {
        float ls = L.tyz < 0.f ? -L.limy : L.limy;
        dt2 += c.fy * ls * itz2 * dJ12;
    } else {
        dt1 += -c.fy * itz2 * dJ12;
        dt2 += 2.f * c.fy * L.t[1] * itz2 * itz * dJ12;
    }
    // t = W mu + t_w
    dmu[0] += Wm[0] * dt0 + Wm[4] * dt1 + Wm[8] * dt2;
    dmu[1] += Wm[1] * dt0 + Wm[5] * dt1 + Wm[9] * dt2;
    dmu[2] += Wm[2] * dt0 + Wm[6] * dt1 + Wm[10] * dt2;
}

// dL/dSigma -> dL/d(un-normalised quaternion) and dL/ds; writes d_mean and
// d_quat of row j.
__device__ __forceinline__ void bwd_finish(const ProjectParams &p, const GaussLocal &G, int64_t j,
                                           const float *dmu, const float *dS, float *ds)
{
    // Sigma = M M^T, M = R diag(s): dR = 2 dSigma M diag(s)
    float dSf[9] = {dS[0], dS[1], dS[2], dS[1], dS[3], dS[4], dS[2], dS[4], dS[5]};
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[3 * r + c] = G.R[3 * r + c] * G.s[c];
    float dR[9];
    ds[0] = ds[1] = ds[2] = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // dM = 2 dSigma M; M = R diag(s): dR = dM diag(s), ds_c = sum_r dM_rc R_rc
            const float dM = 2.f * (dSf[3 * r] * M[c] + dSf[3 * r + 1] * M[3 + c] + dSf[3 * r + 2] * M[6 + c]);
            dR[3 * r + c] = dM * G.s[c];
            ds[c] = fmaf(dM, G.R[3 * r + c], ds[c]);
        }
    float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
    float dqn[4];
    dqn[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dqn[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                    w * dR[7] - 2.f * x * dR[8]);
    dqn[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                    z * dR[7] - 2.f * y * dR[8]);
    dqn[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] +
                    y * dR[5] + x * dR[6] + y * dR[7]);
    float dot = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
    float iq = 1.f / G.qlen;
    p.d_mean[3 * j] = dmu[0];
    p.d_mean[3 * j + 1] = dmu[1];
    p.d_mean[3 * j + 2] = dmu[2];
    reinterpret_cast<float4 *>(p.d_quat)[j] =
        make_float4((dqn[0] - w * dot) * iq, (dqn[1] - x * dot) * iq, (dqn[2] - y * dot) * iq,
                    (dqn[3] - z * dot) * iq);
}

// FULL = false: gradients wrt mean and rotation of every Gaussian (Stage 1).
// FULL = true: gradients wrt every parameter of Gaussians [first, first + count)
// (Stage 2), written at row j = i - first.
template <bool FULL, int DEG>
__global__ void __launch_bounds__(128) project_bwd_kernel(ProjectParams p)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    extern __shared__ gs_camera s_cams[];
    for (int k = threadIdx.x; k < p.V; k += blockDim.x) s_cams[k] = p.cams[k];
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (FULL ? p.count : p.n)) return;
    const int64_t i = FULL ? p.first + j : j;
    GaussLocal G;
    load_gauss(p, i, G);
    const float *sh = p.sh + (int64_t)3 * K * i;
    float *dsh = FULL ? p.d_sh + (int64_t)3 * K * j : nullptr;
    if (FULL)
#pragma unroll
        for (int k = 0; k < 3 * K; ++k) dsh[k] = 0.f;
    float dmu[3] = {0.f, 0.f, 0.f};
    float dS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/dSigma, symmetric (00 01 02 11 12 22)
    float dop = 0.f;
    for (int v = 0; v < p.V; ++v) {
        const gs_camera &c = s_cams[v];
        ViewLocal L;
        project_view<DEG>(p, G, sh, c, L);
        if (!L.valid) continue;
        const float4 *gp = reinterpret_cast<const float4 *>(p.grads + 8 * ((int64_t)v * p.n + i));
        float4 g0 = gp[0], g1 = gp[1];
        float drgb[3] = {g1.y, g1.z, g1.w};
        if (FULL) {
            // SH coefficients: d rgb_raw / d sh_k = Y_k where the colour is not clamped
            float Y[16];
            sh_basis(DEG, L.dir.x, L.dir.y, L.dir.z, Y);
#pragma unroll
            for (int k = 0; k < K; ++k)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
                    if (L.rgb_raw[ch] > 0.f) dsh[3 * k + ch] = fmaf(Y[k], drgb[ch], dsh[3 * k + ch]);
            if (p.d_opacity) dop += p.d_opacity[(int64_t)v * p.n + i];
        }
        bwd_view<DEG>(G, sh, c, L, g0, g1, dmu, dS);
    }
    float ds[3];
    bwd_finish(p, G, j, dmu, dS, ds);
    if (FULL) {
        p.d_scale[3 * j] = ds[0];
        p.d_scale[3 * j + 1] = ds[1];
        p.d_scale[3 * j + 2] = ds[2];
        p.d_ologit[j] = dop * G.op * (1.f - G.op);  // opacity = sigmoid(logit)
    }
}

// Stage-1 reverse with the views of a Gaussian in parallel: VP adjacent lanes
// (VP the power of two >= V, <= 32) take one Gaussian, lane v its view v;
// the per-view sums of dL/dmu and dL/dSigma are reduced over the lanes with
// shuffles and the group's first lane finishes the Gaussian.
template <int DEG, int VP>
__global__ void __launch_bounds__(128) project_bwd_views_kernel(ProjectParams p)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    extern __shared__ gs_camera s_cams[];
    for (int k = threadIdx.x; k < p.V; k += blockDim.x) s_cams[k] = p.cams[k];
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / VP;
    const int v = (int)(t % VP);
    const bool live = i < p.n;
    float dmu[3] = {0.f, 0.f, 0.f};
    float dS[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    GaussLocal G;
    if (live) {
        load_gauss(p, i, G);
        if (v < p.V) {
            float sh[3 * K];
            load_sh<DEG>(p, i, sh);
            const gs_camera &c = s_cams[v];
            ViewLocal L;
            project_view<DEG>(p, G, sh, c, L);
            if (L.valid) {
                const float4 *gp = reinterpret_cast<const float4 *>(p.grads + 8 * ((int64_t)v * p.n + i));
                bwd_view<DEG>(G, sh, c, L, gp[0], gp[1], dmu, dS);
            }
        }
    }
#pragma unroll
    for (int o = VP / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) dmu[a] += __shfl_xor_sync(0xffffffffu, dmu[a], o);
#pragma unroll
        for (int a = 0; a < 6; ++a) dS[a] += __shfl_xor_sync(0xffffffffu, dS[a], o);
    }
    if (live && v == 0) {
        float ds[3];
        bwd_finish(p, G, i, dmu, dS, ds);
    }
}

template <int DEG>
static void launch_bwd_views(const ProjectParams &p, size_t shm, cudaStream_t s)
{
    const int threads = 128;
    auto go = [&](auto vp) {
        constexpr int VP = decltype(vp)::value;
        const int blocks = (int)ceil_div(p.n * VP, threads);
        project_bwd_views_kernel<DEG, VP><<<blocks, threads, shm, s>>>(p);
    };
    if (p.V <= 1) go(std::integral_constant<int, 1>());
    else if (p.V <= 2) go(std::integral_constant<int, 2>());
    else if (p.V <= 4) go(std::integral_constant<int, 4>());
    else if (p.V <= 8) go(std::integral_constant<int, 8>());
    else if (p.V <= 16) go(std::integral_constant<int, 16>());
    else go(std::integral_constant<int, 32>());
}

template <bool FULL>
static void launch_bwd(const ProjectParams &p, int blocks, int threads, size_t shm, cudaStream_t s)
{
    switch (p.deg) {
    case 0: project_bwd_kernel<FULL, 0><<<blocks, threads, shm, s>>>(p); break;
    case 1: project_bwd_kernel<FULL, 1><<<blocks, threads, shm, s>>>(p); break;
    case 2: project_bwd_kernel<FULL, 2><<<blocks, threads, shm, s>>>(p); break;
    default: project_bwd_kernel<FULL, 3><<<blocks, threads, shm, s>>>(p); break;
    }
}

static gs_status fill_params(const gs_gaussians *g, const gs_camera *d_cams, int V, int W, int H,
                             ProjectParams &p)
{
    GS_REQUIRE(g && d_cams, "gs_project: null argument");
    GS_REQUIRE(g->n >= 0 && g->n < (int64_t(1) << 31), "gs_project: n out of range");
    GS_REQUIRE(g->sh_deg >= 0 && g->sh_deg <= 3, "gs_project: sh_deg must be 0..3");
    GS_REQUIRE(V >= 1 && V <= GS_MAX_VIEWS, "gs_project: V must be 1..%d", GS_MAX_VIEWS);
    GS_REQUIRE(W > 0 && H > 0 && W <= 16384 && H <= 16384, "gs_project: bad image size");
    GS_REQUIRE(aligned(g->quat, 16), "gs_project: quat must be 16-byte aligned");
    p.mean = g->mean;
    p.quat = g->quat;
    p.scale = g->scale;
    p.opl = g->opacity_logit;
    p.sh = g->sh;
    p.sh_vec4 = aligned(g->sh, 16);
    p.n = g->n;
    p.deg = g->sh_deg;
    p.K = (g->sh_deg + 1) * (g->sh_deg + 1);
    p.cams = d_cams;
    p.V = V;
    p.W = W;
    p.H = H;
    p.tx = tiles_x_of(W);
    p.ty = tiles_y_of(H);
    return GS_OK;
}

}  // namespace gs3

using namespace gs3;

extern "C" gs_status gs_project(const gs_gaussians *g, const gs_camera *d_cams, int V, int W, int H,
                                const gs_projected *out, int32_t *d_err, gs_stream stream)
{
    ProjectParams p{};
    gs_status st = fill_params(g, d_cams, V, W, H, p);
    if (st != GS_OK) return st;
    if (p.n == 0) return GS_OK;   // empty arrays may be null
    GS_REQUIRE(out && out->mean2d && out->conic_opacity && out->rgb && out->depth && out->radius &&
                   out->tiles_touched,
               "gs_project: null output");
    GS_REQUIRE(aligned(out->mean2d, 8) && aligned(out->conic_opacity, 16),
               "gs_project: mean2d / conic_opacity misaligned");
    p.mean2d = reinterpret_cast<float2 *>(out->mean2d);
    p.conic_op = reinterpret_cast<float4 *>(out->conic_opacity);
    p.rgb = out->rgb;
    p.depth = out->depth;
    p.radius = out->radius;
    p.tiles = out->tiles_touched;
    p.d_err = d_err;
    int threads = 256;
    int blocks = (int)ceil_div(p.n, threads);
    note_launch();
    const size_t shm = sizeof(gs_camera) * V;
    cudaStream_t s = as_stream(stream);
    switch (p.deg) {
    case 0: project_fwd_kernel<0><<<blocks, threads, shm, s>>>(p); break;
    case 1: project_fwd_kernel<1><<<blocks, threads, shm, s>>>(p); break;
    case 2: project_fwd_kernel<2><<<blocks, threads, shm, s>>>(p); break;
    default: project_fwd_kernel<3><<<blocks, threads, shm, s>>>(p); break;
    }
    return launch_status("gs_project");
}

extern "C" gs_status gs_project_bwd(const gs_gaussians *g, const gs_camera *d_cams, int V, int W,
                                    int H, const float *grads, float *d_mean, float *d_quat,
                                    gs_stream stream)
{
    ProjectParams p{};
    gs_status st = fill_params(g, d_cams, V, W, H, p);
    if (st != GS_OK) return st;
    if (p.n == 0) return GS_OK;
    GS_REQUIRE(grads && d_mean && d_quat, "gs_project_bwd: null argument");
    GS_REQUIRE(aligned(grads, 16) && aligned(d_quat, 16), "gs_project_bwd: misaligned arrays");
    p.grads = grads;
    p.d_mean = d_mean;
    p.d_quat = d_quat;
    int threads = 128;
    int blocks = (int)ceil_div(p.n, threads);
    note_launch();
    const size_t shm = sizeof(gs_camera) * V;
    cudaStream_t s = as_stream(stream);
    if (V <= 32) {
        switch (p.deg) {
        case 0: launch_bwd_views<0>(p, shm, s); break;
        case 1: launch_bwd_views<1>(p, shm, s); break;
        case 2: launch_bwd_views<2>(p, shm, s); break;
        default: launch_bwd_views<3>(p, shm, s); break;
        }
    } else {
        launch_bwd<false>(p, blocks, threads, shm, s);
    }
    return launch_status("gs_project_bwd");
}

extern "C" gs_status gs_project_bwd_full(const gs_gaussians *g, const gs_camera *d_cams, int V,
                                         int W, int H, const float *grads, const float *d_opacity,
                                         int64_t first, int64_t count, float *d_mean,
                                         float *d_quat, float *d_scale, float *d_opacity_logit,
                                         float *d_sh, gs_stream stream)
{
    ProjectParams p{};
    gs_status st = fill_params(g, d_cams, V, W, H, p);
    if (st != GS_OK) return st;
    GS_REQUIRE(first >= 0 && count >= 0 && first + count <= g->n,
               "gs_project_bwd_full: range [first, first + count) outside the Gaussians");
    if (count == 0) return GS_OK;
    GS_REQUIRE(grads && d_mean && d_quat && d_scale && d_opacity_logit && d_sh,
               "gs_project_bwd_full: null argument");
    GS_REQUIRE(aligned(grads, 16) && aligned(d_quat, 16), "gs_project_bwd_full: misaligned arrays");
    p.grads = grads;
    p.d_opacity = d_opacity;
    p.first = first;
    p.count = count;
    p.d_mean = d_mean;
    p.d_quat = d_quat;
    p.d_scale = d_scale;
    p.d_ologit = d_opacity_logit;
    p.d_sh = d_sh;
    int threads = 128;
    int blocks = (int)ceil_div(count, threads);
    note_launch();
    launch_bwd<true>(p, blocks, threads, sizeof(gs_camera) * V, as_stream(stream));
    return launch_status("gs_project_bwd_full");
}

// SH rotation (Suppl. B): after a Gaussian is rotated by the world rotation
// Rw = R(q_to) R(q_from)^T, its view-dependent colour f(d) becomes f(Rw^T d),
// which rotates each SH band l >= 1 by the matrix M_l with
//   M_l P_l(N) = P_l(Rw N)  for every direction N,
// P_l(N) being the band-l basis values at N.  With 2l + 1 fixed directions
// N_k and A_l = [P_l(N_0) ... P_l(N_2l)] invertible,
//   M_l = [P_l(Rw N_0) ... P_l(Rw N_2l)] A_l^-1,
// and the band's coefficients (per colour channel) become M_l c.  Band 1 uses
// the coordinate axes (the supplement's choice); bands 2 and 3 use 5 and 7
// points of a Fibonacci lattice on the sphere (offset 0.1; condition numbers
// of A_l about 8 and 4).  A_l^-1 is computed once on the host in double.
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "sh.cuh"

namespace gs3 {

struct ShRotParams {
    float dirs[3 + 5 + 7][3];   // N_k of bands 1, 2, 3
    float ainv[9 + 25 + 49];    // A_l^-1 of bands 1, 2, 3, row-major
};

static const int kBandOff[4] = {0, 0, 3, 8};          // first direction of band l
static const int kAinvOff[4] = {0, 0, 9, 34};         // first entry of A_l^-1

static void fibonacci_dirs(int n, double off, double (*out)[3])
{
    const double ga = 3.14159265358979323846 * (3.0 - sqrt(5.0));  // golden angle
    for (int i = 0; i < n; ++i) {
        double t = i + off, z = 1.0 - 2.0 * t / n, r = sqrt(1.0 - z * z), phi = t * ga;
        out[i][0] = r * cos(phi);
        out[i][1] = r * sin(phi);
        out[i][2] = z;
    }
}

// Gauss-Jordan inverse with partial pivoting of an n x n matrix (n <= 7).
static bool invert(int n, double *a, double *inv)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[i * n + j] = i == j ? 1.0 : 0.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(a[r * n + c]) > fabs(a[p * n + c])) p = r;
        if (fabs(a[p * n + c]) < 1e-12) return false;
        for (int j = 0; j < n; ++j) {
            double t = a[c * n + j]; a[c * n + j] = a[p * n + j]; a[p * n + j] = t;
            t = inv[c * n + j]; inv[c * n + j] = inv[p * n + j]; inv[p * n + j] = t;
        }
        double d = a[c * n + c];
        for (int j = 0; j < n; ++j) {
            a[c * n + j] /= d;
            inv[c * n + j] /= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = a[r * n + c];
            for (int j = 0; j < n; ++j) {
                a[r * n + j] -= f * a[c * n + j];
                inv[r * n + j] -= f * inv[c * n + j];
            }
        }
    }
    return true;
}

static const ShRotParams &shrot_params()
{
    static ShRotParams P;
    static std::once_flag once;
    std::call_once(once, [] {
        double d[15][3];
        const double axes[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) d[k][a] = axes[k][a];
        fibonacci_dirs(5, 0.1, d + 3);
        fibonacci_dirs(7, 0.1, d + 8);
        for (int k = 0; k < 15; ++k)
            for (int a = 0; a < 3; ++a) P.dirs[k][a] = (float)d[k][a];
        for (int l = 1; l <= 3; ++l) {
            const int n = 2 * l + 1, b0 = l * l;
            double A[49], inv[49], Y[16];
            for (int k = 0; k < n; ++k) {  // column k = P_l(N_k)
                const double *v = d[kBandOff[l] + k];
                sh_basis_t<double>(3, v[0], v[1], v[2], Y);
                for (int r = 0; r < n; ++r) A[r * n + k] = Y[b0 + r];
            }
            invert(n, A, inv);
            for (int e = 0; e < n * n; ++e) P.ainv[kAinvOff[l] + e] = (float)inv[e];
        }
    });
    return P;
}

__device__ __forceinline__ void quat_rot(const float *q, float *R)
{
    float l = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    float il = 1.f / fmaxf(l, 1e-12f);
    float w = q[0] * il, x = q[1] * il, y = q[2] * il, z = q[3] * il;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

template <int DEG>
__global__ void sh_rotate_kernel(const float4 *q_from, const float4 *q_to, const float *sh_in,
                                 int64_t n, float *sh_out, ShRotParams P)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float c[K][3];
    const float *src = sh_in + (int64_t)3 * K * i;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) c[k][ch] = src[3 * k + ch];
    float Ra[9], Rb[9], Rw[9];
    const float4 qa = q_from[i], qb = q_to[i];
    const float fa[4] = {qa.x, qa.y, qa.z, qa.w}, fb[4] = {qb.x, qb.y, qb.z, qb.w};
    quat_rot(fa, Ra);
    quat_rot(fb, Rb);
#pragma unroll
    for (int r = 0; r < 3; ++r)  // Rw = Rb Ra^T
#pragma unroll
        for (int s = 0; s < 3; ++s)
            Rw[3 * r + s] = Rb[3 * r] * Ra[3 * s] + Rb[3 * r + 1] * Ra[3 * s + 1] + Rb[3 * r + 2] * Ra[3 * s + 2];
    float *dst = sh_out + (int64_t)3 * K * i;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) dst[ch] = c[0][ch];  // band 0 is rotation invariant
#pragma unroll
    for (int l = 1; l <= DEG; ++l) {
        const int nl = 2 * l + 1, b0 = l * l;
        // B[r][k] = P_l(Rw N_k)[r]
        float B[7][7];
#pragma unroll
        for (int k = 0; k < nl; ++k) {
            const float *v = P.dirs[(l == 1 ? 0 : l == 2 ? 3 : 8) + k];
            float x = Rw[0] * v[0] + Rw[1] * v[1] + Rw[2] * v[2];
            float y = Rw[3] * v[0] + Rw[4] * v[1] + Rw[5] * v[2];
            float z = Rw[6] * v[0] + Rw[7] * v[1] + Rw[8] * v[2];
            float Y[16];
            sh_basis_t<float>(l, x, y, z, Y);
#pragma unroll
            for (int r = 0; r < nl; ++r) B[r][k] = Y[b0 + r];
        }
        const float *Ai = P.ainv + (l == 1 ? 0 : l == 2 ? 9 : 34);
        // M = B A^-1;  c'_band = M c_band
#pragma unroll
        for (int r = 0; r < nl; ++r) {
            float m[7];
#pragma unroll
            for (int s = 0; s < nl; ++s) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < nl; ++k) acc = fmaf(B[r][k], Ai[k * nl + s], acc);
                m[s] = acc;
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float acc = 0.f;
#pragma unroll
                for (int s = 0; s < nl; ++s) acc = fmaf(m[s], c[b0 + s][ch], acc);
                dst[3 * (b0 + r) + ch] = acc;
            }
        }
    }
}

}  // namespace gs3

using namespace gs3;

extern "C" gs_status gs_sh_rotate(const float *quat_from, const float *quat_to, const float *sh_in,
                                  int64_t n, int sh_deg, float *sh_out, gs_stream stream)
{
    GS_REQUIRE(quat_from && quat_to && sh_in && sh_out, "gs_sh_rotate: null argument");
    GS_REQUIRE(n >= 0 && sh_deg >= 0 && sh_deg <= 3, "gs_sh_rotate: bad n or sh_deg");
    GS_REQUIRE(aligned(quat_from, 16) && aligned(quat_to, 16), "gs_sh_rotate: quaternions misaligned");
    if (n == 0) return GS_OK;
    const ShRotParams &P = shrot_params();
    const float4 *qa = reinterpret_cast<const float4 *>(quat_from);
    const float4 *qb = reinterpret_cast<const float4 *>(quat_to);
    const int blocks = (int)ceil_div(n, 128);
    cudaStream_t s = as_stream(stream);
    note_launch();
    switch (sh_deg) {
    case 0: sh_rotate_kernel<0><<<blocks, 128, 0, s>>>(qa, qb, sh_in, n, sh_out, P); break;
    case 1: sh_rotate_kernel<1><<<blocks, 128, 0, s>>>(qa, qb, sh_in, n, sh_out, P); break;
    case 2: sh_rotate_kernel<2><<<blocks, 128, 0, s>>>(qa, qb, sh_in, n, sh_out, P); break;
    default: sh_rotate_kernel<3><<<blocks, 128, 0, s>>>(qa, qb, sh_in, n, sh_out, P); break;
    }
    return launch_status("gs_sh_rotate");
}

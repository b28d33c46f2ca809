// Stage 2 of the per-frame reconstruction (Section 4.2, adaptive 3DG
// addition): view-space gradient statistics, selection of the Gaussians above
// the gradient threshold, spawning of added Gaussians around them, the
// per-epoch split-and-prune of the added set, and their Adam update.
//
// The added Gaussians live as rows of trainable parameters
//   [mean 3 | quat 4 | log scale 3 | opacity logit 1 | SH K x 3]
// with Adam moments in the same layout; after each update their rendered
// attributes are written into the tail of the Gaussian set the rasterizer
// draws (the transformed Gaussians first, fixed, then the added ones).
#include <math.h>

#include "common.cuh"

namespace gs3 {

constexpr int COL_MEAN = 0, COL_QUAT = 3, COL_LOGS = 7, COL_OPL = 10, COL_SH = 11;

__host__ __device__ __forceinline__ int added_cols(int K) { return COL_SH + 3 * K; }

__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float *R)
{
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// mean + f * R(q) diag(s) z: a draw from N(mean, f^2 Sigma) for z ~ N(0, I)
__device__ __forceinline__ void sample_around(const float *mu, const float *q, const float *s,
                                              const float *z, float f, float *out)
{
    float l = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    float il = 1.f / fmaxf(l, 1e-12f);
    float R[9];
    quat_to_rot(q[0] * il, q[1] * il, q[2] * il, q[3] * il, R);
    const float a = s[0] * z[0], b = s[1] * z[1], c = s[2] * z[2];
#pragma unroll
    for (int r = 0; r < 3; ++r) out[r] = mu[r] + f * (R[3 * r] * a + R[3 * r + 1] * b + R[3 * r + 2] * c);
}

// ------------------------------------------------------------ statistics
__global__ void viewspace_accum_kernel(const float *grads, const int32_t *radius, int V, int64_t n,
                                       int64_t first, int64_t count, float hw, float hh,
                                       float grad_scale, float *accum, int32_t *denom)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const int64_t i = first + j;
    float acc = 0.f;
    int cnt = 0;
    for (int v = 0; v < V; ++v) {
        const int64_t o = (int64_t)v * n + i;
        if (radius[o] <= 0) continue;
        const float2 g = *reinterpret_cast<const float2 *>(grads + 8 * o);
        const float gx = g.x * hw, gy = g.y * hh;
        acc += grad_scale * sqrtf(gx * gx + gy * gy);
        ++cnt;
    }
    accum[j] += acc;
    denom[j] += cnt;
}

// ------------------------------------------------------------- selection
constexpr int SEL_THREADS = 1024;

__device__ __forceinline__ bool above(const float *accum, const int32_t *denom, int64_t j, float tau)
{
    const int d = denom[j];
    return d > 0 && accum[j] / (float)d > tau;
}

// Block-wide exclusive scan of one int per thread; returns the total.  Ends
// with a barrier, so it can be called again at once.
__device__ __forceinline__ int block_scan(int x, int &excl)
{
    constexpr int NW = SEL_THREADS / 32;
    __shared__ int s_w[NW];
    __shared__ int s_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < NW ? s_w[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NW) s_w[lane] = wi - w;  // exclusive offsets of the warps
        if (lane == NW - 1) s_tot = wi;
    }
    __syncthreads();
    excl = s_w[warp] + incl - x;
    const int total = s_tot;
    __syncthreads();
    return total;
}

// One block: thread t owns the contiguous chunk [t c, (t + 1) c).
__global__ void __launch_bounds__(SEL_THREADS) select_above_kernel(const float *accum,
                                                                   const int32_t *denom,
                                                                   int64_t count, float tau,
                                                                   int32_t *idx, int64_t *d_nsel)
{
    const int64_t c = (count + SEL_THREADS - 1) / SEL_THREADS;
    const int64_t b = threadIdx.x * c, e = min(count, b + c);
    int mine = 0;
    for (int64_t j = b; j < e; ++j) mine += above(accum, denom, j, tau);
    int off;
    const int total = block_scan(mine, off);
    for (int64_t j = b; j < e; ++j)
        if (above(accum, denom, j, tau)) idx[off++] = (int32_t)j;
    if (threadIdx.x == 0) *d_nsel = total;
}

// ------------------------------------------------------------------ spawn
__global__ void spawn_kernel(gs_gaussians src, const int32_t *idx, const int64_t *d_nsel,
                             const float *z, float opl_init, gs_added dst, int64_t *d_nadd,
                             int32_t *d_err)
{
    const int64_t nsel = *d_nsel, n0 = *d_nadd;
    const int K = (src.sh_deg + 1) * (src.sh_deg + 1), P = added_cols(K);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nsel;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = n0 + k;
        if (row >= dst.capacity) {
            *d_err = GS_ERR_CAPACITY;
            continue;
        }
        const int64_t i = idx[k];
        float *r = dst.rows + row * P;
        float q[4] = {src.quat[4 * i], src.quat[4 * i + 1], src.quat[4 * i + 2], src.quat[4 * i + 3]};
        sample_around(src.mean + 3 * i, q, src.scale + 3 * i, z + 3 * k, 1.41421356237f, r + COL_MEAN);
        r[COL_QUAT] = 1.f;
        r[COL_QUAT + 1] = 0.f;
        r[COL_QUAT + 2] = 0.f;
        r[COL_QUAT + 3] = 0.f;
        for (int a = 0; a < 3; ++a) r[COL_LOGS + a] = logf(src.scale[3 * i + a]);
        r[COL_OPL] = opl_init;
        for (int e = 0; e < 3 * K; ++e) r[COL_SH + e] = src.sh[(int64_t)3 * K * i + e];
        for (int e = 0; e < P; ++e) {
            dst.m[row * P + e] = 0.f;
            dst.v[row * P + e] = 0.f;
        }
    }
}

__global__ void spawn_count_kernel(const int64_t *d_nsel, int64_t cap, int64_t *d_nadd)
{
    *d_nadd = min(cap, *d_nadd + *d_nsel);
}

// ------------------------------------------------------- split and prune
__global__ void __launch_bounds__(SEL_THREADS) densify_prune_kernel(
    gs_added src, int64_t n_src, const float *accum, const int32_t *denom, float tau_grad,
    float opl_min, float log_split, float opl_child, const float *z, gs_added dst, int64_t *d_ndst,
    int32_t *d_err)
{
    const int K = (src.sh_deg + 1) * (src.sh_deg + 1), P = added_cols(K);
    const int64_t c = (n_src + SEL_THREADS - 1) / SEL_THREADS;
    const int64_t b = threadIdx.x * c, e = min(n_src, b + c);
    auto kept = [&](int64_t j) { return src.rows[j * P + COL_OPL] >= opl_min; };
    int nk = 0, ns = 0;
    for (int64_t j = b; j < e; ++j) {
        const bool k = kept(j);
        nk += k;
        ns += k && above(accum, denom, j, tau_grad);
    }
    int ok, os;
    const int tk = block_scan(nk, ok);
    block_scan(ns, os);
    os += tk;  // split rows follow all kept rows
    for (int64_t j = b; j < e; ++j) {
        if (!kept(j)) continue;
        const float *r = src.rows + j * P;
        if (ok < dst.capacity) {
            for (int q = 0; q < P; ++q) {
                dst.rows[ok * P + q] = r[q];
                dst.m[ok * P + q] = src.m[j * P + q];
                dst.v[ok * P + q] = src.v[j * P + q];
            }
        } else {
            *d_err = GS_ERR_CAPACITY;
        }
        ++ok;
        if (!above(accum, denom, j, tau_grad)) continue;
        if (os < dst.capacity) {
            float *w = dst.rows + os * P;
            const float s[3] = {expf(r[COL_LOGS]), expf(r[COL_LOGS + 1]), expf(r[COL_LOGS + 2])};
            sample_around(r + COL_MEAN, r + COL_QUAT, s, z + 3 * j, 1.f, w + COL_MEAN);
            for (int q = COL_QUAT; q < P; ++q) w[q] = r[q];
            for (int a = 0; a < 3; ++a) w[COL_LOGS + a] = r[COL_LOGS + a] + log_split;
            w[COL_OPL] = opl_child;
            for (int q = 0; q < P; ++q) {
                dst.m[os * P + q] = 0.f;
                dst.v[os * P + q] = 0.f;
            }
        } else {
            *d_err = GS_ERR_CAPACITY;
        }
        ++os;
    }
    __syncthreads();
    if (threadIdx.x == SEL_THREADS - 1) *d_ndst = min((int64_t)dst.capacity, (int64_t)os);
}

// -------------------------------------------------------- Adam + render
// gs_gaussians holds read-only pointers for the rasterizer; here its arrays
// are the destination of the added rows' rendered attributes.
__device__ __forceinline__ void row_to_render(const float *r, int K, gs_gaussians out, int64_t o)
{
    float *mean = const_cast<float *>(out.mean), *scale = const_cast<float *>(out.scale);
    float *opl = const_cast<float *>(out.opacity_logit), *sh = const_cast<float *>(out.sh);
    float4 *quat = reinterpret_cast<float4 *>(const_cast<float *>(out.quat));
    for (int a = 0; a < 3; ++a) mean[3 * o + a] = r[COL_MEAN + a];
    quat[o] = make_float4(r[COL_QUAT], r[COL_QUAT + 1], r[COL_QUAT + 2], r[COL_QUAT + 3]);
    for (int a = 0; a < 3; ++a) scale[3 * o + a] = expf(r[COL_LOGS + a]);
    opl[o] = r[COL_OPL];
    for (int e = 0; e < 3 * K; ++e) sh[(int64_t)3 * K * o + e] = r[COL_SH + e];
}

struct AdamLr {
    float lr[6];
};

__global__ void added_adam_kernel(gs_added a, int64_t n, const float *d_mean, const float *d_quat,
                                  const float *d_scale, const float *d_ologit, const float *d_sh,
                                  AdamLr lr, float b1, float b2, float eps,
                                  const gs_train_state *st, gs_gaussians out, int64_t out_first)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int K = (a.sh_deg + 1) * (a.sh_deg + 1), P = added_cols(K);
    float *r = a.rows + j * P, *m = a.m + j * P, *v = a.v + j * P;
    if (st->found_inf == 0) {
        // 1 - b^t as -expm1(t log b): no cancellation when b is close to 1
        const int t = st->step + 1;
        const float bc1 = -expm1f((float)t * logf(b1)), bc2 = -expm1f((float)t * logf(b2));
        for (int q = 0; q < P; ++q) {
            float g, l;
            if (q < COL_QUAT) {
                g = d_mean[3 * j + q];
                l = lr.lr[0];
            } else if (q < COL_LOGS) {
                g = d_quat[4 * j + q - COL_QUAT];
                l = lr.lr[1];
            } else if (q < COL_OPL) {
                // d/d log s = d/ds * s
                g = d_scale[3 * j + q - COL_LOGS] * expf(r[q]);
                l = lr.lr[2];
            } else if (q == COL_OPL) {
                g = d_ologit[j];
                l = lr.lr[3];
            } else {
                g = d_sh[(int64_t)3 * K * j + q - COL_SH];
                l = q < COL_SH + 3 ? lr.lr[4] : lr.lr[5];
            }
            const float mi = fmaf(b1, m[q], (1.f - b1) * g);
            const float vi = fmaf(b2, v[q], (1.f - b2) * g * g);
            m[q] = mi;
            v[q] = vi;
            r[q] = r[q] - l * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        }
    }
    row_to_render(r, K, out, out_first + j);
}

__global__ void added_render_kernel(gs_added a, int64_t n, gs_gaussians out, int64_t out_first)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int K = (a.sh_deg + 1) * (a.sh_deg + 1);
    row_to_render(a.rows + j * added_cols(K), K, out, out_first + j);
}

static bool added_ok(const gs_added *a)
{
    return a && a->rows && a->m && a->v && a->capacity >= 0 && a->sh_deg >= 0 && a->sh_deg <= 3;
}

}  // namespace gs3

using namespace gs3;

extern "C" gs_status gs_viewspace_grad_accum(const float *grads, const int32_t *radius, int V,
                                             int64_t n, int64_t first, int64_t count, int W, int H,
                                             float grad_scale, float *accum, int32_t *denom,
                                             gs_stream stream)
{
    GS_REQUIRE(grads && radius && accum && denom, "gs_viewspace_grad_accum: null argument");
    GS_REQUIRE(V >= 1 && n >= 0 && first >= 0 && count >= 0 && first + count <= n,
               "gs_viewspace_grad_accum: bad range");
    GS_REQUIRE(aligned(grads, 8), "gs_viewspace_grad_accum: grads misaligned");
    if (count == 0) return GS_OK;
    note_launch();
    viewspace_accum_kernel<<<(int)ceil_div(count, 256), 256, 0, as_stream(stream)>>>(
        grads, radius, V, n, first, count, 0.5f * (float)W, 0.5f * (float)H, grad_scale, accum, denom);
    return launch_status("gs_viewspace_grad_accum");
}

extern "C" gs_status gs_select_above(const float *accum, const int32_t *denom, int64_t count,
                                     float tau, int32_t *idx, int64_t *d_nsel, gs_stream stream)
{
    GS_REQUIRE(accum && denom && idx && d_nsel, "gs_select_above: null argument");
    GS_REQUIRE(count >= 0 && count < (int64_t(1) << 31), "gs_select_above: bad count");
    note_launch();
    select_above_kernel<<<1, SEL_THREADS, 0, as_stream(stream)>>>(accum, denom, count, tau, idx, d_nsel);
    return launch_status("gs_select_above");
}

extern "C" gs_status gs_added_spawn(const gs_gaussians *src, const int32_t *idx,
                                    const int64_t *d_nsel, const float *z, float opacity_init,
                                    gs_added *dst, int64_t *d_nadd, int32_t *d_err,
                                    gs_stream stream)
{
    GS_REQUIRE(src && idx && d_nsel && z && d_nadd && d_err && added_ok(dst),
               "gs_added_spawn: null argument");
    GS_REQUIRE(src->sh_deg == dst->sh_deg, "gs_added_spawn: SH degrees differ");
    GS_REQUIRE(opacity_init > 0.f && opacity_init < 1.f, "gs_added_spawn: opacity_init in (0, 1)");
    GS_REQUIRE(aligned(src->quat, 16), "gs_added_spawn: quat misaligned");
    cudaStream_t s = as_stream(stream);
    const float opl = logf(opacity_init / (1.f - opacity_init));
    note_launch();
    spawn_kernel<<<num_sms() * 4, 256, 0, s>>>(*src, idx, d_nsel, z, opl, *dst, d_nadd, d_err);
    note_launch();
    spawn_count_kernel<<<1, 1, 0, s>>>(d_nsel, dst->capacity, d_nadd);
    return launch_status("gs_added_spawn");
}

extern "C" gs_status gs_added_densify_prune(const gs_added *src, int64_t n_src, const float *accum,
                                            const int32_t *denom, float tau_grad,
                                            float tau_opacity, float split_scale,
                                            float opacity_init, const float *z, gs_added *dst,
                                            int64_t *d_ndst, int32_t *d_err, gs_stream stream)
{
    GS_REQUIRE(added_ok(src) && added_ok(dst) && accum && denom && z && d_ndst && d_err,
               "gs_added_densify_prune: null argument");
    GS_REQUIRE(src->sh_deg == dst->sh_deg && src->rows != dst->rows,
               "gs_added_densify_prune: dst must be another buffer of the same SH degree");
    GS_REQUIRE(n_src >= 0 && n_src <= src->capacity, "gs_added_densify_prune: bad n_src");
    GS_REQUIRE(tau_opacity > 0.f && tau_opacity < 1.f && split_scale > 0.f && opacity_init > 0.f &&
                   opacity_init < 1.f,
               "gs_added_densify_prune: bad thresholds");
    note_launch();
    densify_prune_kernel<<<1, SEL_THREADS, 0, as_stream(stream)>>>(
        *src, n_src, accum, denom, tau_grad, logf(tau_opacity / (1.f - tau_opacity)),
        logf(split_scale), logf(opacity_init / (1.f - opacity_init)), z, *dst, d_ndst, d_err);
    return launch_status("gs_added_densify_prune");
}

extern "C" gs_status gs_added_adam(gs_added *a, int64_t n, const float *d_mean, const float *d_quat,
                                   const float *d_scale, const float *d_opacity_logit,
                                   const float *d_sh, const float *lr, float beta1, float beta2,
                                   float eps, const gs_train_state *d_state,
                                   const gs_gaussians *out, int64_t out_first, gs_stream stream)
{
    GS_REQUIRE(added_ok(a) && d_mean && d_quat && d_scale && d_opacity_logit && d_sh && lr &&
                   d_state && out,
               "gs_added_adam: null argument");
    GS_REQUIRE(n >= 0 && n <= a->capacity && out_first >= 0 && out_first + n <= out->n,
               "gs_added_adam: bad row range");
    GS_REQUIRE(out->sh_deg == a->sh_deg && aligned(out->quat, 16), "gs_added_adam: bad output set");
    if (n == 0) return GS_OK;
    AdamLr l;
    for (int k = 0; k < 6; ++k) l.lr[k] = lr[k];
    note_launch();
    added_adam_kernel<<<(int)ceil_div(n, 128), 128, 0, as_stream(stream)>>>(
        *a, n, d_mean, d_quat, d_scale, d_opacity_logit, d_sh, l, beta1, beta2, eps, d_state, *out,
        out_first);
    return launch_status("gs_added_adam");
}

extern "C" gs_status gs_added_to_render(const gs_added *a, int64_t n, const gs_gaussians *out,
                                        int64_t out_first, gs_stream stream)
{
    GS_REQUIRE(added_ok(a) && out, "gs_added_to_render: null argument");
    GS_REQUIRE(n >= 0 && n <= a->capacity && out_first >= 0 && out_first + n <= out->n,
               "gs_added_to_render: bad row range");
    GS_REQUIRE(out->sh_deg == a->sh_deg && aligned(out->quat, 16), "gs_added_to_render: bad output set");
    if (n == 0) return GS_OK;
    note_launch();
    added_render_kernel<<<(int)ceil_div(n, 128), 128, 0, as_stream(stream)>>>(*a, n, *out, out_first);
    return launch_status("gs_added_to_render");
}

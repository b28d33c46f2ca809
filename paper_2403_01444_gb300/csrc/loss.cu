// L1 + D-SSIM loss and its gradient (Section 4.1, Eq. 6).
// Pass 1 filters (x, y, x^2, y^2, xy) with the separable 11x11 Gaussian window
// through shared memory, forms the SSIM map and the three per-pixel
// coefficients of its derivative wrt (mu_x, E[x^2], E[xy]); pass 2 filters
// those coefficients (the window is symmetric, so the adjoint is the same
// filter) and assembles dL/dI; pass 3 reduces the block partial sums in FP64.
#include <math.h>

#include "common.cuh"

namespace gs3 {

constexpr int LT = 32;          // output tile side
constexpr int LH = 5;           // window half-width
constexpr int LS = LT + 2 * LH; // staged tile side (42)
constexpr int LTHREADS = 256;

// Normalised 11-tap Gaussian window (sigma 1.5), built by each block in
// shared memory (no constant-memory upload, so the call is capture-safe).
__device__ __forceinline__ void build_window(float *w)
{
    if (threadIdx.x < 11) {
        float s = 0.f;
        for (int i = 0; i < 11; ++i) s += expf(-(float)((i - 5) * (i - 5)) / 4.5f);
        int i = threadIdx.x;
        w[i] = expf(-(float)((i - 5) * (i - 5)) / 4.5f) / s;
    }
}

struct LossParams {
    const float *x, *y;
    int P, H, W;
    float lam;
    float *ca, *cb, *cc;  // per-pixel derivative coefficients
    double *partial;      // [blocks][2]: sum of SSIM map, sum |x - y|
    float *d_img;
    float *d_loss, *d_ssim;
    int nblocks;
};

// Horizontal pass work split: a thread filters HSEG consecutive outputs of
// one staged row, keeping the HSEG + 10 inputs in registers; the vertical
// pass gives a thread VSEG consecutive rows of one column.
constexpr int HSEG = 8;
constexpr int VSEG = 4;
static_assert(LT % HSEG == 0 && LT % VSEG == 0, "tile split");
static_assert((LT / VSEG) * LT == LTHREADS, "vertical pass: one item per thread");

__global__ void __launch_bounds__(LTHREADS) ssim_fwd_kernel(LossParams p)
{
    __shared__ float sx[LS][LS + 1], sy[LS][LS + 1];
    __shared__ float hs[5][LS][LT + 1];
    __shared__ double red[2][LTHREADS / 32];
    __shared__ float c_win[11];
    build_window(c_win);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * LT, y0 = blockIdx.y * LT, pl = blockIdx.z;
    const int64_t HW = (int64_t)p.H * p.W;
    const float *X = p.x + pl * HW, *Y = p.y + pl * HW;
    for (int i = tid; i < LS * LS; i += LTHREADS) {
        int r = i / LS, c = i % LS;
        int gy = y0 - LH + r, gx = x0 - LH + c;
        bool in = gy >= 0 && gy < p.H && gx >= 0 && gx < p.W;
        int64_t o = (int64_t)gy * p.W + gx;
        sx[r][c] = in ? X[o] : 0.f;
        sy[r][c] = in ? Y[o] : 0.f;
    }
    __syncthreads();
    float w[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) w[k] = c_win[k];
    // horizontal: (x, y, x^2, y^2, xy) filtered along rows.  Each staged input
    // is read and squared once and added into the HSEG outputs it reaches;
    // every output still sums its taps in increasing order.
    for (int item = tid; item < LS * (LT / HSEG); item += LTHREADS) {
        const int r = item / (LT / HSEG), c0 = (item % (LT / HSEG)) * HSEG;
        float acc[HSEG][5];
#pragma unroll
        for (int o = 0; o < HSEG; ++o)
#pragma unroll
            for (int q = 0; q < 5; ++q) acc[o][q] = 0.f;
#pragma unroll
        for (int k = 0; k < HSEG + 10; ++k) {
            const float a = sx[r][c0 + k], b = sy[r][c0 + k];
            const float aa = a * a, bb = b * b, ab = a * b;
#pragma unroll
            for (int o = 0; o < HSEG; ++o) {
                const int t = k - o;
                if (t < 0 || t > 10) continue;
                acc[o][0] = fmaf(w[t], a, acc[o][0]);
                acc[o][1] = fmaf(w[t], b, acc[o][1]);
                acc[o][2] = fmaf(w[t], aa, acc[o][2]);
                acc[o][3] = fmaf(w[t], bb, acc[o][3]);
                acc[o][4] = fmaf(w[t], ab, acc[o][4]);
            }
        }
#pragma unroll
        for (int o = 0; o < HSEG; ++o)
#pragma unroll
            for (int q = 0; q < 5; ++q) hs[q][r][c0 + o] = acc[o][q];
    }
    __syncthreads();
    // vertical: thread -> column c, rows r0 .. r0 + VSEG - 1
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    const int c = tid % LT, r0 = (tid / LT) * VSEG;
    float f[5][VSEG];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        float col[VSEG + 10];
#pragma unroll
        for (int k = 0; k < VSEG + 10; ++k) col[k] = hs[m][r0 + k][c];
#pragma unroll
        for (int o = 0; o < VSEG; ++o) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) acc = fmaf(w[k], col[o + k], acc);
            f[m][o] = acc;
        }
    }
    // per-thread and per-warp sums in FP32 (at most VSEG * 32 terms), the
    // block's and the final reduction in FP64
    float ssum = 0.f, lsum = 0.f;
    const int gx = x0 + c;
#pragma unroll
    for (int o = 0; o < VSEG; ++o) {
        const int r = r0 + o, gy = y0 + r;
        if (gy >= p.H || gx >= p.W) continue;
        float mx = f[0][o], my = f[1][o], exx = f[2][o], eyy = f[3][o], exy = f[4][o];
        float sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
        float n1 = 2.f * mx * my + C1, n2 = 2.f * sxy + C2;
        float d1 = mx * mx + my * my + C1, d2 = sxx + syy + C2;
        float idd = 1.f / (d1 * d2);
        float sv = n1 * n2 * idd;
        float ds_dmx = 2.f * my * n2 * idd - sv * 2.f * mx / d1;
        float ds_dsxx = -sv / d2;
        float ds_dsxy = 2.f * n1 * idd;
        int64_t oo = pl * HW + (int64_t)gy * p.W + gx;
        p.ca[oo] = ds_dmx - 2.f * mx * ds_dsxx - my * ds_dsxy;
        p.cb[oo] = ds_dsxx;
        p.cc[oo] = ds_dsxy;
        ssum += sv;
        lsum += fabsf(sx[r + LH][c + LH] - sy[r + LH][c + LH]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = (double)ssum;
        red[1][tid >> 5] = (double)lsum;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int ww = 0; ww < LTHREADS / 32; ++ww) {
            a += red[0][ww];
            b += red[1][ww];
        }
        int64_t bid = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        p.partial[2 * bid] = a;
        p.partial[2 * bid + 1] = b;
    }
}

__global__ void __launch_bounds__(LTHREADS) ssim_bwd_kernel(LossParams p)
{
    __shared__ float sa[LS][LS + 1], sb[LS][LS + 1], sc[LS][LS + 1];
    __shared__ float hs[3][LS][LT + 1];
    __shared__ float c_win[11];
    build_window(c_win);
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * LT, y0 = blockIdx.y * LT, pl = blockIdx.z;
    const int64_t HW = (int64_t)p.H * p.W;
    for (int i = tid; i < LS * LS; i += LTHREADS) {
        int r = i / LS, c = i % LS;
        int gy = y0 - LH + r, gx = x0 - LH + c;
        bool in = gy >= 0 && gy < p.H && gx >= 0 && gx < p.W;
        int64_t o = pl * HW + (int64_t)gy * p.W + gx;
        sa[r][c] = in ? p.ca[o] : 0.f;
        sb[r][c] = in ? p.cb[o] : 0.f;
        sc[r][c] = in ? p.cc[o] : 0.f;
    }
    __syncthreads();
    float w[11];
#pragma unroll
    for (int k = 0; k < 11; ++k) w[k] = c_win[k];
    for (int item = tid; item < LS * (LT / HSEG); item += LTHREADS) {
        const int r = item / (LT / HSEG), c0 = (item % (LT / HSEG)) * HSEG;
        float acc[HSEG][3];
#pragma unroll
        for (int o = 0; o < HSEG; ++o)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc[o][q] = 0.f;
#pragma unroll
        for (int k = 0; k < HSEG + 10; ++k) {
            const float a = sa[r][c0 + k], b = sb[r][c0 + k], cc = sc[r][c0 + k];
#pragma unroll
            for (int o = 0; o < HSEG; ++o) {
                const int t = k - o;
                if (t < 0 || t > 10) continue;
                acc[o][0] = fmaf(w[t], a, acc[o][0]);
                acc[o][1] = fmaf(w[t], b, acc[o][1]);
                acc[o][2] = fmaf(w[t], cc, acc[o][2]);
            }
        }
#pragma unroll
        for (int o = 0; o < HSEG; ++o)
#pragma unroll
            for (int q = 0; q < 3; ++q) hs[q][r][c0 + o] = acc[o][q];
    }
    __syncthreads();
    const float invM = 1.f / (float)((double)p.P * (double)HW);
    const int c = tid % LT, r0 = (tid / LT) * VSEG;
    float f[3][VSEG];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        float col[VSEG + 10];
#pragma unroll
        for (int k = 0; k < VSEG + 10; ++k) col[k] = hs[m][r0 + k][c];
#pragma unroll
        for (int o = 0; o < VSEG; ++o) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 11; ++k) acc = fmaf(w[k], col[o + k], acc);
            f[m][o] = acc;
        }
    }
    const int gx = x0 + c;
#pragma unroll
    for (int o = 0; o < VSEG; ++o) {
        const int gy = y0 + r0 + o;
        if (gy >= p.H || gx >= p.W) continue;
        int64_t oo = pl * HW + (int64_t)gy * p.W + gx;
        float xv = p.x[oo], yv = p.y[oo];
        float diff = xv - yv;
        float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        float dssim = f[0][o] + 2.f * xv * f[1][o] + yv * f[2][o];
        p.d_img[oo] = ((1.f - p.lam) * sgn - p.lam * dssim) * invM;
    }
}

__global__ void __launch_bounds__(1024) loss_final_kernel(LossParams p)
{
    __shared__ double red[2][32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < p.nblocks; i += blockDim.x) {
        a += p.partial[2 * i];
        b += p.partial[2 * i + 1];
    }
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
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            sa += red[0][w];
            sb += red[1][w];
        }
        double M = (double)p.P * p.H * p.W;
        double ssim = sa / M;
        double loss = (1.0 - p.lam) * sb / M + p.lam * (1.0 - ssim);
        *p.d_loss = (float)loss;
        if (p.d_ssim) *p.d_ssim = (float)ssim;
    }
}

static size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace gs3

using namespace gs3;

extern "C" size_t gs_loss_workspace_size(int planes, int H, int W)
{
    if (planes <= 0 || H <= 0 || W <= 0) return 0;
    size_t px = (size_t)planes * H * W;
    size_t nb = (size_t)ceil_div(W, LT) * ceil_div(H, LT) * planes;
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
    p.x = img;
    p.y = target;
    p.P = planes;
    p.H = H;
    p.W = W;
    p.lam = lambda;
    size_t px = (size_t)planes * H * W;
    char *b = reinterpret_cast<char *>(ws);
    p.ca = reinterpret_cast<float *>(b);
    p.cb = reinterpret_cast<float *>(b + a256(4 * px));
    p.cc = reinterpret_cast<float *>(b + 2 * a256(4 * px));
    p.partial = reinterpret_cast<double *>(b + 3 * a256(4 * px));
    p.d_img = d_img;
    p.d_loss = d_loss;
    p.d_ssim = d_ssim;
    dim3 grid((unsigned)ceil_div(W, LT), (unsigned)ceil_div(H, LT), (unsigned)planes);
    p.nblocks = (int)(grid.x * grid.y * grid.z);
    cudaStream_t s = as_stream(stream);
    note_launch();
    ssim_fwd_kernel<<<grid, LTHREADS, 0, s>>>(p);
    note_launch();
    ssim_bwd_kernel<<<grid, LTHREADS, 0, s>>>(p);
    note_launch();
    loss_final_kernel<<<1, 1024, 0, s>>>(p);
    return launch_status("gs_loss_l1_dssim");
}

/*
 * FP64 CPU oracle for the Stage-1 training step of 3DGStream
 * (arXiv 2403.01444).  TEST INFRASTRUCTURE ONLY: only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark load this library.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is computed in double precision, plainly, in the order the
 * paper (and the 3D Gaussian Splatting renderer it builds on) defines it:
 *
 *   hash encoding ........ Section 4.1 (multi-resolution hash encoding, I-NGP)
 *   MLP .................. Section 4.1, Eq. 5; Suppl. A (2 hidden layers, 64, ReLU)
 *   transformation ....... Section 4.1 (mu' = mu + dmu, q' = norm(q) x norm(dq))
 *   projection ........... Section 3.2, Eq. 3 (Sigma' = J W Sigma W^T J^T), Eq. 2
 *   compositing .......... Section 3.2, Eq. 4 (front-to-back alpha blending)
 *   loss ................. Section 4.1, Eq. 6 ((1-l) L1 + l D-SSIM, l = 0.2)
 *   warm-up loss ......... Section 4.1, Eq. 7
 *   Adam ................. Suppl. A (NTC learning rate 0.002)
 *
 * Readings where the paper is silent (3DG-S renderer constants, hash details,
 * pixel-centre convention, SH sign convention) are listed in the design notes
 * and restated beside the code below.  Backward passes are the analytic
 * reverse of each forward, derived by hand.
 *
 * Parity pins: every function is pinned by the CPU tests against closed
 * forms, invariants, library routines or brute force (none is unpinned).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

ORC_API int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ======================================================================
 * Multi-resolution hash encoding (Section 4.1; I-NGP).
 *   resolutions N_l = floor(Nmin * b^l + 1e-6), b = exp((ln Nmax - ln Nmin)/(L-1))
 *   level l is a dense (N_l+1)^3 grid when that fits in T = 2^log2T entries,
 *   otherwise the I-NGP spatial hash (x*1 ^ y*2654435761 ^ z*805459861) mod T.
 * ====================================================================== */
ORC_API int64_t orc_grid_levels(int L, int Nmin, int Nmax, int log2T,
                                int32_t *res, int64_t *offset, int32_t *dense)
{
    double b = (L > 1) ? exp((log((double)Nmax) - log((double)Nmin)) / (double)(L - 1)) : 1.0;
    int64_t T = (int64_t)1 << log2T;
    int64_t off = 0;
    for (int l = 0; l < L; ++l) {
        int n = (int)floor((double)Nmin * pow(b, (double)l) + 1e-6);
        int64_t side = (int64_t)n + 1;
        int64_t full = side * side * side;
        res[l] = n;
        offset[l] = off;
        dense[l] = full <= T ? 1 : 0;
        off += dense[l] ? full : T;
    }
    return off;
}

ORC_API int64_t orc_corner_index(int n, int is_dense, int log2T, int64_t x, int64_t y, int64_t z)
{
    if (is_dense) {
        int64_t s = (int64_t)n + 1;
        return x + y * s + z * s * s;
    }
    uint32_t h = ((uint32_t)x * 1u) ^ ((uint32_t)y * 2654435761u) ^ ((uint32_t)z * 805459861u);
    return (int64_t)(h % (uint32_t)(1u << log2T));
}

/* corners and trilinear weights of point mu at one level */
static void level_corners(const double *mu, const double *aabb, int n, int is_dense, int log2T,
                          int64_t off, int64_t idx[8], double w[8])
{
    int64_t c[3];
    double f[3];
    for (int k = 0; k < 3; ++k) {
        double x = (mu[k] - aabb[k]) / (aabb[3 + k] - aabb[k]);
        if (x < 0.0) x = 0.0;
        if (x > 1.0) x = 1.0;
        double p = x * (double)n;
        double fl = floor(p);
        if (fl > (double)(n - 1)) fl = (double)(n - 1);
        c[k] = (int64_t)fl;
        f[k] = p - fl;
    }
    for (int corner = 0; corner < 8; ++corner) {
        int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
        double wt = (bx ? f[0] : 1.0 - f[0]) * (by ? f[1] : 1.0 - f[1]) * (bz ? f[2] : 1.0 - f[2]);
        idx[corner] = off + orc_corner_index(n, is_dense, log2T, c[0] + bx, c[1] + by, c[2] + bz);
        w[corner] = wt;
    }
}

/* enc[i][l*F + f] = sum over the 8 corners of w * table[idx][f] */
ORC_API void orc_encode(const double *mean, int64_t N, int L, int F, int log2T,
                        const int32_t *res, const int64_t *offset, const int32_t *dense,
                        const double *aabb, const double *table, double *enc)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int l = 0; l < L; ++l) {
            int64_t idx[8];
            double w[8];
            level_corners(mean + 3 * i, aabb, res[l], dense[l], log2T, offset[l], idx, w);
            for (int f = 0; f < F; ++f) {
                double s = 0.0;
                for (int c = 0; c < 8; ++c) s += w[c] * table[idx[c] * F + f];
                enc[i * (int64_t)(L * F) + l * F + f] = s;
            }
        }
    }
}

/* d_table[idx][f] += w * d_enc[i][l*F + f]  (d_table is accumulated into) */
ORC_API void orc_encode_bwd(const double *mean, int64_t N, int L, int F, int log2T,
                            const int32_t *res, const int64_t *offset, const int32_t *dense,
                            const double *aabb, const double *d_enc, double *d_table)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int l = 0; l < L; ++l) {
            int64_t idx[8];
            double w[8];
            level_corners(mean + 3 * i, aabb, res[l], dense[l], log2T, offset[l], idx, w);
            for (int f = 0; f < F; ++f) {
                double g = d_enc[i * (int64_t)(L * F) + l * F + f];
                for (int c = 0; c < 8; ++c) {
#pragma omp atomic
                    d_table[idx[c] * F + f] += w[c] * g;
                }
            }
        }
    }
}

/* ======================================================================
 * MLP (Section 4.1 Eq. 5; Suppl. A): out = W3 relu(W2 relu(W1 h)), no biases.
 * Weights are [out][in] row-major.  h1, h2 hold the post-ReLU activations.
 * ====================================================================== */
ORC_API void orc_mlp_fwd(const double *enc, int64_t N, int din, int dh, int dout,
                         const double *W1, const double *W2, const double *W3,
                         double *h1, double *h2, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        const double *x = enc + i * din;
        double *a1 = h1 + i * dh, *a2 = h2 + i * dh, *y = out + i * dout;
        for (int j = 0; j < dh; ++j) {
            double s = 0.0;
            for (int k = 0; k < din; ++k) s += W1[j * din + k] * x[k];
            a1[j] = s > 0.0 ? s : 0.0;
        }
        for (int j = 0; j < dh; ++j) {
            double s = 0.0;
            for (int k = 0; k < dh; ++k) s += W2[j * dh + k] * a1[k];
            a2[j] = s > 0.0 ? s : 0.0;
        }
        for (int j = 0; j < dout; ++j) {
            double s = 0.0;
            for (int k = 0; k < dh; ++k) s += W3[j * dh + k] * a2[k];
            y[j] = s;
        }
    }
}

/* Reverse of orc_mlp_fwd.  dW1..dW3 are overwritten (sums over all N rows),
 * d_enc[i] is written.  ReLU derivative: 1 where the activation is > 0. */
ORC_API void orc_mlp_bwd(const double *enc, int64_t N, int din, int dh, int dout,
                         const double *W1, const double *W2, const double *W3,
                         const double *h1, const double *h2, const double *d_out,
                         double *dW1, double *dW2, double *dW3, double *d_enc)
{
    memset(dW1, 0, sizeof(double) * dh * din);
    memset(dW2, 0, sizeof(double) * dh * dh);
    memset(dW3, 0, sizeof(double) * dout * dh);
    double *g2 = (double *)malloc(sizeof(double) * dh);
    double *g1 = (double *)malloc(sizeof(double) * dh);
    for (int64_t i = 0; i < N; ++i) {
        const double *x = enc + i * din, *a1 = h1 + i * dh, *a2 = h2 + i * dh, *gy = d_out + i * dout;
        for (int o = 0; o < dout; ++o)
            for (int j = 0; j < dh; ++j) dW3[o * dh + j] += gy[o] * a2[j];
        for (int j = 0; j < dh; ++j) {
            double s = 0.0;
            for (int o = 0; o < dout; ++o) s += W3[o * dh + j] * gy[o];
            g2[j] = a2[j] > 0.0 ? s : 0.0;
        }
        for (int j = 0; j < dh; ++j)
            for (int k = 0; k < dh; ++k) dW2[j * dh + k] += g2[j] * a1[k];
        for (int k = 0; k < dh; ++k) {
            double s = 0.0;
            for (int j = 0; j < dh; ++j) s += W2[j * dh + k] * g2[j];
            g1[k] = a1[k] > 0.0 ? s : 0.0;
        }
        for (int k = 0; k < dh; ++k)
            for (int m = 0; m < din; ++m) dW1[k * din + m] += g1[k] * x[m];
        for (int m = 0; m < din; ++m) {
            double s = 0.0;
            for (int k = 0; k < dh; ++k) s += W1[k * din + m] * g1[k];
            d_enc[i * din + m] = s;
        }
    }
    free(g2);
    free(g1);
}

/* ======================================================================
 * Transformation (Section 4.1): mu' = mu + dmu, q' = norm(q) x norm(dq),
 * Hamilton product, quaternions stored (w, x, y, z).  order = 0 applies the
 * literal product norm(q) x norm(dq); order = 1 the reverse norm(dq) x norm(q).
 * Points outside the hash-grid box keep mu and norm(q) (Suppl. A discards them
 * from the cache).  norm(v) = v / max(|v|, 1e-12).
 * ====================================================================== */
ORC_API void orc_qmul(const double *a, const double *b, double *o)
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

static double qnorm4(const double *q, double *qn)
{
    double len = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double d = len > 1e-12 ? len : 1e-12;
    for (int k = 0; k < 4; ++k) qn[k] = q[k] / d;
    return d;
}

static int inside_box(const double *mu, const double *aabb)
{
    for (int k = 0; k < 3; ++k)
        if (!(mu[k] >= aabb[k] && mu[k] <= aabb[3 + k])) return 0;
    return 1;
}

ORC_API void orc_apply(const double *mean, const double *quat, const double *raw7, int64_t N,
                       const double *aabb, int order, double *mean_out, double *quat_out)
{
    for (int64_t i = 0; i < N; ++i) {
        const double *mu = mean + 3 * i, *r = raw7 + 7 * i;
        double qn[4], dqn[4];
        qnorm4(quat + 4 * i, qn);
        if (!inside_box(mu, aabb)) {
            for (int k = 0; k < 3; ++k) mean_out[3 * i + k] = mu[k];
            for (int k = 0; k < 4; ++k) quat_out[4 * i + k] = qn[k];
            continue;
        }
        qnorm4(r + 3, dqn);
        for (int k = 0; k < 3; ++k) mean_out[3 * i + k] = mu[k] + r[k];
        if (order == 0) orc_qmul(qn, dqn, quat_out + 4 * i);
        else orc_qmul(dqn, qn, quat_out + 4 * i);
    }
}

ORC_API void orc_apply_bwd(const double *mean, const double *quat, const double *raw7, int64_t N,
                           const double *aabb, int order, const double *d_mean_out,
                           const double *d_quat_out, double *d_raw7)
{
    for (int64_t i = 0; i < N; ++i) {
        const double *mu = mean + 3 * i, *r = raw7 + 7 * i, *g = d_quat_out + 4 * i;
        double *o = d_raw7 + 7 * i;
        if (!inside_box(mu, aabb)) {
            for (int k = 0; k < 7; ++k) o[k] = 0.0;
            continue;
        }
        for (int k = 0; k < 3; ++k) o[k] = d_mean_out[3 * i + k];
        double qn[4], dqn[4];
        qnorm4(quat + 4 * i, qn);
        double len = qnorm4(r + 3, dqn);
        /* q' = P dqn with P the 4x4 matrix of left (order 0) or right (order 1)
         * multiplication by qn; dL/ddqn = P^T dL/dq'.  Built column by column
         * from unit basis quaternions so no product formula is retyped. */
        double gd[4] = {0, 0, 0, 0};
        for (int c = 0; c < 4; ++c) {
            double e[4] = {0, 0, 0, 0}, col[4];
            e[c] = 1.0;
            if (order == 0) orc_qmul(qn, e, col);
            else orc_qmul(e, qn, col);
            gd[c] = col[0] * g[0] + col[1] * g[1] + col[2] * g[2] + col[3] * g[3];
        }
        /* normalisation: dqn = dq / len, d/d dq = (I - dqn dqn^T) / len */
        double dot = dqn[0] * gd[0] + dqn[1] * gd[1] + dqn[2] * gd[2] + dqn[3] * gd[3];
        int clamped = !(sqrt(r[3] * r[3] + r[4] * r[4] + r[5] * r[5] + r[6] * r[6]) > 1e-12);
        for (int k = 0; k < 4; ++k) o[3 + k] = clamped ? gd[k] / len : (gd[k] - dqn[k] * dot) / len;
    }
}

/* ======================================================================
 * Spherical harmonics, real basis to degree 3 with the Condon-Shortley sign
 * convention used by the 3DG-S renderer; constants from their closed forms.
 * ====================================================================== */
static void sh_consts(double *c)
{
    const double pi = 3.14159265358979323846;
    c[0] = 0.5 * sqrt(1.0 / pi);            /* l=0 */
    c[1] = 0.5 * sqrt(3.0 / pi);            /* l=1 */
    c[2] = 0.5 * sqrt(15.0 / pi);           /* l=2: xy, yz, xz */
    c[3] = 0.25 * sqrt(5.0 / pi);           /* l=2: 2z^2 - x^2 - y^2 */
    c[4] = 0.25 * sqrt(15.0 / pi);          /* l=2: x^2 - y^2 */
    c[5] = 0.25 * sqrt(35.0 / (2.0 * pi));  /* l=3: y(3x^2-y^2), x(x^2-3y^2) */
    c[6] = 0.5 * sqrt(105.0 / pi);          /* l=3: xyz */
    c[7] = 0.25 * sqrt(21.0 / (2.0 * pi));  /* l=3: y(4z^2-x^2-y^2), x(...) */
    c[8] = 0.25 * sqrt(7.0 / pi);           /* l=3: z(2z^2-3x^2-3y^2) */
    c[9] = 0.25 * sqrt(105.0 / pi);         /* l=3: z(x^2-y^2) */
}

/* Y[k] for k < (deg+1)^2 at direction (x,y,z); gradient wrt (x,y,z) if G != NULL */
ORC_API void orc_sh_basis(int deg, double x, double y, double z, double *Y, double *G)
{
    double c[10];
    sh_consts(c);
    double gl[16][3];
    memset(gl, 0, sizeof(gl));
    Y[0] = c[0];
    if (deg >= 1) {
        Y[1] = -c[1] * y;  gl[1][1] = -c[1];
        Y[2] = c[1] * z;   gl[2][2] = c[1];
        Y[3] = -c[1] * x;  gl[3][0] = -c[1];
    }
    if (deg >= 2) {
        Y[4] = c[2] * x * y;                   gl[4][0] = c[2] * y; gl[4][1] = c[2] * x;
        Y[5] = -c[2] * y * z;                  gl[5][1] = -c[2] * z; gl[5][2] = -c[2] * y;
        Y[6] = c[3] * (2 * z * z - x * x - y * y);
        gl[6][0] = -2 * c[3] * x; gl[6][1] = -2 * c[3] * y; gl[6][2] = 4 * c[3] * z;
        Y[7] = -c[2] * x * z;                  gl[7][0] = -c[2] * z; gl[7][2] = -c[2] * x;
        Y[8] = c[4] * (x * x - y * y);         gl[8][0] = 2 * c[4] * x; gl[8][1] = -2 * c[4] * y;
    }
    if (deg >= 3) {
        Y[9] = -c[5] * y * (3 * x * x - y * y);
        gl[9][0] = -6 * c[5] * x * y; gl[9][1] = -c[5] * (3 * x * x - 3 * y * y);
        Y[10] = c[6] * x * y * z;
        gl[10][0] = c[6] * y * z; gl[10][1] = c[6] * x * z; gl[10][2] = c[6] * x * y;
        Y[11] = -c[7] * y * (4 * z * z - x * x - y * y);
        gl[11][0] = 2 * c[7] * x * y; gl[11][1] = -c[7] * (4 * z * z - x * x - 3 * y * y);
        gl[11][2] = -8 * c[7] * y * z;
        Y[12] = c[8] * z * (2 * z * z - 3 * x * x - 3 * y * y);
        gl[12][0] = -6 * c[8] * x * z; gl[12][1] = -6 * c[8] * y * z;
        gl[12][2] = c[8] * (6 * z * z - 3 * x * x - 3 * y * y);
        Y[13] = -c[7] * x * (4 * z * z - x * x - y * y);
        gl[13][0] = -c[7] * (4 * z * z - 3 * x * x - y * y); gl[13][1] = 2 * c[7] * x * y;
        gl[13][2] = -8 * c[7] * x * z;
        Y[14] = c[9] * z * (x * x - y * y);
        gl[14][0] = 2 * c[9] * x * z; gl[14][1] = -2 * c[9] * y * z; gl[14][2] = c[9] * (x * x - y * y);
        Y[15] = -c[5] * x * (x * x - 3 * y * y);
        gl[15][0] = -c[5] * (3 * x * x - 3 * y * y); gl[15][1] = 6 * c[5] * x * y;
    }
    if (G) {
        int K = (deg + 1) * (deg + 1);
        for (int k = 0; k < K; ++k)
            for (int a = 0; a < 3; ++a) G[3 * k + a] = gl[k][a];
    }
}

/* ======================================================================
 * Projection (Section 3.2, Eq. 2-3).  Camera record (21 doubles):
 *   viewmat[12] (world->camera [R|t], row-major 3x4), fx, fy, cx, cy, W, H, campos[3].
 * Renderer constants of 3DG-S (the paper's code base): near plane 0.2, J
 * evaluated at a mean clamped to 1.3x the half field of view, +0.3 pixel^2
 * on the 2D covariance diagonal, radius ceil(3 sqrt(lambda_max)) with a 0.1
 * floor under the discriminant, SH colour + 0.5 clamped at 0.
 * Pixel (i, j) has its centre at (i + 0.5, j + 0.5); cx = W/2, cy = H/2.
 * Tile rectangle: x in [floor((u-r)/T), floor((u+r+T-1)/T)) clamped to
 * [0, tiles_x], likewise y; an empty rectangle culls.
 * ====================================================================== */
static void tile_rect(double u, double v, int r, int tile, int tx, int ty, int rect[4])
{
    double x0 = floor((u - r) / tile), x1 = floor((u + r + tile - 1) / tile);
    double y0 = floor((v - r) / tile), y1 = floor((v + r + tile - 1) / tile);
    double lo[4] = {x0, y0, x1, y1};
    int hi[4] = {tx, ty, tx, ty};
    for (int k = 0; k < 4; ++k) {
        double a = lo[k];
        if (a < 0) a = 0;
        if (a > hi[k]) a = hi[k];
        rect[k] = (int)a;
    }
}

static double frac_dist(double x) { return fabs(x - floor(x + 0.5)); }

typedef struct {
    int valid;
    double t[3], qn[4], qlen, R[9], M[9], Sig[9];
    double txz, tyz, limx, limy;
    int clx, cly;
    double J[6], Tm[6], a, b, c, det, conic[3], lam;
    int radius;
    double u, v;
    int rect[4];
    double dir[3], dlen, Y[16], rgb_raw[3], rgb[3], opacity, margin;
} pstate;

static void project_one(const double *mu, const double *q, const double *s, double ologit,
                        const double *sh, int deg, const double *cam, int tile, pstate *P)
{
    const double *Wm = cam;
    double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    int W = (int)cam[16], H = (int)cam[17];
    const double *cp = cam + 18;
    int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    memset(P, 0, sizeof(*P));
    P->margin = 1e30;
    for (int r = 0; r < 3; ++r)
        P->t[r] = Wm[4 * r] * mu[0] + Wm[4 * r + 1] * mu[1] + Wm[4 * r + 2] * mu[2] + Wm[4 * r + 3];
    if (!(P->t[2] > 0.2)) return;
    P->margin = fabs(P->t[2] - 0.2);
    P->qlen = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) P->qn[k] = q[k] / P->qlen;
    double w = P->qn[0], x = P->qn[1], y = P->qn[2], z = P->qn[3];
    double *R = P->R;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P->M[3 * i + j] = R[3 * i + j] * s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += P->M[3 * i + k] * P->M[3 * j + k];
            P->Sig[3 * i + j] = acc;
        }
    double tz = P->t[2];
    P->limx = 1.3 * (W / (2.0 * fx));
    P->limy = 1.3 * (H / (2.0 * fy));
    P->txz = P->t[0] / tz;
    P->tyz = P->t[1] / tz;
    double txc = P->txz, tyc = P->tyz;
    if (txc < -P->limx) { txc = -P->limx; P->clx = 1; }
    if (txc > P->limx) { txc = P->limx; P->clx = 1; }
    if (tyc < -P->limy) { tyc = -P->limy; P->cly = 1; }
    if (tyc > P->limy) { tyc = P->limy; P->cly = 1; }
    double *J = P->J;
    J[0] = fx / tz; J[1] = 0;       J[2] = -fx * txc / tz;
    J[3] = 0;       J[4] = fy / tz; J[5] = -fy * tyc / tz;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += J[3 * i + k] * Wm[4 * k + j];
            P->Tm[3 * i + j] = acc;
        }
    double C2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += P->Tm[3 * i + k] * P->Sig[3 * k + l] * P->Tm[3 * j + l];
            C2[2 * i + j] = acc;
        }
    P->a = C2[0] + 0.3;
    P->b = C2[1];
    P->c = C2[3] + 0.3;
    P->det = P->a * P->c - P->b * P->b;
    if (!(P->det > 0)) return;
    P->conic[0] = P->c / P->det;
    P->conic[1] = -P->b / P->det;
    P->conic[2] = P->a / P->det;
    double mid = 0.5 * (P->a + P->c);
    double disc = mid * mid - P->det;
    P->lam = mid + sqrt(disc > 0.1 ? disc : 0.1);
    double r3 = 3.0 * sqrt(P->lam);
    P->radius = (int)ceil(r3);
    P->u = fx * P->t[0] / tz + cx;
    P->v = fy * P->t[1] / tz + cy;
    tile_rect(P->u, P->v, P->radius, tile, tx, ty, P->rect);
    if ((P->rect[2] - P->rect[0]) * (P->rect[3] - P->rect[1]) == 0) return;
    /* margins of the discrete decisions, in their own units */
    double m = frac_dist(r3);
    double mm[4] = {frac_dist((P->u - P->radius) / tile) * tile,
                    frac_dist((P->u + P->radius + tile - 1) / tile) * tile,
                    frac_dist((P->v - P->radius) / tile) * tile,
                    frac_dist((P->v + P->radius + tile - 1) / tile) * tile};
    for (int k = 0; k < 4; ++k) m = mm[k] < m ? mm[k] : m;
    if (P->margin < m) m = P->margin;
    P->margin = m;
    /* colour */
    double d[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
    P->dlen = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) P->dir[k] = d[k] / P->dlen;
    orc_sh_basis(deg, P->dir[0], P->dir[1], P->dir[2], P->Y, NULL);
    int K = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0;
        for (int k = 0; k < K; ++k) acc += P->Y[k] * sh[3 * k + ch];
        P->rgb_raw[ch] = acc + 0.5;
        P->rgb[ch] = P->rgb_raw[ch] > 0 ? P->rgb_raw[ch] : 0.0;
    }
    P->opacity = 1.0 / (1.0 + exp(-ologit));
    P->valid = 1;
}

ORC_API void orc_project(int64_t N, int V, const double *mean, const double *quat,
                         const double *scale, const double *opac_logit, const double *sh,
                         int sh_deg, const double *cams, int tile, double *mean2d, double *conic,
                         double *opacity, double *rgb, double *depth, int32_t *radius,
                         int32_t *rect, double *margin)
{
    int K = (sh_deg + 1) * (sh_deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int v = 0; v < V; ++v) {
            pstate P;
            project_one(mean + 3 * i, quat + 4 * i, scale + 3 * i, opac_logit[i], sh + 3 * K * i,
                        sh_deg, cams + 21 * v, tile, &P);
            int64_t o = (int64_t)v * N + i;
            mean2d[2 * o] = P.u;
            mean2d[2 * o + 1] = P.v;
            for (int k = 0; k < 3; ++k) {
                conic[3 * o + k] = P.conic[k];
                rgb[3 * o + k] = P.rgb[k];
            }
            opacity[o] = P.opacity;
            depth[o] = P.t[2];
            radius[o] = P.valid ? P.radius : 0;
            for (int k = 0; k < 4; ++k) rect[4 * o + k] = P.valid ? P.rect[k] : 0;
            margin[o] = P.margin;
        }
    }
}

/* Reverse of the projection for one (Gaussian, view); g = (du, dv, dA, dB, dC,
 * dr, dg, db).  Adds into dmu[3] and dq[4] (gradient wrt the raw quaternion). */
static void project_one_bwd(const pstate *P, const double *s, const double *sh, int deg,
                            const double *cam, const double *g, double *dmu, double *dq,
                            double *ds, double *dsh)
{
    const double *Wm = cam;
    double fx = cam[12], fy = cam[13];
    int K = (deg + 1) * (deg + 1);
    /* colour: rgb = max(0, sum_k Y_k(dir) sh_k + 0.5), dir = (mu - campos)/|mu - campos| */
    double drr[3];
    for (int ch = 0; ch < 3; ++ch) drr[ch] = P->rgb_raw[ch] > 0 ? g[5 + ch] : 0.0;
    double Y[16], GY[48];
    orc_sh_basis(deg, P->dir[0], P->dir[1], P->dir[2], Y, GY);
    double ddir[3] = {0, 0, 0};
    for (int k = 0; k < K; ++k) {
        double dy = drr[0] * sh[3 * k] + drr[1] * sh[3 * k + 1] + drr[2] * sh[3 * k + 2];
        for (int a = 0; a < 3; ++a) ddir[a] += dy * GY[3 * k + a];
    }
    double dd = P->dir[0] * ddir[0] + P->dir[1] * ddir[1] + P->dir[2] * ddir[2];
    for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - P->dir[a] * dd) / P->dlen;
    /* SH coefficients: d rgb_raw / d sh_k = Y_k (per channel) */
    if (dsh)
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) dsh[3 * k + ch] += Y[k] * drr[ch];

    /* 2D mean: u = fx tx/tz + cx, v = fy ty/tz + cy */
    double tz = P->t[2];
    double dt[3];
    dt[0] = g[0] * fx / tz;
    dt[1] = g[1] * fy / tz;
    dt[2] = -g[0] * fx * P->t[0] / (tz * tz) - g[1] * fy * P->t[1] / (tz * tz);

    /* conic = inverse of [[a, b], [b, c]] */
    double a = P->a, b = P->b, c = P->c, det2 = P->det * P->det;
    double dA = g[2], dB = g[3], dC = g[4];
    double da = (-c * c * dA + b * c * dB - b * b * dC) / det2;
    double db = (2 * b * c * dA - (a * c + b * b) * dB + 2 * a * b * dC) / det2;
    double dc = (-b * b * dA + a * b * dB - a * a * dC) / det2;
    double G[4] = {da, 0.5 * db, 0.5 * db, dc};
    /* cov2 = Tm Sig Tm^T:  dSig = Tm^T G Tm,  dTm = 2 G Tm Sig */
    double dSig[9], dTm[6], GT[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) GT[3 * i + j] = G[2 * i] * P->Tm[j] + G[2 * i + 1] * P->Tm[3 + j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) dSig[3 * i + j] = P->Tm[i] * GT[j] + P->Tm[3 + i] * GT[3 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += GT[3 * i + k] * P->Sig[3 * k + j];
            dTm[3 * i + j] = 2.0 * acc;
        }
    /* Tm = J Wr  ->  dJ = dTm Wr^T */
    double dJ[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += dTm[3 * i + k] * Wm[4 * j + k];
            dJ[3 * i + j] = acc;
        }
    double tz2 = tz * tz, tz3 = tz2 * tz;
    dt[2] += -fx / tz2 * dJ[0] - fy / tz2 * dJ[4];
    if (P->clx) {
        double ls = P->txz < 0 ? -P->limx : P->limx; /* J02 = -fx ls / tz */
        dt[2] += fx * ls / tz2 * dJ[2];
    } else { /* J02 = -fx tx / tz^2 */
        dt[0] += -fx / tz2 * dJ[2];
        dt[2] += 2.0 * fx * P->t[0] / tz3 * dJ[2];
    }
    if (P->cly) {
        double ls = P->tyz < 0 ? -P->limy : P->limy;
        dt[2] += fy * ls / tz2 * dJ[5];
    } else {
        dt[1] += -fy / tz2 * dJ[5];
        dt[2] += 2.0 * fy * P->t[1] / tz3 * dJ[5];
    }
    /* t = Wr mu + tw */
    for (int j = 0; j < 3; ++j) dmu[j] += Wm[j] * dt[0] + Wm[4 + j] * dt[1] + Wm[8 + j] * dt[2];

    /* Sig = M M^T (dSig symmetric) -> dM = 2 dSig M; M = R diag(s) -> dR = dM diag(s) */
    double dR[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += dSig[3 * i + k] * P->M[3 * k + j];
            dR[3 * i + j] = 2.0 * acc * s[j];
            /* M = R diag(s): dL/ds_j = sum_i dM_ij R_ij */
            if (ds) ds[j] += 2.0 * acc * P->R[3 * i + j];
        }
    double w = P->qn[0], x = P->qn[1], y = P->qn[2], z = P->qn[3];
    double dqn[4];
    dqn[0] = 2 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dqn[1] = 2 * (y * dR[1] + z * dR[2] + y * dR[3] - 2 * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2 * x * dR[8]);
    dqn[2] = 2 * (-2 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2 * y * dR[8]);
    dqn[3] = 2 * (-2 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2 * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
    double dot = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
    for (int k = 0; k < 4; ++k) dq[k] += (dqn[k] - P->qn[k] * dot) / P->qlen;
}

ORC_API void orc_project_bwd(int64_t N, int V, const double *mean, const double *quat,
                             const double *scale, const double *opac_logit, const double *sh,
                             int sh_deg, const double *cams, int tile, const double *grads,
                             double *d_mean, double *d_quat)
{
    int K = (sh_deg + 1) * (sh_deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double dmu[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0};
        for (int v = 0; v < V; ++v) {
            pstate P;
            project_one(mean + 3 * i, quat + 4 * i, scale + 3 * i, opac_logit[i], sh + 3 * K * i,
                        sh_deg, cams + 21 * v, tile, &P);
            if (!P.valid) continue;
            project_one_bwd(&P, scale + 3 * i, sh + 3 * K * i, sh_deg, cams + 21 * v,
                            grads + 8 * ((int64_t)v * N + i), dmu, dq, NULL, NULL);
        }
        for (int k = 0; k < 3; ++k) d_mean[3 * i + k] = dmu[k];
        for (int k = 0; k < 4; ++k) d_quat[4 * i + k] = dq[k];
    }
}

/* ======================================================================
 * Tile binning (Section 3.2: the tile-based pipeline of 3DG-S).  Pure integer
 * work on FP32 inputs: every (view, Gaussian, tile in its rectangle) gives a
 * 64-bit key ((view * tiles + tile) << 32 | IEEE bits of the FP32 depth) and
 * value = Gaussian index; pairs are sorted by (key, value); ranges[k] =
 * [first, last+1) of tile-key k (zeros when empty).  Returns the pair count;
 * writes at most `capacity` pairs.
 * ====================================================================== */
/* Reverse of the projection wrt every Gaussian parameter (Stage 2 trains all
 * attributes of the added Gaussians, Section 4.2): from grads[V][N][8] and
 * d_opacity[V][N] (dL/d opacity of each record, NULL = 0), writes d_mean[N][3],
 * d_quat[N][4], d_scale[N][3] (wrt s), d_ologit[N] (opacity = sigmoid(ologit))
 * and d_sh[N][K][3], summed over the views. */
ORC_API void orc_project_bwd_full(int64_t N, int V, const double *mean, const double *quat,
                                  const double *scale, const double *opac_logit, const double *sh,
                                  int sh_deg, const double *cams, int tile, const double *grads,
                                  const double *d_opacity, double *d_mean, double *d_quat,
                                  double *d_scale, double *d_ologit, double *d_sh)
{
    int K = (sh_deg + 1) * (sh_deg + 1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double dmu[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, ds[3] = {0, 0, 0}, dop = 0.0;
        double *dsh = d_sh + 3 * K * i;
        for (int k = 0; k < 3 * K; ++k) dsh[k] = 0.0;
        double o = 1.0 / (1.0 + exp(-opac_logit[i]));
        for (int v = 0; v < V; ++v) {
            pstate P;
            project_one(mean + 3 * i, quat + 4 * i, scale + 3 * i, opac_logit[i], sh + 3 * K * i,
                        sh_deg, cams + 21 * v, tile, &P);
            if (!P.valid) continue;
            project_one_bwd(&P, scale + 3 * i, sh + 3 * K * i, sh_deg, cams + 21 * v,
                            grads + 8 * ((int64_t)v * N + i), dmu, dq, ds, dsh);
            if (d_opacity) dop += d_opacity[(int64_t)v * N + i];
        }
        for (int k = 0; k < 3; ++k) d_mean[3 * i + k] = dmu[k];
        for (int k = 0; k < 4; ++k) d_quat[4 * i + k] = dq[k];
        for (int k = 0; k < 3; ++k) d_scale[3 * i + k] = ds[k];
        d_ologit[i] = dop * o * (1.0 - o);
    }
}

typedef struct { uint64_t key; uint32_t val; } kv_t;
static int cmp_kv(const void *pa, const void *pb)
{
    const kv_t *a = (const kv_t *)pa, *b = (const kv_t *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->val < b->val ? -1 : (a->val > b->val);
}

ORC_API int64_t orc_bin_sort(int V, int64_t N, int W, int H, int tile, const float *mean2d,
                             const int32_t *radius, const float *depth, int64_t capacity,
                             uint64_t *keys, uint32_t *vals, uint32_t *ranges)
{
    int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    int64_t tiles = (int64_t)tx * ty;
    int64_t count = 0;
    for (int v = 0; v < V; ++v)
        for (int64_t i = 0; i < N; ++i) {
            int64_t o = (int64_t)v * N + i;
            if (radius[o] <= 0) continue;
            int r[4];
            tile_rect((double)mean2d[2 * o], (double)mean2d[2 * o + 1], radius[o], tile, tx, ty, r);
            count += (int64_t)(r[2] - r[0]) * (r[3] - r[1]);
        }
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (count > 0 ? count : 1));
    int64_t n = 0;
    for (int v = 0; v < V; ++v)
        for (int64_t i = 0; i < N; ++i) {
            int64_t o = (int64_t)v * N + i;
            if (radius[o] <= 0) continue;
            int r[4];
            tile_rect((double)mean2d[2 * o], (double)mean2d[2 * o + 1], radius[o], tile, tx, ty, r);
            uint32_t dbits;
            memcpy(&dbits, depth + o, 4);
            for (int y = r[1]; y < r[3]; ++y)
                for (int x = r[0]; x < r[2]; ++x) {
                    uint64_t tk = (uint64_t)v * tiles + (uint64_t)y * tx + x;
                    kv[n].key = (tk << 32) | dbits;
                    kv[n].val = (uint32_t)i;
                    ++n;
                }
        }
    qsort(kv, (size_t)n, sizeof(kv_t), cmp_kv);
    memset(ranges, 0, sizeof(uint32_t) * 2 * V * tiles);
    if (count <= capacity) {
        for (int64_t k = 0; k < n; ++k) {
            keys[k] = kv[k].key;
            vals[k] = kv[k].val;
            uint64_t tk = kv[k].key >> 32;
            if (k == 0 || (kv[k - 1].key >> 32) != tk) ranges[2 * tk] = (uint32_t)k;
            if (k == n - 1 || (kv[k + 1].key >> 32) != tk) ranges[2 * tk + 1] = (uint32_t)(k + 1);
        }
    }
    free(kv);
    return count;
}

/* ======================================================================
 * Compositing (Section 3.2, Eq. 4), per pixel, over the Gaussians whose tile
 * rectangle holds the pixel's tile, in ascending (depth, index) order:
 *   d = pixel centre - mu2d; power = -0.5 (A dx^2 + C dy^2) - B dx dy
 *   skip if power > 0; alpha = min(0.99, o exp(power)); skip if alpha < 1/255
 *   stop (without adding) when T (1 - alpha) < 1e-4; else C += c alpha T, T *= 1 - alpha
 *   output C + T bg; T_final = T; last = 1 + list position of the last added.
 * ambig[p] = 1 when a decision of pixel p may fall the other way in a
 * computation that differs from this one by rounding or by a small
 * perturbation of its inputs:
 *  - a threshold (power > 0, alpha against 1/255 and 0.99, T (1 - alpha)
 *    against 1e-4) lies within its relative rounding margin, widened by the
 *    reach of the perturbation: a displacement of up to pos_eps[v][g] pixels
 *    of the 2D mean (|grad power| pos_eps) and a change of the conic of up to
 *    rel_eps[v][g] relative to its smallest eigenvalue (|power| rel_eps); NULL
 *    arrays mean 0, for exact-input comparisons;
 *  - two consecutive added Gaussians lie within `tie` (relative) plus their
 *    depth reaches depth_eps[v][g] (absolute; NULL means 0) in depth, so that
 *    their order may differ.  Swapping two adjacent added Gaussians i, j
 *    changes the pixel by exactly T_i alpha_i alpha_j (c_i - c_j) (T_i the
 *    transmittance before both; the product of (1 - alpha) is unchanged), so
 *    such pairs add that amount to a per-pixel bound and only flag the pixel
 *    when the bound exceeds tie_budget; a run of three or more tied Gaussians,
 *    or a tie with the Gaussian that ends the pixel, always flags it.
 * win (optional, tiles x0 y0 x1 y1): only pixels of those tiles are
 * composited (a crop of the same definition); other outputs are untouched.
 * ====================================================================== */
typedef struct { double depth; int64_t g; } item_t;
static int cmp_item(const void *pa, const void *pb)
{
    const item_t *a = (const item_t *)pa, *b = (const item_t *)pb;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    return a->g < b->g ? -1 : (a->g > b->g);
}

/* win: optional tile window (tx0, ty0, tx1, ty1); lists of other tiles stay empty */
static int in_win(const int32_t *win, int x, int y)
{
    return !win || (x >= win[0] && x < win[2] && y >= win[1] && y < win[3]);
}

static void build_lists(int V, int64_t N, int W, int H, int tile, const double *mean2d,
                        const int32_t *radius, const double *depth, const int32_t *win,
                        int64_t **off_out, item_t **items_out)
{
    int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    int64_t tiles = (int64_t)tx * ty, nt = tiles * V;
    int64_t *cnt = (int64_t *)calloc((size_t)nt + 1, sizeof(int64_t));
    for (int v = 0; v < V; ++v)
        for (int64_t i = 0; i < N; ++i) {
            int64_t o = (int64_t)v * N + i;
            if (radius[o] <= 0) continue;
            int r[4];
            tile_rect(mean2d[2 * o], mean2d[2 * o + 1], radius[o], tile, tx, ty, r);
            for (int y = r[1]; y < r[3]; ++y)
                for (int x = r[0]; x < r[2]; ++x)
                    if (in_win(win, x, y)) cnt[v * tiles + (int64_t)y * tx + x + 1]++;
        }
    for (int64_t k = 0; k < nt; ++k) cnt[k + 1] += cnt[k];
    item_t *items = (item_t *)malloc(sizeof(item_t) * (cnt[nt] > 0 ? cnt[nt] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nt > 0 ? nt : 1));
    memcpy(fill, cnt, sizeof(int64_t) * nt);
    for (int v = 0; v < V; ++v)
        for (int64_t i = 0; i < N; ++i) {
            int64_t o = (int64_t)v * N + i;
            if (radius[o] <= 0) continue;
            int r[4];
            tile_rect(mean2d[2 * o], mean2d[2 * o + 1], radius[o], tile, tx, ty, r);
            for (int y = r[1]; y < r[3]; ++y)
                for (int x = r[0]; x < r[2]; ++x) {
                    if (!in_win(win, x, y)) continue;
                    int64_t k = v * tiles + (int64_t)y * tx + x;
                    items[fill[k]].depth = depth[o];
                    items[fill[k]].g = i;
                    fill[k]++;
                }
        }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nt; ++k)
        qsort(items + cnt[k], (size_t)(cnt[k + 1] - cnt[k]), sizeof(item_t), cmp_item);
    free(fill);
    *off_out = cnt;
    *items_out = items;
}

#define A_MIN (1.0 / 255.0)
#define A_CAP 0.99
#define T_EPS 1e-4
#define RM_ALPHA 2e-5
#define RM_T 1e-3
#define M_POWER 1e-5

ORC_API void orc_raster_fwd(int V, int64_t N, int W, int H, int tile, const double *mean2d,
                            const double *conic, const double *opacity, const double *rgb,
                            const double *depth, const int32_t *radius, const double *bg,
                            const int32_t *win, double tie, double tie_budget,
                            const double *depth_eps, const double *pos_eps,
                            const double *rel_eps, double *img, double *T_final, int32_t *last,
                            int32_t *ambig)
{
    int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    int64_t tiles = (int64_t)tx * ty;
    int64_t *off;
    item_t *items;
    build_lists(V, N, W, H, tile, mean2d, radius, depth, win, &off, &items);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < V * tiles; ++k) {
        int v = (int)(k / tiles);
        int64_t t = k % tiles;
        int bx = (int)(t % tx), by = (int)(t / tx);
        if (!in_win(win, bx, by)) continue;
        for (int py = by * tile; py < (by + 1) * tile && py < H; ++py)
            for (int px = bx * tile; px < (bx + 1) * tile && px < W; ++px) {
                double T = 1.0, C[3] = {0, 0, 0};
                double prev_depth = -1.0, prev_T = 0.0, prev_alpha = 0.0, tie_err = 0.0, t_reach = 0.0;
                int64_t prev_o = -1;
                const double *prev_c = NULL;
                int lst = 0, amb = 0, run = 0;
                for (int64_t j = off[k]; j < off[k + 1]; ++j) {
                    int64_t o = (int64_t)v * N + items[j].g;
                    double dx = px + 0.5 - mean2d[2 * o], dy = py + 0.5 - mean2d[2 * o + 1];
                    const double *cn = conic + 3 * o;
                    double power = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
                    /* reach of power under the input perturbation */
                    double gx = cn[0] * dx + cn[1] * dy, gy = cn[1] * dx + cn[2] * dy;
                    double reach = (pos_eps ? sqrt(gx * gx + gy * gy) * pos_eps[o] : 0.0) +
                                   (rel_eps ? fabs(power) * rel_eps[o] : 0.0);
                    if (fabs(power) < M_POWER + reach) amb = 1;
                    if (power > 0) continue;
                    double araw = opacity[o] * exp(power);
                    if (fabs(log(araw / A_MIN)) <= RM_ALPHA + reach) amb = 1;
                    if (fabs(log(araw / A_CAP)) <= RM_ALPHA + reach) amb = 1;
                    double alpha = araw < A_CAP ? araw : A_CAP;
                    if (alpha < A_MIN) continue;
                    double tt = T * (1.0 - alpha);
                    /* relative reach of T (1 - alpha): every uncapped alpha so far may move */
                    if (araw < A_CAP) t_reach += alpha * reach / (1.0 - alpha);
                    if (fabs(log(tt / T_EPS)) <= RM_T + t_reach) amb = 1;
                    double gap = tie * depth[o] + (depth_eps && prev_o >= 0 ? depth_eps[o] + depth_eps[prev_o] : 0.0);
                    if (prev_depth > 0 && fabs(depth[o] - prev_depth) <= gap) {
                        if (tt < T_EPS || run > 0) {
                            amb = 1;
                        } else {
                            double dc = 0.0;
                            for (int ch = 0; ch < 3; ++ch) {
                                double d = fabs(prev_c[ch] - rgb[3 * o + ch]);
                                if (d > dc) dc = d;
                            }
                            tie_err += prev_T * prev_alpha * alpha * dc;
                        }
                        run = 1;
                    } else {
                        run = 0;
                    }
                    if (tt < T_EPS) break;
                    for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * o + ch] * alpha * T;
                    prev_T = T;
                    prev_alpha = alpha;
                    prev_c = rgb + 3 * o;
                    prev_depth = depth[o];
                    prev_o = o;
                    T = tt;
                    lst = (int)(j - off[k]) + 1;
                }
                if (tie_err > tie_budget) amb = 1;
                int64_t p = ((int64_t)v * H + py) * W + px;
                for (int ch = 0; ch < 3; ++ch)
                    img[(((int64_t)v * 3 + ch) * H + py) * W + px] = C[ch] + T * bg[ch];
                T_final[p] = T;
                last[p] = lst;
                ambig[p] = amb;
            }
    }
    free(off);
    free(items);
}

/* Reverse of the compositing: walks each pixel's list back to front from its
 * last added Gaussian, recovering T_i = T_{i+1} / (1 - alpha_i) from T_final.
 * grads[v][g] (8 doubles: du, dv, dA, dB, dC, dr, dg, db) are accumulated;
 * d_opacity[v][g] too when non-NULL.  The alpha cap and the skips take their
 * piecewise derivative (zero where capped or skipped). */
ORC_API void orc_raster_bwd(int V, int64_t N, int W, int H, int tile, const double *mean2d,
                            const double *conic, const double *opacity, const double *rgb,
                            const double *depth, const int32_t *radius, const double *bg,
                            const int32_t *win, const double *T_final, const int32_t *last,
                            const double *d_img, double *grads, double *d_opacity)
{
    int tx = (W + tile - 1) / tile, ty = (H + tile - 1) / tile;
    int64_t tiles = (int64_t)tx * ty;
    int64_t *off;
    item_t *items;
    build_lists(V, N, W, H, tile, mean2d, radius, depth, win, &off, &items);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < V * tiles; ++k) {
        int v = (int)(k / tiles);
        int64_t t = k % tiles;
        int bx = (int)(t % tx), by = (int)(t / tx);
        if (!in_win(win, bx, by)) continue;
        for (int py = by * tile; py < (by + 1) * tile && py < H; ++py)
            for (int px = bx * tile; px < (bx + 1) * tile && px < W; ++px) {
                int64_t p = ((int64_t)v * H + py) * W + px;
                double dC[3], Bk[3];
                for (int ch = 0; ch < 3; ++ch) {
                    dC[ch] = d_img[(((int64_t)v * 3 + ch) * H + py) * W + px];
                    Bk[ch] = bg[ch];
                }
                double T = T_final[p];
                for (int64_t j = off[k] + last[p] - 1; j >= off[k]; --j) {
                    int64_t o = (int64_t)v * N + items[j].g;
                    double dx = px + 0.5 - mean2d[2 * o], dy = py + 0.5 - mean2d[2 * o + 1];
                    const double *cn = conic + 3 * o;
                    double power = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
                    if (power > 0) continue;
                    double G = exp(power);
                    double araw = opacity[o] * G;
                    int capped = !(araw < A_CAP);
                    double alpha = capped ? A_CAP : araw;
                    if (alpha < A_MIN) continue;
                    T = T / (1.0 - alpha);
                    const double *c = rgb + 3 * o;
                    double dalpha = 0;
                    double *gr = grads + 8 * o;
                    for (int ch = 0; ch < 3; ++ch) {
                        dalpha += dC[ch] * T * (c[ch] - Bk[ch]);
#pragma omp atomic
                        gr[5 + ch] += dC[ch] * alpha * T;
                        Bk[ch] = alpha * c[ch] + (1.0 - alpha) * Bk[ch];
                    }
                    if (capped) continue;
                    double dpow = dalpha * alpha;
                    double du = dpow * (cn[0] * dx + cn[1] * dy);
                    double dv = dpow * (cn[2] * dy + cn[1] * dx);
#pragma omp atomic
                    gr[0] += du;
#pragma omp atomic
                    gr[1] += dv;
#pragma omp atomic
                    gr[2] += dpow * (-0.5 * dx * dx);
#pragma omp atomic
                    gr[3] += dpow * (-dx * dy);
#pragma omp atomic
                    gr[4] += dpow * (-0.5 * dy * dy);
                    if (d_opacity) {
#pragma omp atomic
                        d_opacity[o] += dalpha * G;
                    }
                }
            }
    }
    free(off);
    free(items);
}

/* ======================================================================
 * Loss (Section 4.1, Eq. 6): L = (1 - lam) mean|I - I*| + lam (1 - SSIM),
 * SSIM with an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2,
 * zero padding, mean over views, channels and pixels (3DG-S's loss).
 * Images are planar [P][H][W] (P = views x 3).  Returns L, writes dL/dI.
 * The subgradient of |x| at 0 is 0.
 * ====================================================================== */
ORC_API void orc_ssim_window(double *g11)
{
    double s = 0;
    for (int i = 0; i < 11; ++i) {
        g11[i] = exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
        s += g11[i];
    }
    for (int i = 0; i < 11; ++i) g11[i] /= s;
}

ORC_API double orc_loss_l1_dssim(const double *img, const double *tgt, int P, int H, int W,
                                 double lam, double *d_img, double *ssim_out)
{
    double g[11];
    orc_ssim_window(g);
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    int64_t HW = (int64_t)H * W, M = (int64_t)P * HW;
    double *ca = (double *)malloc(sizeof(double) * M);
    double *cb = (double *)malloc(sizeof(double) * M);
    double *cc = (double *)malloc(sizeof(double) * M);
    double l1 = 0, ss = 0;
#pragma omp parallel for schedule(static) reduction(+ : l1, ss)
    for (int64_t pr = 0; pr < (int64_t)P * H; ++pr) {
        int64_t pl = pr / H;
        int y = (int)(pr % H);
        const double *X = img + pl * HW, *Yt = tgt + pl * HW;
        for (int x = 0; x < W; ++x) {
            double mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
            for (int a = -5; a <= 5; ++a)
                for (int b = -5; b <= 5; ++b) {
                    int yy = y + a, xx = x + b;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    double w = g[a + 5] * g[b + 5];
                    double xv = X[(int64_t)yy * W + xx], yv = Yt[(int64_t)yy * W + xx];
                    mx += w * xv; my += w * yv;
                    exx += w * xv * xv; eyy += w * yv * yv; exy += w * xv * yv;
                }
            double sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
            double n1 = 2 * mx * my + C1, n2 = 2 * sxy + C2;
            double d1 = mx * mx + my * my + C1, d2 = sxx + syy + C2;
            double s = n1 * n2 / (d1 * d2);
            ss += s;
            /* partial derivatives wrt (mx, sxx, sxy), then wrt (mx, exx, exy) */
            double ds_dmx = 2 * my * n2 / (d1 * d2) - s * 2 * mx / d1;
            double ds_dsxx = -s / d2;
            double ds_dsxy = 2 * n1 / (d1 * d2);
            int64_t q = pl * HW + (int64_t)y * W + x;
            ca[q] = ds_dmx - 2 * mx * ds_dsxx - my * ds_dsxy;
            cb[q] = ds_dsxx;
            cc[q] = ds_dsxy;
            l1 += fabs(X[(int64_t)y * W + x] - Yt[(int64_t)y * W + x]);
        }
    }
    double ssim = ss / (double)M;
    if (ssim_out) *ssim_out = ssim;
    double L = (1.0 - lam) * l1 / (double)M + lam * (1.0 - ssim);
    if (d_img) {
#pragma omp parallel for schedule(static)
        for (int64_t pr = 0; pr < (int64_t)P * H; ++pr) {
            int64_t pl = pr / H;
            int y = (int)(pr % H);
            const double *X = img + pl * HW, *Yt = tgt + pl * HW;
            for (int x = 0; x < W; ++x) {
                double sa = 0, sb = 0, sc = 0;
                for (int a = -5; a <= 5; ++a)
                    for (int b = -5; b <= 5; ++b) {
                        int yy = y + a, xx = x + b; /* window centres p whose window holds q */
                        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                        double w = g[a + 5] * g[b + 5];
                        int64_t pp = pl * HW + (int64_t)yy * W + xx;
                        sa += w * ca[pp]; sb += w * cb[pp]; sc += w * cc[pp];
                    }
                double xv = X[(int64_t)y * W + x], yv = Yt[(int64_t)y * W + x];
                double dssim = (sa + 2 * xv * sb + yv * sc) / (double)M;
                double diff = xv - yv;
                double sgn = diff > 0 ? 1.0 : (diff < 0 ? -1.0 : 0.0);
                d_img[pl * HW + (int64_t)y * W + x] = (1.0 - lam) * sgn / (double)M - lam * dssim;
            }
        }
    }
    free(ca); free(cb); free(cc);
    return L;
}

/* ======================================================================
 * Warm-up loss (Section 4.1, Eq. 7): mean over points of
 *   |dmu|_1 - cos^2(norm(dq), Q),  Q = (1, 0, 0, 0)  ->  cos = dq_w / |dq|.
 * ====================================================================== */
ORC_API double orc_warmup_loss(const double *raw7, int64_t N, double *d_raw7)
{
    double L = 0;
    for (int64_t i = 0; i < N; ++i) {
        const double *r = raw7 + 7 * i;
        double n2 = r[3] * r[3] + r[4] * r[4] + r[5] * r[5] + r[6] * r[6];
        L += fabs(r[0]) + fabs(r[1]) + fabs(r[2]) - r[3] * r[3] / n2;
        if (d_raw7) {
            double *o = d_raw7 + 7 * i;
            for (int k = 0; k < 3; ++k) o[k] = (r[k] > 0 ? 1.0 : (r[k] < 0 ? -1.0 : 0.0)) / (double)N;
            /* d/dq of -w^2/|q|^2 = -(2 w e_w)/|q|^2 + 2 w^2 q / |q|^4 */
            for (int k = 0; k < 4; ++k) {
                double v = 2.0 * r[3] * r[3] * r[3 + k] / (n2 * n2);
                if (k == 0) v -= 2.0 * r[3] / n2;
                o[3 + k] = v / (double)N;
            }
        }
    }
    return L / (double)N;
}

/* ======================================================================
 * Adam (Suppl. A: NTC learning rate 0.002; beta1 0.9, beta2 0.99, eps 1e-15
 * as in I-NGP), bias-corrected, on the gradient g * inv_scale.
 * step is the 1-based step number of this update.
 * ====================================================================== */
ORC_API void orc_adam(double *p, const double *g, double *m, double *v, int64_t n, double lr,
                      double b1, double b2, double eps, int step, double inv_scale)
{
    double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
    for (int64_t i = 0; i < n; ++i) {
        double gi = g[i] * inv_scale;
        m[i] = b1 * m[i] + (1.0 - b1) * gi;
        v[i] = b2 * v[i] + (1.0 - b2) * gi * gi;
        double mh = m[i] / bc1, vh = v[i] / bc2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

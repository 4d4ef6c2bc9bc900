/*
 * Plain CPU oracle for rasterised Steered Mixture of Experts (R-SMoE) image
 * regression.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg may call it; the product path never does.
 * It shares no code, header or constant table with the CUDA library.
 *
 * What it computes (paper: "Rasterized Steered Mixture of Experts for
 * Efficient 2D Image Regression", arXiv 2510.05814):
 *   K_k(x) = exp(-1/2 (x-mu_k)^T P_k (x-mu_k)),  P_k = L_k L_k^T       (Eq. 2)
 *   w_k(x) = pi_k K_k(x) / sum_i pi_i K_i(x)      (Eq. 4; pi_k = exp(logpi_k),
 *                                                  pi = 1 when logpi is NULL)
 *   y(x)   = sum_k m_k(x) w_k(x)             (Eq. 3, restricted as in Eq. 5)
 * or, in the RBF mode (rbf = 1, the Gaussian-splatting regression of Eq. 1),
 *   y(x)   = sum_k m_k(x) pi_k K_k(x)        (no normalisation: D = 1)
 * with the kernel support truncated (Sec. IV): a pair (pixel, kernel) takes
 * part only if its Mahalanobis distance q is <= q_max.  Every pixel is
 * evaluated against EVERY kernel (no binning): the truncated model is defined
 * pointwise, so binning cannot change it.
 *
 * Precision: all values (q, exp, sums, gradients, Adam) are FP64.  Two things
 * are FP32 on purpose because they decide integers and must agree bit for bit
 * with any FP32 implementation of the same definition:
 *   - the inclusion predicate q32 <= q_max (om_included), and
 *   - the per-kernel bounding box / tile rectangle (om_rect, Sec. IV-B).
 * Both are written as explicit single-rounding float operations; the file is
 * compiled with -ffp-contract=off so the compiler cannot fuse them.
 *
 * Conventions: pixel (i, j) is column i, row j, with centre (i+0.5, j+0.5);
 * images are channel-planar C x H x W; parameters are structure-of-arrays:
 * mu[K][2] in normalised [0,1] units (pixel centre = mu * (W, H)),
 * chol[K][3] = (a, b, c) with L = [[a, 0], [b, c]] in pixel units,
 * ea[K][C] expert offsets, eW[K][C][2] linear expert slopes (pixel units),
 * m_k(x) = ea_k + eW_k (x - mu_k).  A render at scale s uses
 * L' = L / s and eW' = eW / s (Sec. II-B and VII-C: resampling the continuous
 * regression function on another raster).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t W, H, C, T, linear;
    float qmax, scale;
    int64_t K;
    const float *mu, *chol, *ea, *eW;
    int32_t rbf;            /* 0: softmax gates (Eq. 4); 1: RBF sum (Eq. 1) */
    const float *logpi;     /* K gate weights log pi_k (Eq. 4), or NULL: pi = 1 */
} om_model;

/* ------------------------------------------------------------------------ */
/* FP32 pieces: the kernel in output-pixel units, the predicate, the box.    */
/* ------------------------------------------------------------------------ */

/* Kernel k in output-pixel units, rounded to float once per operation:
 * mu_px = mu_n * (W, H);  (a, b, c) / s when s != 1.  (Sec. II-B resampling.) */
static void kernel_px(const om_model *m, int64_t k, float *mx, float *my,
                      float *a, float *b, float *c)
{
    float w = (float)m->W, h = (float)m->H;
    *mx = m->mu[2 * k] * w;
    *my = m->mu[2 * k + 1] * h;
    *a = m->chol[3 * k];
    *b = m->chol[3 * k + 1];
    *c = m->chol[3 * k + 2];
    if (m->scale != 1.0f) {
        *a = *a / m->scale;
        *b = *b / m->scale;
        *c = *c / m->scale;
    }
}

/* Truncation predicate (Sec. IV, 99% / q_max ellipse), FP32, one rounding per
 * step:  dx = x0-mx, dy = y0-my, t = b*dy, z0 = fma(a,dx,t), z1 = c*dy,
 * q32 = fma(z0, z0, z1*z1);  included <=> q32 <= q_max. */
static int included_at(const om_model *m, int64_t k, float x0, float y0)
{
    float mx, my, a, b, c;
    kernel_px(m, k, &mx, &my, &a, &b, &c);
    float dx = x0 - mx;
    float dy = y0 - my;
    float t = b * dy;
    float z0 = fmaf(a, dx, t);
    float z1 = c * dy;
    float u = z1 * z1;
    float q32 = fmaf(z0, z0, u);
    return q32 <= m->qmax;
}

/* The predicate at the centre (i + 0.5, j + 0.5) of pixel (i, j). */
int om_included(const om_model *m, int64_t k, int32_t i, int32_t j)
{
    return included_at(m, k, (float)i + 0.5f, (float)j + 0.5f);
}

/* Bounding box of kernel k as an inclusive tile rectangle (Sec. IV-B, the
 * "geometry shader"; Fig. 3b: a square centred on mu whose side is the major
 * axis of the q_max ellipse).  Half side r = sqrt(q_max * lambda_max(Sigma))
 * * (1 + 2^-10), lambda_max(Sigma) = 1 / lambda_min(P) = lambda_max(P)/det(P).
 * rect = {tx0, ty0, tx1, ty1}; an empty box has tx0 > tx1 (rect {0,0,-1,-1}).
 * Returns the number of tiles. */
int64_t om_rect(const om_model *m, int64_t k, int32_t rect[4])
{
    float mx, my, a, b, c;
    kernel_px(m, k, &mx, &my, &a, &b, &c);
    int32_t tiles_x = (m->W + m->T - 1) / m->T;
    int32_t tiles_y = (m->H + m->T - 1) / m->T;
    rect[0] = 0; rect[1] = 0; rect[2] = -1; rect[3] = -1;
    if (!isfinite(mx) || !isfinite(my) || !isfinite(a) || !isfinite(b) ||
        !isfinite(c))
        return 0;                       /* no pixel can pass the predicate */
    float p00 = a * a;
    float p01 = a * b;
    float cc = c * c;
    float p11 = fmaf(b, b, cc);
    float h = 0.5f * (p00 - p11);
    float p01sq = p01 * p01;
    float rt = sqrtf(fmaf(h, h, p01sq));
    float half_tr = 0.5f * (p00 + p11);
    float lmax_p = half_tr + rt;
    float ac = a * c;
    float det = ac * ac;
    int whole = 0;
    float lo_x = 0, hi_x = 0, lo_y = 0, hi_y = 0;
    if (det == 0.0f) {
        whole = 1;
    } else {
        float lmax_s = lmax_p / det;
        float r = sqrtf(m->qmax * lmax_s);
        r = r * (1.0f + 0x1p-10f);
        float T = (float)m->T;
        lo_x = (mx - r) / T;
        hi_x = (mx + r) / T;
        lo_y = (my - r) / T;
        hi_y = (my + r) / T;
        if (!isfinite(r) || !isfinite(lo_x) || !isfinite(hi_x) ||
            !isfinite(lo_y) || !isfinite(hi_y))
            whole = 1;
    }
    if (whole) {
        rect[0] = 0; rect[1] = 0; rect[2] = tiles_x - 1; rect[3] = tiles_y - 1;
        return (int64_t)tiles_x * tiles_y;
    }
    float fx0 = fmaxf(floorf(lo_x), 0.0f);
    float fy0 = fmaxf(floorf(lo_y), 0.0f);
    float fx1 = fminf(floorf(hi_x), (float)(tiles_x - 1));
    float fy1 = fminf(floorf(hi_y), (float)(tiles_y - 1));
    if (fx0 > fx1 || fy0 > fy1)
        return 0;
    rect[0] = (int32_t)fx0; rect[1] = (int32_t)fy0;
    rect[2] = (int32_t)fx1; rect[3] = (int32_t)fy1;
    return (int64_t)(rect[2] - rect[0] + 1) * (rect[3] - rect[1] + 1);
}

/* Subset kernel selection per block (Sec. IV-C, Eq. 5): K_n = {k : tile n
 * lies in rect_k}, listed in ascending k, tiles in row-major order.  Built by
 * the plain double loop over tiles x kernels.  If tiles != NULL only the
 * n_sel listed tiles are built (their lists are concatenated in that order
 * and tile_off has n_sel+1 entries).  Writes at most cap kernel ids and
 * returns the total number of pairs. */
int64_t om_bin(const om_model *m, int64_t n_sel, const int64_t *tiles,
               int64_t *tile_off, int32_t *pair_k, int64_t cap)
{
    int32_t tiles_x = (m->W + m->T - 1) / m->T;
    int32_t tiles_y = (m->H + m->T - 1) / m->T;
    int64_t n_tiles = (int64_t)tiles_x * tiles_y;
    if (!tiles) n_sel = n_tiles;
    int32_t *rects = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(m->K + 1));
    for (int64_t k = 0; k < m->K; ++k)
        om_rect(m, k, rects + 4 * k);
    int64_t p = 0;
    for (int64_t s = 0; s < n_sel; ++s) {
        int64_t t = tiles ? tiles[s] : s;
        int32_t tx = (int32_t)(t % tiles_x), ty = (int32_t)(t / tiles_x);
        tile_off[s] = p;
        for (int64_t k = 0; k < m->K; ++k) {
            const int32_t *r = rects + 4 * k;
            if (tx >= r[0] && tx <= r[2] && ty >= r[1] && ty <= r[3]) {
                if (p < cap) pair_k[p] = (int32_t)k;
                ++p;
            }
        }
    }
    tile_off[n_sel] = p;
    free(rects);
    return p;
}

/* ------------------------------------------------------------------------ */
/* FP64 values.                                                              */
/* ------------------------------------------------------------------------ */

/* Gate numerator and expert of kernel k at pixel (i, j), FP64, for an
 * included pair.  dx, dy use the FP32 kernel centre (the model's centre is
 * defined as the float product mu_n * W); the rest is exact FP64. */
typedef struct { double dx, dy, z0, z1, e; double mexp[3], mabs[3]; } om_pair;

static void pair_value_at(const om_model *m, int64_t k, double x, double y,
                          om_pair *pr)
{
    float mx, my, a, b, c;
    kernel_px(m, k, &mx, &my, &a, &b, &c);
    double dx = x - (double)mx;
    double dy = y - (double)my;
    double z0 = (double)a * dx + (double)b * dy;
    double z1 = (double)c * dy;
    double q = z0 * z0 + z1 * z1;
    pr->dx = dx; pr->dy = dy; pr->z0 = z0; pr->z1 = z1;
    double lp = m->logpi ? (double)m->logpi[k] : 0.0;
    pr->e = exp(lp - 0.5 * q);                     /* pi_k K_k(x), Eqs. 2 and 4 */
    for (int ch = 0; ch < m->C; ++ch) {
        double v = (double)m->ea[k * m->C + ch];
        if (m->linear) {
            double w0 = (double)m->eW[(k * m->C + ch) * 2];
            double w1 = (double)m->eW[(k * m->C + ch) * 2 + 1];
            if (m->scale != 1.0f) {
                /* eW' = eW / s, rounded to float like L' */
                w0 = (double)(m->eW[(k * m->C + ch) * 2] / m->scale);
                w1 = (double)(m->eW[(k * m->C + ch) * 2 + 1] / m->scale);
            }
            v += w0 * dx + w1 * dy;
            pr->mabs[ch] = fabs((double)m->ea[k * m->C + ch]) + fabs(w0 * dx) + fabs(w1 * dy);
        } else {
            pr->mabs[ch] = fabs(v);
        }
        pr->mexp[ch] = v;
    }
}

static void pair_value(const om_model *m, int64_t k, int32_t i, int32_t j,
                       om_pair *pr)
{
    pair_value_at(m, k, (double)i + 0.5, (double)j + 0.5, pr);
}

/* Gate denominator D and numerators N_c at the sample point (x, y) (FP32
 * pixel units) over all K kernels; A_c (if non-NULL) receives
 * sum_k e_k (|a_kc| + |W_kc0 dx| + |W_kc1 dy|), the size of the terms that
 * make up the gated sum (the scale of its rounding error). */
static void point_sums(const om_model *m, float x, float y, double *D,
                       double *N, double *A)
{
    double d = 0.0;
    for (int ch = 0; ch < m->C; ++ch) { N[ch] = 0.0; if (A) A[ch] = 0.0; }
    for (int64_t k = 0; k < m->K; ++k) {
        if (!included_at(m, k, x, y)) continue;
        om_pair pr;
        pair_value_at(m, k, (double)x, (double)y, &pr);
        d += pr.e;
        for (int ch = 0; ch < m->C; ++ch) {
            N[ch] += pr.e * pr.mexp[ch];
            if (A) A[ch] += pr.e * pr.mabs[ch];
        }
    }
    *D = d;
}

static void pixel_sums(const om_model *m, int32_t i, int32_t j, double *D,
                       double *N, double *A)
{
    point_sums(m, (float)i + 0.5f, (float)j + 0.5f, D, N, A);
}

/* Forward render (Eqs. 2-5): y_c = N_c / D, invd = 1/D; a pixel with no
 * included kernel (D = 0) gets y = 0 and invd = 0.  px == NULL renders all
 * H*W pixels in row-major order; otherwise the n_px listed flat pixel indices
 * (j*W + i).  y is channel-planar over the rendered pixels: y[c*n + p].
 * absm (optional, same layout as y) receives sum_k w_k (|a_kc| + |W_kc (x - mu_k)|
 * taken term by term), the size of the terms of the gated sum (used to scale
 * a tolerance). */
void om_render(const om_model *m, int64_t n_px, const int64_t *px, double *y,
               double *invd, double *absm)
{
    int64_t n = px ? n_px : (int64_t)m->W * m->H;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < n; ++p) {
        int64_t f = px ? px[p] : p;
        int32_t i = (int32_t)(f % m->W), j = (int32_t)(f / m->W);
        double D, N[3], A[3];
        pixel_sums(m, i, j, &D, N, A);
        double nrm = m->rbf ? 1.0 : D;      /* Eq. 4 normalises by D, Eq. 1 does not */
        for (int ch = 0; ch < m->C; ++ch) {
            y[ch * n + p] = D > 0.0 ? N[ch] / nrm : 0.0;
            if (absm) absm[ch * n + p] = D > 0.0 ? A[ch] / nrm : 0.0;
        }
        if (invd) invd[p] = D > 0.0 ? 1.0 / D : 0.0;
    }
}

/* Resampling of the continuous regression function (Sec. II-B: "pixel
 * interpolation to any size, with regular or irregular pixel raster"): y(x)
 * at n sample points xy[2p], xy[2p+1] given in the raster's pixel units
 * (pixel (i, j) has centre (i + 0.5, j + 0.5)).  The truncated model is the
 * same pointwise definition as om_render (predicate in FP32 at the given
 * coordinates, values in FP64).  A point outside [0, W) x [0, H), or with a
 * non-finite coordinate, gets y = 0 and invd = 0.  Layout as om_render with
 * the points in place of pixels. */
void om_render_points(const om_model *m, int64_t n, const float *xy, double *y,
                      double *invd, double *absm)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < n; ++p) {
        float x = xy[2 * p], yy = xy[2 * p + 1];
        double D = 0.0, N[3] = {0.0, 0.0, 0.0}, A[3] = {0.0, 0.0, 0.0};
        if (x >= 0.0f && x < (float)m->W && yy >= 0.0f && yy < (float)m->H)
            point_sums(m, x, yy, &D, N, A);
        double nrm = m->rbf ? 1.0 : D;
        for (int ch = 0; ch < m->C; ++ch) {
            y[ch * n + p] = D > 0.0 ? N[ch] / nrm : 0.0;
            if (absm) absm[ch * n + p] = D > 0.0 ? A[ch] / nrm : 0.0;
        }
        if (invd) invd[p] = D > 0.0 ? 1.0 / D : 0.0;
    }
}

/* Backward pass of the truncated model (the gradient-descent fit of Sec. III-D
 * through the rasteriser), FP64, summed over all pixels.  Upstream gradient:
 * gy (C x H x W) if non-NULL, else the MSE against target,
 * G = 2 (y - t) / (C H W).  For an included pair with e = pi K, gate
 * g = e / D and s = g * sum_c G_c (m_c - y_c) (RBF mode: g = e and
 * s = g * sum_c G_c m_c):
 *   dL/da = -s z0 dx, dL/db = -s z0 dy, dL/dc = -s z1 dy,
 *   dL/dmu_px = (s z0 a, s (z0 b + z1 c)) - g eW^T G   (last term: linear),
 *   dL/dea_c = g G_c,  dL/deW_c = g G_c (dx, dy),  dL/dlogpi = s.
 * The indicator [q32 <= q_max] is locally constant (a.e. derivative).  Then
 * the chain rule to API units: dL/dmu_n = dL/dmu_px * (W, H) and
 * dL/d(a,b,c,eW) = dL/d(a',b',c',eW') / s.
 * ksel == NULL: all K kernels, outputs indexed by k.  Otherwise only the n_sel
 * listed kernels, outputs indexed by position in ksel.  g_pi / s_pi (the
 * gate-weight gradient and its term-magnitude sum) may be NULL. */
void om_backward(const om_model *m, const double *gy, const float *target,
                 int64_t n_sel, const int64_t *ksel, double *g_mu,
                 double *g_chol, double *g_ea, double *g_eW, double *s_mu,
                 double *s_chol, double *s_ea, double *s_eW, double *g_pi,
                 double *s_pi)
{
    const int64_t HW = (int64_t)m->W * m->H;
    const int C = m->C;
    if (!ksel) n_sel = m->K;
    /* Pixels whose state is needed: those where a selected kernel is included. */
    unsigned char *need = (unsigned char *)calloc((size_t)HW, 1);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < HW; ++p) {
        int32_t i = (int32_t)(p % m->W), j = (int32_t)(p / m->W);
        for (int64_t s = 0; s < n_sel; ++s) {
            int64_t k = ksel ? ksel[s] : s;
            if (om_included(m, k, i, j)) { need[p] = 1; break; }
        }
    }
    double *D = (double *)calloc((size_t)HW, sizeof(double));
    double *Y = (double *)calloc((size_t)HW * C, sizeof(double));
    double *G = (double *)calloc((size_t)HW * C, sizeof(double));
    const double norm = 2.0 / ((double)C * (double)HW);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < HW; ++p) {
        if (!need[p]) continue;
        int32_t i = (int32_t)(p % m->W), j = (int32_t)(p / m->W);
        double d, N[3];
        pixel_sums(m, i, j, &d, N, NULL);
        D[p] = d;
        for (int ch = 0; ch < C; ++ch) {
            double yv = d > 0.0 ? N[ch] / (m->rbf ? 1.0 : d) : 0.0;
            Y[ch * HW + p] = yv;
            G[ch * HW + p] = gy ? gy[ch * HW + p]
                                : norm * (yv - (double)target[ch * HW + p]);
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < n_sel; ++s) {
        int64_t k = ksel ? ksel[s] : s;
        float mx, my, a, b, c;
        kernel_px(m, k, &mx, &my, &a, &b, &c);
        double ga = 0, gb = 0, gc = 0, gmx = 0, gmy = 0, gpi = 0, spi = 0;
        double gea[3] = {0, 0, 0}, gw[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        /* the same sums with every factor replaced by its magnitude: the
         * size of the terms that cancel (optional outputs s_*) */
        double sa = 0, sb = 0, sc = 0, smx = 0, smy = 0;
        double sea[3] = {0, 0, 0}, sw[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        double w[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        for (int ch = 0; ch < C && m->linear; ++ch) {
            for (int d2 = 0; d2 < 2; ++d2) {
                float wf = m->eW[(k * C + ch) * 2 + d2];
                if (m->scale != 1.0f) wf = wf / m->scale;
                w[ch][d2] = (double)wf;
            }
        }
        for (int64_t p = 0; p < HW; ++p) {
            int32_t i = (int32_t)(p % m->W), j = (int32_t)(p / m->W);
            if (!om_included(m, k, i, j)) continue;
            om_pair pr;
            pair_value(m, k, i, j, &pr);
            /* softmax: dy/de_k = (m_k - y) / D; RBF: dy/de_k = m_k */
            double g = m->rbf ? pr.e : pr.e / D[p];
            double r = 0.0;
            for (int ch = 0; ch < C; ++ch)
                r += G[ch * HW + p] * (pr.mexp[ch] - (m->rbf ? 0.0 : Y[ch * HW + p]));
            double sv = g * r;
            double sabs = 0.0;
            for (int ch = 0; ch < C; ++ch)
                sabs += fabs(G[ch * HW + p]) *
                        (pr.mabs[ch] + (m->rbf ? 0.0 : fabs(Y[ch * HW + p])));
            sabs *= g;
            gpi += sv;                                /* d e_k / d logpi_k = e_k */
            spi += sabs;
            sa += sabs * fabs(pr.z0 * pr.dx);
            sb += sabs * fabs(pr.z0 * pr.dy);
            sc += sabs * fabs(pr.z1 * pr.dy);
            smx += sabs * fabs(pr.z0 * (double)a);
            smy += sabs * (fabs(pr.z0 * (double)b) + fabs(pr.z1 * (double)c));
            ga += -sv * pr.z0 * pr.dx;
            gb += -sv * pr.z0 * pr.dy;
            gc += -sv * pr.z1 * pr.dy;
            gmx += sv * pr.z0 * (double)a;
            gmy += sv * (pr.z0 * (double)b + pr.z1 * (double)c);
            for (int ch = 0; ch < C; ++ch) {
                double gG = g * G[ch * HW + p];
                gea[ch] += gG;
                sea[ch] += fabs(gG);
                if (m->linear) {
                    gw[ch][0] += gG * pr.dx;
                    gw[ch][1] += gG * pr.dy;
                    gmx -= gG * w[ch][0];
                    gmy -= gG * w[ch][1];
                    sw[ch][0] += fabs(gG * pr.dx);
                    sw[ch][1] += fabs(gG * pr.dy);
                    smx += fabs(gG * w[ch][0]);
                    smy += fabs(gG * w[ch][1]);
                }
            }
        }
        double inv_s = 1.0 / (double)m->scale;
        if (g_pi) g_pi[s] = gpi;
        if (s_pi) s_pi[s] = spi;
        g_mu[2 * s] = gmx * (double)m->W;
        g_mu[2 * s + 1] = gmy * (double)m->H;
        g_chol[3 * s] = ga * inv_s;
        g_chol[3 * s + 1] = gb * inv_s;
        g_chol[3 * s + 2] = gc * inv_s;
        for (int ch = 0; ch < C; ++ch) {
            g_ea[s * C + ch] = gea[ch];
            if (m->linear && g_eW) {
                g_eW[(s * C + ch) * 2] = gw[ch][0] * inv_s;
                g_eW[(s * C + ch) * 2 + 1] = gw[ch][1] * inv_s;
            }
        }
        if (s_mu) {
            s_mu[2 * s] = smx * (double)m->W;
            s_mu[2 * s + 1] = smy * (double)m->H;
            s_chol[3 * s] = sa * inv_s;
            s_chol[3 * s + 1] = sb * inv_s;
            s_chol[3 * s + 2] = sc * inv_s;
            for (int ch = 0; ch < C; ++ch) {
                s_ea[s * C + ch] = sea[ch];
                if (m->linear && s_eW) {
                    s_eW[(s * C + ch) * 2] = sw[ch][0] * inv_s;
                    s_eW[(s * C + ch) * 2 + 1] = sw[ch][1] * inv_s;
                }
            }
        }
    }
    free(need); free(D); free(Y); free(G);
}

/* Adam (the optimiser of Sec. VI-B), torch semantics, FP64:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps),  t = step >= 1. */
void om_adam(int64_t n, double *p, const double *g, double *mo, double *ve,
             double lr, double b1, double b2, double eps, int32_t step)
{
    double bc1 = 1.0 - pow(b1, (double)step);
    double bc2 = 1.0 - pow(b2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        mo[i] = b1 * mo[i] + (1.0 - b1) * g[i];
        ve[i] = b2 * ve[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (mo[i] / bc1) / (sqrt(ve[i] / bc2) + eps);
    }
}

/* Learning rate of the centre group at iteration it of n_it (Sec. VI-B: the
 * mu rate decays exponentially from lr0 to lr1 over the run). */
double om_lr_mu(double lr0, double lr1, int32_t it, int32_t n_it)
{
    double f = n_it > 1 ? (double)it / (double)(n_it - 1) : 0.0;
    return lr0 * pow(lr1 / lr0, f);
}

/* Gradient-descent fit (Sec. III-D / VI-B): n_it Adam iterations on the MSE
 * loss.  Master parameters and Adam state are FP64; each iteration evaluates
 * the model at the float rounding of the master parameters.  lr = {mu0, mu1,
 * chol, ea, eW}.  loss[it] receives the MSE (unclamped, before the update of
 * iteration it).  Parameters are updated in place (float outputs).  With
 * logpi non-NULL the gate weights are a fifth group at rate lr[5]. */
void om_fit(om_model *m, const float *target, int32_t n_it, const double lr[6],
            double b1, double b2, double eps, float *mu, float *chol,
            float *ea, float *eW, float *logpi, double *loss)
{
    const int64_t K = m->K;
    const int C = m->C;
    const int64_t HW = (int64_t)m->W * m->H;
    int64_t n_g[5] = {2 * K, 3 * K, (int64_t)C * K, m->linear ? 2 * (int64_t)C * K : 0,
                      logpi ? K : 0};
    float *fp[5] = {mu, chol, ea, eW, logpi};
    double *P[5], *G[5], *M[5], *V[5];
    for (int gi = 0; gi < 5; ++gi) {
        size_t n = (size_t)(n_g[gi] > 0 ? n_g[gi] : 1);
        P[gi] = (double *)calloc(n, sizeof(double));
        G[gi] = (double *)calloc(n, sizeof(double));
        M[gi] = (double *)calloc(n, sizeof(double));
        V[gi] = (double *)calloc(n, sizeof(double));
        for (int64_t x = 0; x < n_g[gi]; ++x) P[gi][x] = (double)fp[gi][x];
    }
    double *y = (double *)malloc(sizeof(double) * (size_t)(HW * C));
    m->mu = mu; m->chol = chol; m->ea = ea; m->eW = eW; m->logpi = logpi;
    for (int32_t it = 0; it < n_it; ++it) {
        for (int gi = 0; gi < 5; ++gi)
            for (int64_t x = 0; x < n_g[gi]; ++x) fp[gi][x] = (float)P[gi][x];
        if (loss) {
            om_render(m, 0, NULL, y, NULL, NULL);
            double se = 0.0;
            for (int64_t x = 0; x < HW * C; ++x) {
                double d = y[x] - (double)target[x];
                se += d * d;
            }
            loss[it] = se / (double)(HW * C);
        }
        om_backward(m, NULL, target, 0, NULL, G[0], G[1], G[2],
                    m->linear ? G[3] : NULL, NULL, NULL, NULL, NULL,
                    logpi ? G[4] : NULL, NULL);
        double lrs[5] = {om_lr_mu(lr[0], lr[1], it, n_it), lr[2], lr[3], lr[4], lr[5]};
        for (int gi = 0; gi < 5; ++gi)
            if (n_g[gi] > 0)
                om_adam(n_g[gi], P[gi], G[gi], M[gi], V[gi], lrs[gi], b1, b2,
                        eps, it + 1);
    }
    for (int gi = 0; gi < 5; ++gi) {
        for (int64_t x = 0; x < n_g[gi]; ++x) fp[gi][x] = (float)P[gi][x];
        free(P[gi]); free(G[gi]); free(M[gi]); free(V[gi]);
    }
    free(y);
}

/* The same forward, MSE and backward as om_render + om_backward(target), but
 * each pixel visits only its tile's list (tile_off / pair_k from om_bin over
 * all tiles): the binned CPU baseline.  The lists are conservative, so the
 * result equals the dense one up to the order of the FP64 sums.  Gradients
 * (API units, arrays of K rows, eW may be NULL for constant experts) are
 * overwritten; returns the MSE.  OpenMP over tiles, per-thread gradient
 * buffers added at the end. */
double om_fwd_bwd_binned(const om_model *m, const float *target, const int64_t *tile_off,
                         const int32_t *pair_k, double *g_mu, double *g_chol, double *g_ea,
                         double *g_eW)
{
    const int C = m->C;
    const int32_t T = m->T, tiles_x = (m->W + T - 1) / T, tiles_y = (m->H + T - 1) / T;
    const int64_t n_tiles = (int64_t)tiles_x * tiles_y, HW = (int64_t)m->W * m->H;
    const int64_t K = m->K, G = 2 + 3 + C + 2 * C;     /* per-kernel gradient row */
    const double norm = 2.0 / ((double)C * (double)HW);
    double se = 0.0;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double *buf = (double *)calloc((size_t)nth * (size_t)(K * G), sizeof(double));
#pragma omp parallel reduction(+ : se)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *gb = buf + (int64_t)tid * K * G;
#pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < n_tiles; ++t) {
            const int32_t x0 = (int32_t)(t % tiles_x) * T, y0 = (int32_t)(t / tiles_x) * T;
            for (int32_t j = y0; j < y0 + T && j < m->H; ++j)
                for (int32_t i = x0; i < x0 + T && i < m->W; ++i) {
                    const int64_t px = (int64_t)j * m->W + i;
                    double D = 0.0, N[3] = {0.0, 0.0, 0.0};
                    for (int64_t q = tile_off[t]; q < tile_off[t + 1]; ++q) {
                        const int64_t k = pair_k[q];
                        if (!om_included(m, k, i, j)) continue;
                        om_pair pr;
                        pair_value(m, k, i, j, &pr);
                        D += pr.e;
                        for (int ch = 0; ch < C; ++ch) N[ch] += pr.e * pr.mexp[ch];
                    }
                    if (!(D > 0.0)) {
                        for (int ch = 0; ch < C; ++ch) {
                            const double d = -(double)target[ch * HW + px];
                            se += d * d;
                        }
                        continue;
                    }
                    double Y[3], Gp[3];
                    const double nrm = m->rbf ? 1.0 : D;
                    for (int ch = 0; ch < C; ++ch) {
                        Y[ch] = N[ch] / nrm;
                        const double d = Y[ch] - (double)target[ch * HW + px];
                        se += d * d;
                        Gp[ch] = norm * d;
                    }
                    for (int64_t q = tile_off[t]; q < tile_off[t + 1]; ++q) {
                        const int64_t k = pair_k[q];
                        if (!om_included(m, k, i, j)) continue;
                        om_pair pr;
                        pair_value(m, k, i, j, &pr);
                        float mx, my, a, b, c;
                        kernel_px(m, k, &mx, &my, &a, &b, &c);
                        const double g = m->rbf ? pr.e : pr.e / D;
                        double r = 0.0;
                        for (int ch = 0; ch < C; ++ch)
                            r += Gp[ch] * (pr.mexp[ch] - (m->rbf ? 0.0 : Y[ch]));
                        const double sv = g * r;
                        double *row = gb + k * G;
                        row[0] += sv * pr.z0 * (double)a;                       /* mu_px x */
                        row[1] += sv * (pr.z0 * (double)b + pr.z1 * (double)c); /* mu_px y */
                        row[2] += -sv * pr.z0 * pr.dx;
                        row[3] += -sv * pr.z0 * pr.dy;
                        row[4] += -sv * pr.z1 * pr.dy;
                        for (int ch = 0; ch < C; ++ch) {
                            const double gG = g * Gp[ch];
                            row[5 + ch] += gG;
                            if (m->linear) {
                                float w0 = m->eW[(k * C + ch) * 2], w1 = m->eW[(k * C + ch) * 2 + 1];
                                if (m->scale != 1.0f) { w0 = w0 / m->scale; w1 = w1 / m->scale; }
                                row[0] -= gG * (double)w0;
                                row[1] -= gG * (double)w1;
                                row[5 + C + 2 * ch] += gG * pr.dx;
                                row[5 + C + 2 * ch + 1] += gG * pr.dy;
                            }
                        }
                    }
                }
        }
    }
    const double inv_s = 1.0 / (double)m->scale;
    for (int64_t k = 0; k < K; ++k) {
        double row[2 + 3 + 3 + 6];
        for (int64_t x = 0; x < G; ++x) {
            double v = 0.0;
            for (int th = 0; th < nth; ++th) v += buf[((int64_t)th * K + k) * G + x];
            row[x] = v;
        }
        g_mu[2 * k] = row[0] * (double)m->W;
        g_mu[2 * k + 1] = row[1] * (double)m->H;
        for (int d = 0; d < 3; ++d) g_chol[3 * k + d] = row[2 + d] * inv_s;
        for (int ch = 0; ch < C; ++ch) {
            g_ea[k * C + ch] = row[5 + ch];
            if (m->linear && g_eW) {
                g_eW[(k * C + ch) * 2] = row[5 + C + 2 * ch] * inv_s;
                g_eW[(k * C + ch) * 2 + 1] = row[5 + C + 2 * ch + 1] * inv_s;
            }
        }
    }
    free(buf);
    return se / (double)(HW * C);
}

/* Number of OpenMP threads the oracle uses. */
int32_t om_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

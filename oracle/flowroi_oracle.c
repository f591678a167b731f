/*
 * FlowRoI oracle: plain, slow, single-threaded FP64 C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference legs load this library.  The CUDA
 * product library never links, loads or calls it, and the two share no code:
 * no headers, no tables, no helpers.
 *
 * It follows the method of "FlowRoI" (arXiv 2511.14419):
 *   - §Optical flow extraction: dense two-frame Farneback flow on a Gaussian
 *     pyramid (polynomial expansion, then an iterated, windowed displacement
 *     solve from coarse to fine);
 *   - §Region of Interest extraction: motion saliency combining the flow
 *     magnitude with its spatial gradient at weight 0.7, min-max
 *     normalisation, a quantile ("RoI threshold") cut, opening and closing;
 *   - §Implementation details: the JPEG2000 front end the mask drives, with
 *     scaling-based RoI (DC level shift, lifting DWT 5/3 or 9/7, dead-zone
 *     quantisation, RoI coefficient up-shift by the scaling factor).
 *
 * The paper states none of the numerical constants of these stages.  The
 * readings taken here (each repeated at the function that uses it):
 *   - intensities in 8-bit units: I = raw * 255 / (2^B - 1);
 *   - pyramid: separable [1 4 6 4 1]/16 blur, replicate border, keep even
 *     samples, level size ceil(w/2);
 *   - expansion: basis {1,u,v,u^2,v^2,uv}, Gaussian applicability of
 *     sigma over a (2n+1)^2 square, replicate border, A = [[r_uu, r_uv/2],
 *     [r_uv/2, r_vv]], b = (r_u, r_v);
 *   - displacement: f1 = current frame, f2 = previous frame; prior d~ is the
 *     coarse flow bilinearly upsampled at (x/2, y/2) times 2; per iteration
 *     A = (A1(x) + A2(x+d~))/2, db = -(b2(x+d~) - b1(x))/2 + A d~,
 *     G = A^T A, h = A^T db, box mean over a (2r+1)^2 window clipped to the
 *     image, d = adj(G) h / (det G + lambda);
 *   - saliency S = a*|d| + (1-a)*|grad |d|| (central differences, replicate
 *     border), a = 0.7; S^ = (S - min)/(max - min), 0 when max == min;
 *   - threshold: k = floor(q*N), t = the (k+1)-th largest S^, mask = S^ > t;
 *   - morphology: square structuring elements, opening of radius r_open then
 *     closing of radius r_close, out-of-image pixels ignored;
 *   - DWT: whole-sample symmetric extension, per level all columns
 *     (vertical) then all rows (horizontal), Mallat layout;
 *   - 9/7 quantisation step of subband b: delta_base / sqrt(G_b) rounded to
 *     the JPEG2000 (exponent, mantissa) form; 5/3 is not quantised;
 *   - RoI coefficient: its synthesis support meets the pixel mask; RoI
 *     coefficients are multiplied by 2^s (sign kept).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int orc_version(void) { return 1; }

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------------------ a1 --
 * Frame units: raw integer samples of bit depth B mapped to 8-bit units,
 * I = raw * 255 / (2^B - 1).  (The paper's frames are 8- or 12-bit grey
 * images; flow parameters are stated in 8-bit units.) */
void orc_units(const void *raw, int bytes_per_px, int bit_depth, int64_t n, double *out)
{
    double scale = 255.0 / (double)((1 << bit_depth) - 1);
    for (int64_t i = 0; i < n; i++) {
        double v = bytes_per_px == 1 ? (double)((const uint8_t *)raw)[i]
                                     : (double)((const uint16_t *)raw)[i];
        out[i] = v * scale;
    }
}

/* ------------------------------------------------------------ f1 (opt) --
 * Denoising of the flow input (§Optical flow extraction: a two-step
 * denoising, median filtering then bilateral filtering, before the flow;
 * Table 1 "Denoise": on or off).  The paper gives no sizes; the readings:
 *   - median over the 3x3 neighbourhood, replicate border;
 *   - bilateral over the (2*rb+1)^2 square of the median image, replicate
 *     border, weight of neighbour q of pixel p
 *         exp(-|q - p|^2 / (2 sigma_s^2)) * exp(-(I(q) - I(p))^2 / (2 sigma_r^2)),
 *     output = sum(w I(q)) / sum(w), in 8-bit units.
 * The JPEG2000 front end still codes the raw frame. */
static int cmp_d(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void orc_median3(const double *in, int w, int h, double *out)
{
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double v[9];
            int k = 0;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) v[k++] = in[(size_t)clampi(y + dy, 0, h - 1) * w + clampi(x + dx, 0, w - 1)];
            qsort(v, 9, sizeof(double), cmp_d);
            out[(size_t)y * w + x] = v[4];
        }
}

void orc_bilateral(const double *in, int w, int h, int rb, double sigma_s, double sigma_r, double *out)
{
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            const double c = in[(size_t)y * w + x];
            double num = 0.0, den = 0.0;
            for (int dy = -rb; dy <= rb; dy++)
                for (int dx = -rb; dx <= rb; dx++) {
                    const double q = in[(size_t)clampi(y + dy, 0, h - 1) * w + clampi(x + dx, 0, w - 1)];
                    const double wgt = exp(-(double)(dx * dx + dy * dy) / (2.0 * sigma_s * sigma_s)) *
                                       exp(-(q - c) * (q - c) / (2.0 * sigma_r * sigma_r));
                    num += wgt * q;
                    den += wgt;
                }
            out[(size_t)y * w + x] = num / den;
        }
}

void orc_denoise(const double *in, int w, int h, int rb, double sigma_s, double sigma_r, double *tmp, double *out)
{
    orc_median3(in, w, h, tmp);
    orc_bilateral(tmp, w, h, rb, sigma_s, sigma_r, out);
}

/* ------------------------------------------------------------------ a2 --
 * One Gaussian-pyramid reduction: 5x5 binomial blur (outer product of
 * [1 4 6 4 1]/16), replicate border, sample at even coordinates.  The
 * output has ceil(w/2) x ceil(h/2) pixels. */
void orc_pyr_down(const double *src, int w, int h, double *dst)
{
    static const double b5[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
    for (int j = 0; j < h2; j++)
        for (int i = 0; i < w2; i++) {
            double s = 0.0;
            for (int v = -2; v <= 2; v++)
                for (int u = -2; u <= 2; u++) {
                    int y = clampi(2 * j + v, 0, h - 1), x = clampi(2 * i + u, 0, w - 1);
                    s += b5[u + 2] * b5[v + 2] * src[(int64_t)y * w + x];
                }
            dst[(int64_t)j * w2 + i] = s;
        }
}

/* ------------------------------------------------------------------ a3 --
 * Polynomial expansion (Farneback's signal model, cited by the paper's
 * §Optical flow extraction): in the neighbourhood of every pixel the image
 * is fitted, by weighted least squares, with
 *     f(u, v) ~ r1 + r2 u + r3 v + r4 u^2 + r5 v^2 + r6 u v
 * (u along x / columns, v along y / rows), weights a(u,v) =
 * exp(-(u^2+v^2)/(2 sigma^2)) over u,v in [-n, n].
 *
 * r = (B^T W B)^-1 B^T W f is a fixed linear map of the (2n+1)^2 samples;
 * orc_poly_projector writes that 6 x (2n+1)^2 matrix P (row-major; column
 * index (v+n)*(2n+1) + (u+n)).  Returns 0, or -1 if the Gram matrix is
 * singular. */
int orc_poly_projector(int n, double sigma, double *P)
{
    int m = 2 * n + 1, ns = m * m;
    double *B = (double *)malloc(sizeof(double) * 6 * ns);
    double *W = (double *)malloc(sizeof(double) * ns);
    double G[6][12];
    for (int v = -n; v <= n; v++)
        for (int u = -n; u <= n; u++) {
            int s = (v + n) * m + (u + n);
            double *b = B + 6 * s;
            b[0] = 1.0; b[1] = u; b[2] = v; b[3] = (double)u * u; b[4] = (double)v * v; b[5] = (double)u * v;
            W[s] = exp(-((double)u * u + (double)v * v) / (2.0 * sigma * sigma));
        }
    /* Gram matrix B^T W B, augmented with the identity for Gauss-Jordan. */
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 12; j++) G[i][j] = 0.0;
    for (int s = 0; s < ns; s++)
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) G[i][j] += B[6 * s + i] * W[s] * B[6 * s + j];
    for (int i = 0; i < 6; i++) G[i][6 + i] = 1.0;
    for (int c = 0; c < 6; c++) {
        int piv = c;
        for (int r = c + 1; r < 6; r++)
            if (fabs(G[r][c]) > fabs(G[piv][c])) piv = r;
        if (fabs(G[piv][c]) < 1e-300) { free(B); free(W); return -1; }
        if (piv != c)
            for (int j = 0; j < 12; j++) { double t = G[c][j]; G[c][j] = G[piv][j]; G[piv][j] = t; }
        double d = G[c][c];
        for (int j = 0; j < 12; j++) G[c][j] /= d;
        for (int r = 0; r < 6; r++)
            if (r != c) {
                double f = G[r][c];
                for (int j = 0; j < 12; j++) G[r][j] -= f * G[c][j];
            }
    }
    /* P = G^-1 B^T W */
    for (int i = 0; i < 6; i++)
        for (int s = 0; s < ns; s++) {
            double acc = 0.0;
            for (int k = 0; k < 6; k++) acc += G[i][6 + k] * B[6 * s + k];
            P[(int64_t)i * ns + s] = acc * W[s];
        }
    free(B);
    free(W);
    return 0;
}

/* Expansion of a whole image: five planes of w*h doubles in the order
 * A11 (= r4, the u^2 term), A12 (= r6/2), A22 (= r5), b1 (= r2), b2 (= r3).
 * Samples outside the image replicate the nearest edge pixel. */
int orc_poly_expand(const double *img, int w, int h, int n, double sigma, double *fields)
{
    int m = 2 * n + 1, ns = m * m;
    double *P = (double *)malloc(sizeof(double) * 6 * ns);
    if (orc_poly_projector(n, sigma, P) != 0) { free(P); return -1; }
    int64_t np = (int64_t)w * h;
    double *A11 = fields, *A12 = fields + np, *A22 = fields + 2 * np, *b1 = fields + 3 * np, *b2 = fields + 4 * np;
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double r[6] = {0, 0, 0, 0, 0, 0};
            for (int v = -n; v <= n; v++)
                for (int u = -n; u <= n; u++) {
                    double f = img[(int64_t)clampi(y + v, 0, h - 1) * w + clampi(x + u, 0, w - 1)];
                    int s = (v + n) * m + (u + n);
                    for (int i = 0; i < 6; i++) r[i] += P[(int64_t)i * ns + s] * f;
                }
            int64_t p = (int64_t)y * w + x;
            A11[p] = r[3];
            A12[p] = 0.5 * r[5];
            A22[p] = r[4];
            b1[p] = r[1];
            b2[p] = r[2];
        }
    free(P);
    return 0;
}

/* ------------------------------------------------------------------ a4 --
 * Bilinear sample of a w x h plane at (x, y); the coordinates are first
 * clamped to [0, w-1] x [0, h-1]. */
static double bilinear(const double *f, int w, int h, double x, double y)
{
    if (x < 0) x = 0;
    if (x > w - 1) x = w - 1;
    if (y < 0) y = 0;
    if (y > h - 1) y = h - 1;
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < w ? x0 + 1 : w - 1, y1 = y0 + 1 < h ? y0 + 1 : h - 1;
    double fx = x - x0, fy = y - y0;
    double top = (1 - fx) * f[(int64_t)y0 * w + x0] + fx * f[(int64_t)y0 * w + x1];
    double bot = (1 - fx) * f[(int64_t)y1 * w + x0] + fx * f[(int64_t)y1 * w + x1];
    return (1 - fy) * top + fy * bot;
}

/* Prior for a finer level: d~(x, y) = 2 * bilinear(d_coarse, x/2, y/2).
 * d planes: dx at [0, w*h), dy at [w*h, 2*w*h). */
void orc_flow_upsample(const double *dc, int wc, int hc, int w, int h, double *dp)
{
    int64_t nc = (int64_t)wc * hc, n = (int64_t)w * h;
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            dp[(int64_t)y * w + x] = 2.0 * bilinear(dc, wc, hc, 0.5 * x, 0.5 * y);
            dp[n + (int64_t)y * w + x] = 2.0 * bilinear(dc + nc, wc, hc, 0.5 * x, 0.5 * y);
        }
}

/* Displacement estimation at one level (Farneback two-frame method).
 * f1: the current frame's five expansion planes, f2: the previous frame's.
 * With f2(x) = f1(x - d), the expansions satisfy A2 = A1 and
 * b2 = b1 - 2 A1 d, so d solves A d = -(b2 - b1)/2; with a prior d~ the
 * second expansion is read at x + d~ and the known part A d~ is added back.
 * Each iteration: per pixel
 *     A  = (A1(x) + A2(x + d~)) / 2
 *     db = -(b2(x + d~) - b1(x)) / 2 + A d~
 *     G  = A^T A,  h = A^T db,
 * then G and h are averaged over a (2r+1)^2 box clipped to the image (mean
 * over the in-image samples) and d = adj(G) h / (det G + lambda); d becomes
 * the next iteration's d~.  dprior and d: dx plane then dy plane. */
void orc_flow_iterate_off(const double *f1, const double *f2, int w, int h, const double *dprior,
                          int iters, int win_r, double lambda, double ox, double oy, double *d);

void orc_flow_iterate(const double *f1, const double *f2, int w, int h, const double *dprior,
                      int iters, int win_r, double lambda, double *d)
{
    orc_flow_iterate_off(f1, f2, w, h, dprior, iters, win_r, lambda, 0.0, 0.0, d);
}

/* The same with the second expansion translated by (-ox, -oy): it is read
 * at x + d~ + (ox, oy).  Registration aligns the predecessor this way. */
void orc_flow_iterate_off(const double *f1, const double *f2, int w, int h, const double *dprior,
                          int iters, int win_r, double lambda, double ox, double oy, double *d)
{
    int64_t n = (int64_t)w * h;
    const double *A11a = f1, *A12a = f1 + n, *A22a = f1 + 2 * n, *b1a = f1 + 3 * n, *b2a = f1 + 4 * n;
    const double *A11b = f2, *A12b = f2 + n, *A22b = f2 + 2 * n, *b1b = f2 + 3 * n, *b2b = f2 + 4 * n;
    double *gh = (double *)malloc(sizeof(double) * 5 * n);
    double *cur = (double *)malloc(sizeof(double) * 2 * n);
    memcpy(cur, dprior, sizeof(double) * 2 * n);
    for (int it = 0; it < iters; it++) {
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                int64_t p = (int64_t)y * w + x;
                double ddx = cur[p], ddy = cur[n + p];
                double xs = x + ddx + ox, ys = y + ddy + oy;
                double a11 = 0.5 * (A11a[p] + bilinear(A11b, w, h, xs, ys));
                double a12 = 0.5 * (A12a[p] + bilinear(A12b, w, h, xs, ys));
                double a22 = 0.5 * (A22a[p] + bilinear(A22b, w, h, xs, ys));
                double db1 = -0.5 * (bilinear(b1b, w, h, xs, ys) - b1a[p]) + (a11 * ddx + a12 * ddy);
                double db2 = -0.5 * (bilinear(b2b, w, h, xs, ys) - b2a[p]) + (a12 * ddx + a22 * ddy);
                /* A is symmetric, so A^T A and A^T db use the same entries. */
                gh[p] = a11 * a11 + a12 * a12;         /* G11 */
                gh[n + p] = a11 * a12 + a12 * a22;     /* G12 */
                gh[2 * n + p] = a12 * a12 + a22 * a22; /* G22 */
                gh[3 * n + p] = a11 * db1 + a12 * db2; /* h1 */
                gh[4 * n + p] = a12 * db1 + a22 * db2; /* h2 */
            }
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                double s[5] = {0, 0, 0, 0, 0};
                int cnt = 0;
                for (int v = -win_r; v <= win_r; v++) {
                    int yy = y + v;
                    if (yy < 0 || yy >= h) continue;
                    for (int u = -win_r; u <= win_r; u++) {
                        int xx = x + u;
                        if (xx < 0 || xx >= w) continue;
                        int64_t q = (int64_t)yy * w + xx;
                        for (int k = 0; k < 5; k++) s[k] += gh[k * n + q];
                        cnt++;
                    }
                }
                double g11 = s[0] / cnt, g12 = s[1] / cnt, g22 = s[2] / cnt, h1 = s[3] / cnt, h2 = s[4] / cnt;
                double det = g11 * g22 - g12 * g12 + lambda;
                int64_t p = (int64_t)y * w + x;
                d[p] = (g22 * h1 - g12 * h2) / det;
                d[n + p] = (g11 * h2 - g12 * h1) / det;
            }
        memcpy(cur, d, sizeof(double) * 2 * n);
    }
    if (iters == 0) memcpy(d, dprior, sizeof(double) * 2 * n);
    free(gh);
    free(cur);
}

/* Full coarse-to-fine flow between the current image f1 and the previous
 * image f2 (both in 8-bit units, w x h), `levels` pyramid levels.  The
 * coarsest level starts from d~ = 0.  Output d: dx plane then dy plane. */
/* Coarse-to-fine flow of the current image against the previous image
 * registered to it: the previous frame translated by the drift (sx, sy)
 * (level-0 pixels; cur(x) ~ prev(x - s)), i.e. at level l its expansion
 * read at x + d~ - s / 2^l.  The expansion is a linear shift-invariant
 * filter, so this is the expansion of the translated frame away from the
 * border.  orc_flow is the zero drift. */
int orc_flow_reg(const double *cur, const double *prev, int w, int h, int levels, int poly_n_half,
                 double sigma, int iters, int win_r, double lambda, double sx, double sy, double *d)
{
    if (levels < 1) return -1;
    int lw[32], lh[32];
    double *p1[32], *p2[32];
    lw[0] = w; lh[0] = h;
    p1[0] = (double *)malloc(sizeof(double) * w * h);
    p2[0] = (double *)malloc(sizeof(double) * w * h);
    memcpy(p1[0], cur, sizeof(double) * w * h);
    memcpy(p2[0], prev, sizeof(double) * w * h);
    for (int l = 1; l < levels; l++) {
        lw[l] = (lw[l - 1] + 1) / 2;
        lh[l] = (lh[l - 1] + 1) / 2;
        p1[l] = (double *)malloc(sizeof(double) * lw[l] * lh[l]);
        p2[l] = (double *)malloc(sizeof(double) * lw[l] * lh[l]);
        orc_pyr_down(p1[l - 1], lw[l - 1], lh[l - 1], p1[l]);
        orc_pyr_down(p2[l - 1], lw[l - 1], lh[l - 1], p2[l]);
    }
    double *dc = NULL;
    int wc = 0, hc = 0;
    for (int l = levels - 1; l >= 0; l--) {
        int64_t n = (int64_t)lw[l] * lh[l];
        double *f1 = (double *)malloc(sizeof(double) * 5 * n);
        double *f2 = (double *)malloc(sizeof(double) * 5 * n);
        double *dp = (double *)calloc(2 * n, sizeof(double));
        double *dl = (double *)malloc(sizeof(double) * 2 * n);
        orc_poly_expand(p1[l], lw[l], lh[l], poly_n_half, sigma, f1);
        orc_poly_expand(p2[l], lw[l], lh[l], poly_n_half, sigma, f2);
        if (dc) orc_flow_upsample(dc, wc, hc, lw[l], lh[l], dp);
        const double sc = 1.0 / (double)(1 << l);
        orc_flow_iterate_off(f1, f2, lw[l], lh[l], dp, iters, win_r, lambda, -sx * sc, -sy * sc, dl);
        free(f1); free(f2); free(dp); free(dc);
        dc = dl; wc = lw[l]; hc = lh[l];
    }
    memcpy(d, dc, sizeof(double) * 2 * w * h);
    free(dc);
    for (int l = 0; l < levels; l++) { free(p1[l]); free(p2[l]); }
    return 0;
}

int orc_flow(const double *cur, const double *prev, int w, int h, int levels, int poly_n_half,
             double sigma, int iters, int win_r, double lambda, double *d)
{
    return orc_flow_reg(cur, prev, w, h, levels, poly_n_half, sigma, iters, win_r, lambda, 0.0, 0.0, d);
}

/* ------------------------------------------------------------------ a5 --
 * Motion saliency from the flow (§Region of Interest extraction: flow
 * magnitude combined with spatial gradients at weight 0.7):
 *     M = |d|,  g = |(dM/dx, dM/dy)| (central differences, replicate border),
 *     S = alpha*M + (1 - alpha)*g. */
void orc_saliency(const double *d, int w, int h, double alpha, double *S)
{
    int64_t n = (int64_t)w * h;
    double *M = (double *)malloc(sizeof(double) * n);
    for (int64_t p = 0; p < n; p++) M[p] = sqrt(d[p] * d[p] + d[n + p] * d[n + p]);
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            double gx = 0.5 * (M[(int64_t)y * w + clampi(x + 1, 0, w - 1)] - M[(int64_t)y * w + clampi(x - 1, 0, w - 1)]);
            double gy = 0.5 * (M[(int64_t)clampi(y + 1, 0, h - 1) * w + x] - M[(int64_t)clampi(y - 1, 0, h - 1) * w + x]);
            S[(int64_t)y * w + x] = alpha * M[(int64_t)y * w + x] + (1.0 - alpha) * sqrt(gx * gx + gy * gy);
        }
    free(M);
}

/* Min-max normalisation to [0, 1]; a constant map becomes all zeros. */
void orc_normalise(const double *S, int64_t n, double *Sh)
{
    double mn = S[0], mx = S[0];
    for (int64_t p = 1; p < n; p++) {
        if (S[p] < mn) mn = S[p];
        if (S[p] > mx) mx = S[p];
    }
    for (int64_t p = 0; p < n; p++) Sh[p] = mx > mn ? (S[p] - mn) / (mx - mn) : 0.0;
}

/* ------------------------------------------------------------------ a6 --
 * Quantile ("RoI threshold") cut: keep the top q fraction.  k = floor(q*N)
 * pixels at most; t = the (k+1)-th largest value (index k of the values
 * sorted in descending order); mask0 = value > t (strict, so ties at t are
 * dropped; k = 0 gives an empty mask).  q is the single-precision value of
 * the parameter, widened to double before the product. */
static int cmp_desc_d(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? 1 : (x > y ? -1 : 0);
}
static int cmp_desc_f(const void *a, const void *b)
{
    float x = *(const float *)a, y = *(const float *)b;
    return x < y ? 1 : (x > y ? -1 : 0);
}

int64_t orc_quantile_k(float q, int64_t n)
{
    int64_t k = (int64_t)floor((double)q * (double)n);
    if (k < 0) k = 0;
    if (k > n - 1) k = n - 1;
    return k;
}

double orc_threshold(const double *Sh, int64_t n, float q, uint8_t *mask0)
{
    double *s = (double *)malloc(sizeof(double) * n);
    memcpy(s, Sh, sizeof(double) * n);
    qsort(s, n, sizeof(double), cmp_desc_d);
    double t = s[orc_quantile_k(q, n)];
    free(s);
    for (int64_t p = 0; p < n; p++) mask0[p] = Sh[p] > t;
    return t;
}

/* The same cut taken on single-precision values (the precision in which a
 * single-precision pipeline makes this decision). */
float orc_threshold_f32(const float *Sh, int64_t n, float q, uint8_t *mask0)
{
    float *s = (float *)malloc(sizeof(float) * n);
    memcpy(s, Sh, sizeof(float) * n);
    qsort(s, n, sizeof(float), cmp_desc_f);
    float t = s[orc_quantile_k(q, n)];
    free(s);
    for (int64_t p = 0; p < n; p++) mask0[p] = Sh[p] > t;
    return t;
}

/* ------------------------------------------------------------------ a7 --
 * Binary morphology with a (2r+1)^2 square; only in-image pixels of the
 * square take part (erosion: AND, dilation: OR). */
void orc_erode(const uint8_t *in, int w, int h, int r, uint8_t *out)
{
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            int v = 1;
            for (int dy = -r; dy <= r && v; dy++)
                for (int dx = -r; dx <= r; dx++) {
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                    if (!in[(int64_t)yy * w + xx]) { v = 0; break; }
                }
            out[(int64_t)y * w + x] = (uint8_t)v;
        }
}

void orc_dilate(const uint8_t *in, int w, int h, int r, uint8_t *out)
{
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            int v = 0;
            for (int dy = -r; dy <= r && !v; dy++)
                for (int dx = -r; dx <= r; dx++) {
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                    if (in[(int64_t)yy * w + xx]) { v = 1; break; }
                }
            out[(int64_t)y * w + x] = (uint8_t)v;
        }
}

/* Opening (erode then dilate, radius r_open) followed by closing (dilate
 * then erode, radius r_close): removes specks, then fills small gaps. */
void orc_morph(const uint8_t *in, int w, int h, int r_open, int r_close, uint8_t *out)
{
    int64_t n = (int64_t)w * h;
    uint8_t *a = (uint8_t *)malloc(n), *b = (uint8_t *)malloc(n);
    orc_erode(in, w, h, r_open, a);
    orc_dilate(a, w, h, r_open, b);
    orc_dilate(b, w, h, r_close, a);
    orc_erode(a, w, h, r_close, out);
    free(a);
    free(b);
}

/* ------------------------------------------------------------ f2 (opt) --
 * Removal of small connected components (§Region of Interest extraction:
 * after opening and closing, residual small connected components are
 * removed by an area criterion).  Readings: 8-connectivity; a component
 * with fewer than min_area pixels is removed; min_area = 0 or 1 keeps
 * every component.  Flood fill with an explicit stack, in place. */
void orc_remove_small(uint8_t *m, int w, int h, int min_area)
{
    int64_t n = (int64_t)w * h;
    if (min_area <= 1 || n == 0) return;
    int32_t *comp = (int32_t *)malloc(n * sizeof(int32_t)); /* pixels of the current component */
    uint8_t *seen = (uint8_t *)calloc(n, 1);
    for (int64_t s = 0; s < n; s++) {
        if (!m[s] || seen[s]) continue;
        int64_t top = 0, len = 0;
        comp[len++] = (int32_t)s;
        seen[s] = 1;
        while (top < len) {
            int64_t p = comp[top++];
            int x = (int)(p % w), y = (int)(p / w);
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int xx = x + dx, yy = y + dy;
                    if ((dx == 0 && dy == 0) || xx < 0 || yy < 0 || xx >= w || yy >= h) continue;
                    int64_t q = (int64_t)yy * w + xx;
                    if (m[q] && !seen[q]) {
                        seen[q] = 1;
                        comp[len++] = (int32_t)q;
                    }
                }
        }
        if (len < min_area)
            for (int64_t i = 0; i < len; i++) m[comp[i]] = 0;
    }
    free(comp);
    free(seen);
}

/* ------------------------------------------------------------------ a8 --
 * JPEG2000 lifting DWT, one dimension, whole-sample symmetric extension
 * (x[-i] = x[i], x[n-1+i] = x[n-1-i]).  A signal of length 1 is left as it
 * is.  Output: the ceil(n/2) low-pass samples, then the floor(n/2)
 * high-pass samples. */
static int mirror(int i, int n)
{
    if (n == 1) return 0;
    int period = 2 * (n - 1);
    i %= period;
    if (i < 0) i += period;
    return i <= n - 1 ? i : period - i;
}

/* Floor division by a power of two on signed integers (arithmetic shift). */
static int32_t floor_shift(int64_t v, int s) { return (int32_t)(v >= 0 ? v >> s : -((-v + (1LL << s) - 1) >> s)); }

/* Reversible 5/3:  H[k] = x[2k+1] - floor((x[2k] + x[2k+2]) / 2)
 *                  L[k] = x[2k]   + floor((H[k-1] + H[k] + 2) / 4). */
void orc_dwt53_1d(int32_t *x, int n, int32_t *tmp)
{
    if (n < 2) return;
    for (int i = 1; i < n; i += 2) x[i] -= floor_shift((int64_t)x[mirror(i - 1, n)] + x[mirror(i + 1, n)], 1);
    for (int i = 0; i < n; i += 2) x[i] += floor_shift((int64_t)x[mirror(i - 1, n)] + x[mirror(i + 1, n)] + 2, 2);
    int nl = (n + 1) / 2;
    for (int i = 0; i < n; i++) tmp[i % 2 ? nl + i / 2 : i / 2] = x[i];
    memcpy(x, tmp, sizeof(int32_t) * n);
}

void orc_idwt53_1d(int32_t *x, int n, int32_t *tmp)
{
    if (n < 2) return;
    int nl = (n + 1) / 2;
    for (int i = 0; i < n; i++) tmp[i] = x[i % 2 ? nl + i / 2 : i / 2];
    for (int i = 0; i < n; i += 2) tmp[i] -= floor_shift((int64_t)tmp[mirror(i - 1, n)] + tmp[mirror(i + 1, n)] + 2, 2);
    for (int i = 1; i < n; i += 2) tmp[i] += floor_shift((int64_t)tmp[mirror(i - 1, n)] + tmp[mirror(i + 1, n)], 1);
    memcpy(x, tmp, sizeof(int32_t) * n);
}

/* Irreversible 9/7 (CDF 9/7 lifting factorisation, Daubechies-Sweldens, as
 * used by JPEG2000): four lifting steps with the constants below, then the
 * low band is divided by K and the high band multiplied by K (unit DC gain
 * in the low band, gain 2 at Nyquist in the high band). */
static const double L97_A = -1.586134342059924, L97_B = -0.052980118572961, L97_G = 0.882911075530934,
                    L97_D = 0.443506852043971, L97_K = 1.230174104914001;

void orc_dwt97_1d(double *x, int n, double *tmp)
{
    if (n < 2) return;
    const double c[4] = {L97_A, L97_B, L97_G, L97_D};
    for (int s = 0; s < 4; s++)
        for (int i = (s % 2 == 0) ? 1 : 0; i < n; i += 2) x[i] += c[s] * (x[mirror(i - 1, n)] + x[mirror(i + 1, n)]);
    int nl = (n + 1) / 2;
    for (int i = 0; i < n; i++) tmp[i % 2 ? nl + i / 2 : i / 2] = i % 2 ? x[i] * L97_K : x[i] / L97_K;
    memcpy(x, tmp, sizeof(double) * n);
}

void orc_idwt97_1d(double *x, int n, double *tmp)
{
    if (n < 2) return;
    const double c[4] = {L97_A, L97_B, L97_G, L97_D};
    int nl = (n + 1) / 2;
    for (int i = 0; i < n; i++) tmp[i] = i % 2 ? x[nl + i / 2] / L97_K : x[i / 2] * L97_K;
    for (int s = 3; s >= 0; s--)
        for (int i = (s % 2 == 0) ? 1 : 0; i < n; i += 2) tmp[i] -= c[s] * (tmp[mirror(i - 1, n)] + tmp[mirror(i + 1, n)]);
    memcpy(x, tmp, sizeof(double) * n);
}

/* Multi-level 2-D transforms in place on a w x h plane (row-major).  Each
 * level transforms the current low-low region: every column (vertical)
 * first, then every row (horizontal); the low-low band of size
 * ceil(cw/2) x ceil(ch/2) lands in the top-left corner (Mallat layout). */
void orc_dwt53_2d(int32_t *p, int w, int h, int levels)
{
    int32_t *line = (int32_t *)malloc(sizeof(int32_t) * (w > h ? w : h));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (w > h ? w : h));
    int cw = w, ch = h;
    for (int l = 0; l < levels; l++) {
        for (int x = 0; x < cw; x++) {
            for (int y = 0; y < ch; y++) line[y] = p[(int64_t)y * w + x];
            orc_dwt53_1d(line, ch, tmp);
            for (int y = 0; y < ch; y++) p[(int64_t)y * w + x] = line[y];
        }
        for (int y = 0; y < ch; y++) orc_dwt53_1d(p + (int64_t)y * w, cw, tmp);
        cw = (cw + 1) / 2;
        ch = (ch + 1) / 2;
    }
    free(line);
    free(tmp);
}

void orc_idwt53_2d(int32_t *p, int w, int h, int levels)
{
    int32_t *line = (int32_t *)malloc(sizeof(int32_t) * (w > h ? w : h));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (w > h ? w : h));
    int cws[64], chs[64];
    cws[0] = w; chs[0] = h;
    for (int l = 1; l <= levels; l++) { cws[l] = (cws[l - 1] + 1) / 2; chs[l] = (chs[l - 1] + 1) / 2; }
    for (int l = levels - 1; l >= 0; l--) {
        int cw = cws[l], ch = chs[l];
        for (int y = 0; y < ch; y++) orc_idwt53_1d(p + (int64_t)y * w, cw, tmp);
        for (int x = 0; x < cw; x++) {
            for (int y = 0; y < ch; y++) line[y] = p[(int64_t)y * w + x];
            orc_idwt53_1d(line, ch, tmp);
            for (int y = 0; y < ch; y++) p[(int64_t)y * w + x] = line[y];
        }
    }
    free(line);
    free(tmp);
}

void orc_dwt97_2d(double *p, int w, int h, int levels)
{
    double *line = (double *)malloc(sizeof(double) * (w > h ? w : h));
    double *tmp = (double *)malloc(sizeof(double) * (w > h ? w : h));
    int cw = w, ch = h;
    for (int l = 0; l < levels; l++) {
        for (int x = 0; x < cw; x++) {
            for (int y = 0; y < ch; y++) line[y] = p[(int64_t)y * w + x];
            orc_dwt97_1d(line, ch, tmp);
            for (int y = 0; y < ch; y++) p[(int64_t)y * w + x] = line[y];
        }
        for (int y = 0; y < ch; y++) orc_dwt97_1d(p + (int64_t)y * w, cw, tmp);
        cw = (cw + 1) / 2;
        ch = (ch + 1) / 2;
    }
    free(line);
    free(tmp);
}

void orc_idwt97_2d(double *p, int w, int h, int levels)
{
    double *line = (double *)malloc(sizeof(double) * (w > h ? w : h));
    double *tmp = (double *)malloc(sizeof(double) * (w > h ? w : h));
    int cws[64], chs[64];
    cws[0] = w; chs[0] = h;
    for (int l = 1; l <= levels; l++) { cws[l] = (cws[l - 1] + 1) / 2; chs[l] = (chs[l - 1] + 1) / 2; }
    for (int l = levels - 1; l >= 0; l--) {
        int cw = cws[l], ch = chs[l];
        for (int y = 0; y < ch; y++) orc_idwt97_1d(p + (int64_t)y * w, cw, tmp);
        for (int x = 0; x < cw; x++) {
            for (int y = 0; y < ch; y++) line[y] = p[(int64_t)y * w + x];
            orc_idwt97_1d(line, ch, tmp);
            for (int y = 0; y < ch; y++) p[(int64_t)y * w + x] = line[y];
        }
    }
    free(line);
    free(tmp);
}

/* DC level shift: x - 2^(B-1) on the raw unsigned samples. */
void orc_dc_shift(const void *raw, int bytes_per_px, int bit_depth, int64_t n, int32_t *out)
{
    int32_t off = 1 << (bit_depth - 1);
    for (int64_t i = 0; i < n; i++)
        out[i] = (bytes_per_px == 1 ? (int32_t)((const uint8_t *)raw)[i] : (int32_t)((const uint16_t *)raw)[i]) - off;
}

/* ------------------------------------------------------------------ a9 --
 * Subband of a Mallat-plane position.  Level l = 1..levels; orientation
 * 0 = HL (high horizontally, low vertically: right of the low-low block),
 * 1 = LH (below it), 2 = HH; the final low-low band is reported as
 * level = levels, orientation 3.  Table index of a subband:
 * 3*(l-1) + orientation, and 3*levels for the low-low band. */
int orc_subband_index(int x, int y, int w, int h, int levels)
{
    int cw = w, ch = h;
    for (int l = 1; l <= levels; l++) {
        int lw = (cw + 1) / 2, lh = (ch + 1) / 2;
        int hx = x >= lw, hy = y >= lh;
        if (hx || hy) return 3 * (l - 1) + (hx && hy ? 2 : (hx ? 0 : 1));
        cw = lw;
        ch = lh;
    }
    return 3 * levels;
}

/* Quantisation steps for the irreversible path.  For every subband b, G_b
 * is the squared L2 norm of its 2-D synthesis basis function, measured by
 * inverse-transforming a unit impulse placed in the middle of b on a
 * 2^(levels+4) square.  The target step delta_base / sqrt(G_b) is written in
 * the JPEG2000 form 2^(R_b - eps) * (1 + mu / 2^11) with R_b = B + gain_b
 * (gain 0 for LL, 1 for HL/LH, 2 for HH), eps in [0, 31] (5 bits), mu in
 * [0, 2047] (11 bits), mu rounded to nearest (a carry into the exponent is
 * propagated).  Outputs (length 3*levels + 1, table index as above): G,
 * the representable step as float, eps, mu.  Returns 0, or -1 when a step
 * does not fit the 5-bit exponent. */
int orc_delta_table(int levels, int bit_depth, double delta_base, double *G, float *delta, int *eps, int *mu)
{
    int S = 1 << (levels + 4);
    double *img = (double *)malloc(sizeof(double) * S * S);
    int rc = 0;
    for (int b = 0; b <= 3 * levels; b++) {
        int l = b == 3 * levels ? levels : b / 3 + 1;
        int o = b == 3 * levels ? 3 : b % 3;
        int bs = S >> l; /* subband side */
        int x = bs / 2, y = bs / 2;
        if (o == 0 || o == 2) x += bs;
        if (o == 1 || o == 2) y += bs;
        memset(img, 0, sizeof(double) * S * S);
        img[(int64_t)y * S + x] = 1.0;
        orc_idwt97_2d(img, S, S, levels);
        double g = 0.0;
        for (int64_t i = 0; i < (int64_t)S * S; i++) g += img[i] * img[i];
        G[b] = g;
        double target = delta_base / sqrt(g);
        int gain = o == 3 ? 0 : (o == 2 ? 2 : 1);
        int Rb = bit_depth + gain;
        int e = (int)floor(log2(target));
        double m = target / ldexp(1.0, e) - 1.0; /* in [0, 1) */
        int mi = (int)floor(m * 2048.0 + 0.5);
        if (mi == 2048) { mi = 0; e += 1; }
        int ep = Rb - e;
        if (ep < 0 || ep > 31) rc = -1;
        eps[b] = ep;
        mu[b] = mi;
        delta[b] = (float)(ldexp(1.0, Rb - ep) * (1.0 + mi / 2048.0));
    }
    free(img);
    return rc;
}

/* Dead-zone scalar quantiser q = sign(y) * floor(|y| / delta_b), decided in
 * single precision (the precision of a single-precision transform's
 * coefficients): the division and floor are float operations. */
void orc_quantise_f32(const float *y, int w, int h, int levels, const float *delta, int32_t *q)
{
    for (int r = 0; r < h; r++)
        for (int c = 0; c < w; c++) {
            float v = y[(int64_t)r * w + c];
            float a = fabsf(v) / delta[orc_subband_index(c, r, w, h, levels)];
            int32_t m = (int32_t)floorf(a);
            q[(int64_t)r * w + c] = v < 0 ? -m : m;
        }
}

/* The same quantiser in double precision. */
void orc_quantise_f64(const double *y, int w, int h, int levels, const float *delta, int32_t *q)
{
    for (int r = 0; r < h; r++)
        for (int c = 0; c < w; c++) {
            double v = y[(int64_t)r * w + c];
            double a = fabs(v) / (double)delta[orc_subband_index(c, r, w, h, levels)];
            int32_t m = (int32_t)floor(a);
            q[(int64_t)r * w + c] = v < 0 ? -m : m;
        }
}

/* Wavelet-domain RoI mask (JPEG2000 RoI mask generation).  A coefficient is
 * RoI when the support of its synthesis basis function meets the RoI.  In
 * one dimension, with k the coefficient index in its band:
 *   5/3: low k -> samples [2k-1, 2k+1], high k -> [2k-1, 2k+3];
 *   9/7: low k -> samples [2k-3, 2k+3], high k -> [2k-3, 2k+5];
 * intervals clipped to the signal.  Each level applies the rule to every
 * column, then every row, of the previous level's low-low mask (level 1:
 * the pixel mask); the result is written in Mallat layout (w x h, 0/1). */
static void mask_rule_1d(const uint8_t *in, int n, int wavelet, uint8_t *out)
{
    int lo0 = wavelet == 97 ? -3 : -1, lo1 = wavelet == 97 ? 3 : 1;
    int hi0 = wavelet == 97 ? -3 : -1, hi1 = wavelet == 97 ? 5 : 3;
    int nl = (n + 1) / 2, nh = n / 2;
    if (n < 2) { out[0] = in[0]; return; }
    for (int k = 0; k < nl; k++) {
        int v = 0;
        for (int i = 2 * k + lo0; i <= 2 * k + lo1; i++)
            if (i >= 0 && i < n && in[i]) v = 1;
        out[k] = (uint8_t)v;
    }
    for (int k = 0; k < nh; k++) {
        int v = 0;
        for (int i = 2 * k + hi0; i <= 2 * k + hi1; i++)
            if (i >= 0 && i < n && in[i]) v = 1;
        out[nl + k] = (uint8_t)v;
    }
}

void orc_wavelet_mask(const uint8_t *pix, int w, int h, int levels, int wavelet, uint8_t *cm)
{
    int m = w > h ? w : h;
    uint8_t *a = (uint8_t *)malloc(m), *b = (uint8_t *)malloc(m);
    memcpy(cm, pix, (size_t)w * h);
    int cw = w, ch = h;
    for (int l = 0; l < levels; l++) {
        for (int x = 0; x < cw; x++) {
            for (int y = 0; y < ch; y++) a[y] = cm[(int64_t)y * w + x];
            mask_rule_1d(a, ch, wavelet, b);
            for (int y = 0; y < ch; y++) cm[(int64_t)y * w + x] = b[y];
        }
        for (int y = 0; y < ch; y++) {
            memcpy(a, cm + (int64_t)y * w, cw);
            mask_rule_1d(a, cw, wavelet, cm + (int64_t)y * w);
        }
        cw = (cw + 1) / 2;
        ch = (ch + 1) / 2;
    }
    free(a);
    free(b);
}

/* Scaling-based RoI: q <- sign(q) * (|q| << s) on RoI coefficients.
 * Returns -1 if a shifted magnitude does not fit in 31 bits. */
int orc_roi_shift(int32_t *q, const uint8_t *cm, int64_t n, int s)
{
    int rc = 0;
    for (int64_t i = 0; i < n; i++) {
        if (!cm[i]) continue;
        int64_t a = q[i] < 0 ? -(int64_t)q[i] : q[i];
        int64_t v = a << s;
        if (v > 2147483647LL) rc = -1;
        q[i] = (int32_t)(q[i] < 0 ? -v : v);
    }
    return rc;
}

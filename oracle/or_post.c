/* Post-process stage of the oracle (Section 3.1): downscale with CoC, tile
 * max-CoC and its dilation, 9-tap prefilter, 81-tap main filter (Eq. 1), 3x3
 * median postfilter.  Test infrastructure (see oracle.h). */
#include "or_internal.h"

/* ---- generic steps -------------------------------------------------------- */

/* k-value median by sorting; for even k the lower of the two middle values */
void or_median9(const double v[9], int k, double *out) {
    double s[9];
    for (int i = 0; i < k; i++) s[i] = v[i];
    for (int i = 1; i < k; i++) {
        double x = s[i];
        int j = i - 1;
        while (j >= 0 && s[j] > x) { s[j + 1] = s[j]; j--; }
        s[j + 1] = x;
    }
    *out = s[(k - 1) / 2];
}

/* 5x5 binomial blur [1 4 6 4 1]^2 / 256 with clamp-to-edge, written as the full
 * 25-tap sum (stands in for the Gaussian of Falcor that the paper used, Section 4.1) */
void or_binomial5(const double *src, int w, int h, int C, double *dst) {
    static const double b[5] = {1, 4, 6, 4, 1};
#pragma omp parallel for schedule(static)
    for (int j = 0; j < h; j++)
        for (int i = 0; i < w; i++)
            for (int c = 0; c < C; c++) {
                double acc = 0.0;
                for (int dy = -2; dy <= 2; dy++)
                    for (int dx = -2; dx <= 2; dx++) {
                        int x = clampi(i + dx, 0, w - 1), y = clampi(j + dy, 0, h - 1);
                        acc += b[dx + 2] * b[dy + 2] * src[((size_t)y * w + x) * C + c];
                    }
                dst[((size_t)j * w + i) * C + c] = acc / 256.0;
            }
}

/* 5x5 Sobel of channel ci: derivative taps [-1 -2 0 2 1] along the axis, smoothing
 * [1 4 6 4 1] across it, normalised by 128 so that a linear ramp of slope g per
 * pixel gives exactly g.  Clamp-to-edge. */
void or_sobel5(const double *src, int w, int h, int C, int ci, double *gx, double *gy) {
    static const double sm[5] = {1, 4, 6, 4, 1}, dv[5] = {-1, -2, 0, 2, 1};
#pragma omp parallel for schedule(static)
    for (int j = 0; j < h; j++)
        for (int i = 0; i < w; i++) {
            double ax = 0.0, ay = 0.0;
            for (int dy = -2; dy <= 2; dy++)
                for (int dx = -2; dx <= 2; dx++) {
                    int x = clampi(i + dx, 0, w - 1), y = clampi(j + dy, 0, h - 1);
                    double v = src[((size_t)y * w + x) * C + ci];
                    ax += dv[dx + 2] * sm[dy + 2] * v;
                    ay += sm[dx + 2] * dv[dy + 2] * v;
                }
            gx[(size_t)j * w + i] = ax / 128.0;
            gy[(size_t)j * w + i] = ay / 128.0;
        }
}

/* ---- A1: CoC, downscale to half resolution, tile max ---------------------- */

/* Each half-resolution pixel takes the mean colour of its 2x2 block (Section 3.1,
 * "downscaled to half its resolution") and, as its depth, the nearest of the four
 * depths (so a thin foreground edge is not averaged away); its CoC radius and
 * normal are those of that nearest sample.  Depths are clamped to z_far first, so
 * the sky is the finite depth z_far everywhere in the pass.
 * rho = clamp(c(z) / 4, +-max_coc_px / 2): c is a full-res diameter, rho a hpx radius. */
void or_downscale(const OrCamera *cam, const OrParams *p, int W, int H, const float *color4,
                  const float *depth, const float *normal4, double *pp_in, double *z_h,
                  double *n_h) {
    int W2 = W / 2, H2 = H / 2;
    double rmax = 0.5 * p->max_coc_px;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H2; j++)
        for (int i = 0; i < W2; i++) {
            size_t q = (size_t)j * W2 + i;
            double col[3] = {0, 0, 0}, zmin = INFINITY;
            int kmin = 0;
            for (int k = 0; k < 4; k++) {
                int x = 2 * i + (k & 1), y = 2 * j + (k >> 1);
                size_t f = (size_t)y * W + x;
                for (int c = 0; c < 3; c++) col[c] += 0.25 * (double)color4[4 * f + c];
                double z = fmin((double)depth[f], p->z_far);
                if (z < zmin) { zmin = z; kmin = k; }
            }
            int x = 2 * i + (kmin & 1), y = 2 * j + (kmin >> 1);
            size_t f = (size_t)y * W + x;
            double rho = clampd(or_coc(cam, W, zmin) / 4.0, -rmax, rmax);
            for (int c = 0; c < 3; c++) {
                pp_in[4 * q + c] = col[c];
                n_h[3 * q + c] = (double)normal4[4 * f + c];
            }
            pp_in[4 * q + 3] = rho;
            z_h[q] = zmin;
        }
}

/* Tile T x T (hpx): max near radius max(0, -rho) and max |rho| (Section 3.1.1,
 * "maximum CoC in the tile neighbourhood"). */
void or_tile_max(const OrParams *p, int W2, int H2, const double *pp_in, double *tiles) {
    int T = p->tile, TW = (W2 + T - 1) / T, TH = (H2 + T - 1) / T;
    for (int ty = 0; ty < TH; ty++)
        for (int tx = 0; tx < TW; tx++) {
            double nm = 0.0, am = 0.0;
            for (int j = ty * T; j < ty * T + T && j < H2; j++)
                for (int i = tx * T; i < tx * T + T && i < W2; i++) {
                    double rho = pp_in[4 * ((size_t)j * W2 + i) + 3];
                    nm = fmax(nm, fmax(0.0, -rho));
                    am = fmax(am, fabs(rho));
                }
            tiles[2 * ((size_t)ty * TW + tx)] = nm;
            tiles[2 * ((size_t)ty * TW + tx) + 1] = am;
        }
}

/* Neighbourhood max over (2K+1)^2 tiles, K = ceil(rmax_hpx / T): any pixel whose
 * blur can reach the tile is seen (Section 3.1.1; also the tile fix of Section 5.3). */
void or_tile_dilate(const OrParams *p, int W2, int H2, const double *tiles, double *dil) {
    int T = p->tile, TW = (W2 + T - 1) / T, TH = (H2 + T - 1) / T;
    int K = (int)ceil(0.5 * p->max_coc_px / T);
    for (int ty = 0; ty < TH; ty++)
        for (int tx = 0; tx < TW; tx++) {
            double nm = 0.0, am = 0.0;
            for (int y = ty - K; y <= ty + K; y++)
                for (int x = tx - K; x <= tx + K; x++) {
                    if (x < 0 || y < 0 || x >= TW || y >= TH) continue;
                    nm = fmax(nm, tiles[2 * ((size_t)y * TW + x)]);
                    am = fmax(am, tiles[2 * ((size_t)y * TW + x) + 1]);
                }
            dil[2 * ((size_t)ty * TW + tx)] = nm;
            dil[2 * ((size_t)ty * TW + tx) + 1] = am;
        }
}

/* ---- A3: 9-tap bilateral prefilter (Section 3.1.1) ------------------------- */

/* Kernel diameter 1/8 of the neighbourhood's maximum CoC diameter, at least sqrt(2)
 * hpx: radius rp = max(R / 8, sqrt(2)/2) with R the dilated max |rho|.  Taps: the
 * centre and 8 taps on the circle of radius rp at angles k pi/4 (the paper's figure
 * is missing; a 3x3 ring is taken).  Bilateral weight (reading): 1 - |rho_j -
 * rho_0| / max(1, |rho_0|), saturated.  CoC and depth pass through unfiltered. */
void or_prefilter(const OrParams *p, int W2, int H2, const double *pp_in, const double *dil,
                  double *pre) {
    int T = p->tile, TW = (W2 + T - 1) / T;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H2; j++)
        for (int i = 0; i < W2; i++) {
            size_t q = (size_t)j * W2 + i;
            double R = dil[2 * ((size_t)(j / T) * TW + (i / T)) + 1];
            double rp = fmax(R / 8.0, sqrt(2.0) / 2.0);
            const double *c0 = pp_in + 4 * q;
            double rho0 = c0[3];
            double acc[3] = {c0[0], c0[1], c0[2]}, wsum = 1.0;
            for (int k = 0; k < 8; k++) {
                double th = k * M_PI / 4.0, s[4];
                bilinear_clamped(pp_in, W2, H2, 4, i + rp * cos(th), j + rp * sin(th), s);
                double w = saturate(1.0 - fabs(s[3] - rho0) / fmax(1.0, fabs(rho0)));
                for (int c = 0; c < 3; c++) acc[c] += w * s[c];
                wsum += w;
            }
            for (int c = 0; c < 3; c++) pre[4 * q + c] = acc[c] / wsum;
            pre[4 * q + 3] = rho0;
        }
}

/* ---- A4: 81-tap main filter (Section 3.1.2, Eq. 1) ------------------------- */

/* tap t of the 81-tap kernel (declared in oracle.h): centre (t = 0), then rings
 * k = 1..4 of 8k taps at angles 2 pi m / (8k), at radius k/4 of the kernel radius on
 * the circle, or on the n-gon boundary in the same direction */
void or_ring_tap(int n, int t, double out[3]) {
    if (t == 0) { out[0] = 0; out[1] = 0; out[2] = 0; return; }
    int k = 1, base = 1;
    while (t >= base + 8 * k) { base += 8 * k; k++; }
    int m = t - base;
    double th = 2.0 * M_PI * m / (8.0 * k);
    double rho = or_poly_rho(n, th);
    out[0] = rho * cos(th);
    out[1] = rho * sin(th);
    out[2] = k / 4.0;
}

/* Coverage test D of Eq. 1: the paper counts a sample when its CoC radius exceeds
 * its distance to the kernel centre; here as the unit-width ramp
 * saturate((r - dist) / ramp + 1/2) so that the output is continuous in r. */
static double coverage(double dist, double r, double ramp) {
    return saturate((r - dist) / ramp + 0.5);
}

/* sampleAlpha (named but not defined in Section 3.1.2): the share of the sample's
 * blur disk that lands on one pixel, 1 / (pi r^2), at most 1; for an n-gon aperture
 * the share of its n-gon of circumradius r, 1 / (A_n r^2). */
static double sample_alpha(int n, double r) {
    double A = or_poly_area(n);
    double rr = fmax(fabs(r), 1.0 / sqrt(A));
    return 1.0 / (A * rr * rr);
}

/* Main filter.  Kernel radius R = the dilated max |rho| of the pixel's tile.  For
 * each tap (bilinear fetch of prefiltered rgb, rho and of the depth):
 *   foreground share  wf = saturate((z0 - zi) / depth_range)
 *   W_f = wf * D(dist, |rho_i|) * alpha(rho_i)                (foreground scatters
 *   W_b = (1 - wf) * D(dist, min(|rho_i|, |rho_0|)) * alpha(rho_i)    as gather)
 *   v_p = sum (W_f + W_b) c_i / sum (W_f + W_b)               (Eq. 1)
 * plus the W-weighted share of bright samples, saturate((lum - bright_lum) /
 * bright_ramp), used for bright bokeh in the composite. */
void or_main_filter(const OrParams *p, int W2, int H2, const double *pre, const double *z_h,
                    const double *dil, double *out) {
    int T = p->tile, TW = (W2 + T - 1) / T;
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < H2; j++)
        for (int i = 0; i < W2; i++) {
            size_t q = (size_t)j * W2 + i;
            double R = dil[2 * ((size_t)(j / T) * TW + (i / T)) + 1];
            double z0 = z_h[q], rho0 = pre[4 * q + 3];
            double acc[3] = {0, 0, 0}, bright = 0.0, wsum = 0.0;
            for (int t = 0; t < 81; t++) {
                double u[3];
                or_ring_tap((int)p->blades, t, u);
                double ux = u[0], uy = u[1], frac = u[2];
                double dist = frac * R;
                double x = i + dist * ux, y = j + dist * uy;
                double s[4], zi;
                bilinear_clamped(pre, W2, H2, 4, x, y, s);
                bilinear_clamped(z_h, W2, H2, 1, x, y, &zi);
                double ri = fabs(s[3]);
                double wf = saturate((z0 - zi) / p->depth_range);
                double a = sample_alpha((int)p->blades, s[3]);
                double Wf = wf * coverage(dist, ri, p->cover_ramp) * a;
                double Wb = (1.0 - wf) * coverage(dist, fmin(ri, fabs(rho0)), p->cover_ramp) * a;
                double Wt = Wf + Wb;
                for (int c = 0; c < 3; c++) acc[c] += Wt * s[c];
                bright += Wt * saturate((luminance(s) - p->bright_lum) / p->bright_ramp);
                wsum += Wt;
            }
            for (int c = 0; c < 3; c++) out[4 * q + c] = acc[c] / wsum;
            out[4 * q + 3] = bright / wsum;
        }
}

/* ---- A5: 3x3 median postfilter (Section 3.1.3) ----------------------------- */

/* per-channel median of the 3x3 neighbourhood (clamp-to-edge), all 4 channels */
void or_median3x3(int W2, int H2, const double *src, double *dst) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H2; j++)
        for (int i = 0; i < W2; i++)
            for (int c = 0; c < 4; c++) {
                double v[9];
                int n = 0;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        int x = clampi(i + dx, 0, W2 - 1), y = clampi(j + dy, 0, H2 - 1);
                        v[n++] = src[4 * ((size_t)y * W2 + x) + c];
                    }
                or_median9(v, 9, &dst[4 * ((size_t)j * W2 + i) + c]);
            }
}

/* Median, spatial reconstruction (Section 3.2.4, Eq. 5, Eq. 8) and composite
 * (Section 3.3, Eq. 6, Eq. 7) of the oracle.  Test infrastructure (see oracle.h). */
#include "or_internal.h"

void or_median9(const double v[9], int k, double *out);

/* ---- A10: 3x3 median of the ray-traced colour (Section 3.2.4) ------------- */

/* Per colour channel, the median over the pixels of the 3x3 neighbourhood that
 * have rays (lower median for an even count); the hit ratio is copied. */
void or_median_rt(int W2, int H2, const double *crt, const int32_t *nrays, double *dst) {
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H2; j++)
        for (int i = 0; i < W2; i++) {
            size_t q = (size_t)j * W2 + i;
            if (nrays[q] <= 0) {
                for (int c = 0; c < 4; c++) dst[4 * q + c] = 0.0;
                continue;
            }
            for (int c = 0; c < 3; c++) {
                double v[9];
                int n = 0;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        int x = i + dx, y = j + dy;
                        if (x < 0 || y < 0 || x >= W2 || y >= H2) continue;
                        if (nrays[(size_t)y * W2 + x] <= 0) continue;
                        v[n++] = crt[4 * ((size_t)y * W2 + x) + c];
                    }
                or_median9(v, n, &dst[4 * q + c]);
            }
            dst[4 * q + 3] = crt[4 * q + 3];
        }
}

/* ---- A11: mip pyramid and reconstruction ---------------------------------- */

/* Level 0 texel: (r, g, b, h, c_t, 1) * v with v = 1 for pixels with rays, else 0.
 * Level k+1 is the 2x2 box average of level k (clamp-to-edge for odd sizes). */
typedef struct { int w[8], h[8], L; double *lv[8]; } Mips;

static void mips_build(Mips *m, int W2, int H2, int L, const double *med, const double *ct,
                       const int32_t *nrays) {
    m->L = L;
    m->w[0] = W2; m->h[0] = H2;
    m->lv[0] = (double *)malloc(sizeof(double) * 6 * (size_t)W2 * H2);
    for (size_t q = 0; q < (size_t)W2 * H2; q++) {
        double v = nrays[q] > 0 ? 1.0 : 0.0;
        double *t = m->lv[0] + 6 * q;
        for (int c = 0; c < 4; c++) t[c] = v * med[4 * q + c];
        t[4] = v * ct[q];
        t[5] = v;
    }
    for (int k = 1; k < L; k++) {
        int w = (m->w[k - 1] + 1) / 2, h = (m->h[k - 1] + 1) / 2;
        m->w[k] = w; m->h[k] = h;
        m->lv[k] = (double *)malloc(sizeof(double) * 6 * (size_t)w * h);
        for (int j = 0; j < h; j++)
            for (int i = 0; i < w; i++)
                for (int c = 0; c < 6; c++) {
                    double a = 0.0;
                    for (int b = 0; b < 4; b++) {
                        int x = clampi(2 * i + (b & 1), 0, m->w[k - 1] - 1);
                        int y = clampi(2 * j + (b >> 1), 0, m->h[k - 1] - 1);
                        a += m->lv[k - 1][6 * ((size_t)y * m->w[k - 1] + x) + c];
                    }
                    m->lv[k][6 * ((size_t)j * w + i) + c] = 0.25 * a;
                }
    }
}

static void mips_free(Mips *m) {
    for (int k = 0; k < m->L; k++) free(m->lv[k]);
}

/* trilinear sample at half-resolution coordinates (x, y) and level `lod` */
static void trilinear(const Mips *m, double x, double y, double lod, double out[6]) {
    int l0 = (int)floor(lod);
    double t = lod - l0;
    if (l0 >= m->L - 1) { l0 = m->L - 1; t = 0.0; }
    int l1 = l0 + 1 < m->L ? l0 + 1 : l0;
    double a[6], b[6];
    double s0 = ldexp(1.0, -l0), s1 = ldexp(1.0, -l1);
    bilinear_clamped(m->lv[l0], m->w[l0], m->h[l0], 6, (x + 0.5) * s0 - 0.5, (y + 0.5) * s0 - 0.5, a);
    bilinear_clamped(m->lv[l1], m->w[l1], m->h[l1], 6, (x + 0.5) * s1 - 0.5, (y + 0.5) * s1 - 0.5, b);
    for (int c = 0; c < 6; c++) out[c] = (1.0 - t) * a[c] + t * b[c];
}

/* Reconstruction: the 81-tap ring kernel (on the aperture's shape, or_ring_tap) scaled to the accumulated CoC radius
 * c_t, sampled trilinearly at lod = clamp(c_t * 0.05, 0, 3) (Eq. 8).  A sample
 * whose CoC radius is below its distance to the centre is rejected (the coverage
 * ramp D of the main filter, on the sample's own c_t).  The filtered colour and
 * hit ratio are blended with the pixel's own by b = clamp(sigma^2 * 2000, 0, 0.9)
 * (Eq. 5), sigma^2 the blurred variance. */
void or_recon(const OrParams *p, int W2, int H2, const double *med, const double *ct,
              const double *var_blur, const int32_t *nrays, double *out) {
    Mips m;
    int L = (int)ceil(p->lod_max) + 1;
    if (L > 8) L = 8;
    mips_build(&m, W2, H2, L, med, ct, nrays);
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < H2; j++)
        for (int i = 0; i < W2; i++) {
            size_t q = (size_t)j * W2 + i;
            if (nrays[q] <= 0) {
                for (int c = 0; c < 4; c++) out[4 * q + c] = 0.0;
                continue;
            }
            double R = ct[q];
            double lod = clampd(R * p->lod_scale, 0.0, p->lod_max);
            double num[4] = {0, 0, 0, 0}, den = 0.0;
            for (int t = 0; t < 81; t++) {
                double u[3], S[6];
                or_ring_tap((int)p->blades, t, u);
                double ux = u[0], uy = u[1], frac = u[2];
                double dist = frac * R;
                trilinear(&m, i + dist * ux, j + dist * uy, lod, S);
                double ri = S[5] > 0.0 ? S[4] / S[5] : 0.0;
                double D = saturate((ri - dist) / p->cover_ramp + 0.5);
                for (int c = 0; c < 4; c++) num[c] += D * S[c];
                den += D * S[5];
            }
            double b = clampd(var_blur[q] * p->var_w_recon, 0.0, p->b_max);
            for (int c = 0; c < 4; c++) {
                double orig = med[4 * q + c];
                double filt = den > 0.0 ? num[c] / den : orig;
                out[4 * q + c] = lerp(orig, filt, b);
            }
        }
    mips_free(&m);
}

/* ---- A12: composite (Section 3.3) ------------------------------------------ */

/* Per full-resolution pixel:
 *  - zone of focus (Eq. 6): |c| <= sqrt(2) keeps the sharp raster colour; here
 *    as the ramp w_sharp = saturate((sqrt(2) - |c| + eps/2) / eps);
 *  - post-process colour PP (rgb, bright) and ray-traced colour RT (rgb, h)
 *    upsampled bilinearly from half resolution; RT over the pixels that have
 *    rays, renormalised, with coverage cov;
 *  - near field (c < 0): lerp(RT, PP, bright)  (bright bokeh from the PP pass);
 *  - far field: lerp(RT, PP, smoothstep(0, 0.3, h))  (Eq. 7);
 *  - without ray coverage the PP colour: lerp(PP, blend, cov);
 *  - out = lerp(blend, sharp, w_sharp). */
void or_composite(const OrCamera *cam, const OrParams *p, int W, int H, const float *color4,
                  const float *depth, const double *pp_med, const double *recon,
                  const int32_t *nrays, double *out) {
    int W2 = W / 2, H2 = H / 2;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H; j++)
        for (int i = 0; i < W; i++) {
            size_t f = (size_t)j * W + i;
            double z = fmin((double)depth[f], p->z_far);
            double c = or_coc(cam, W, z);
            double ws = saturate((sqrt(2.0) - fabs(c) + 0.5 * p->zof_ramp) / p->zof_ramp);
            double xh = 0.5 * (i + 0.5) - 0.5, yh = 0.5 * (j + 0.5) - 0.5;
            double pp[4];
            bilinear_clamped(pp_med, W2, H2, 4, xh, yh, pp);
            /* ray-traced layer, renormalised over pixels with rays */
            double x0f = floor(xh), y0f = floor(yh), fx = xh - x0f, fy = yh - y0f;
            int x0 = (int)x0f, y0 = (int)y0f;
            double rt[4] = {0, 0, 0, 0}, cov = 0.0;
            for (int dy = 0; dy < 2; dy++)
                for (int dx = 0; dx < 2; dx++) {
                    int x = clampi(x0 + dx, 0, W2 - 1), y = clampi(y0 + dy, 0, H2 - 1);
                    size_t q = (size_t)y * W2 + x;
                    if (nrays[q] <= 0) continue;
                    double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy);
                    for (int k = 0; k < 4; k++) rt[k] += w * recon[4 * q + k];
                    cov += w;
                }
            double sharp[3] = {color4[4 * f], color4[4 * f + 1], color4[4 * f + 2]};
            for (int k = 0; k < 3; k++) {
                double blend = pp[k];
                if (cov > 0.0) {
                    double r = rt[k] / cov, hh = rt[3] / cov;
                    double mix = c < 0.0 ? lerp(r, pp[k], pp[3])
                                         : lerp(r, pp[k], smoothstep(0.0, p->h_edge, hh));
                    blend = lerp(pp[k], mix, cov);
                }
                out[4 * f + k] = lerp(blend, sharp[k], ws);
            }
            out[4 * f + 3] = 1.0;
        }
}

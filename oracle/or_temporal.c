/* Temporal accumulation and reprojection of the ray-traced layer (Section 3.2.3)
 * in the oracle.  Test infrastructure (see oracle.h). */
#include "or_internal.h"

static double focal_px(const OrCamera *c, int W) {
    double v = c->f * c->d / (c->d - c->f);
    return (double)W * v / c->ws;
}

/* Position of the world point X in the previous frame, in half-resolution pixel
 * coordinates (texel centres at integers; the previous frame's pixels sampled the
 * sensor at their position plus its jitter).  0 when X is not in front of the
 * previous camera. */
static int project_prev(const OrCamera *c, int W, int H, const double X[3], double *xh,
                        double *yh) {
    double rel[3];
    sub3(X, c->pO, rel);
    double zc = dot3(rel, c->pF);
    if (!(zc > 0.0)) return 0;
    double F = focal_px(c, W);
    double x = 0.5 * W + F * dot3(rel, c->pR) / zc - c->pjx;
    double y = 0.5 * H - F * dot3(rel, c->pU) / zc - c->pjy;
    *xh = 0.5 * x - 0.5;
    *yh = 0.5 * y - 0.5;
    return fabs(*xh) < 1e7 && fabs(*yh) < 1e7;
}

/* Bilinear fetch of history channels at (x, y): taps outside the image or without
 * history (h + g == 0) are dropped.  Returns the covered weight and the weighted
 * channel sums (not renormalised). */
static double fetch(const double *hist, int W2, int H2, double x, double y, const int *ch, int nch,
                    double *acc) {
    double x0f = floor(x), y0f = floor(y), fx = x - x0f, fy = y - y0f, wsum = 0.0;
    int x0 = (int)x0f, y0 = (int)y0f;
    for (int c = 0; c < nch; c++) acc[c] = 0.0;
    for (int dy = 0; dy < 2; dy++)
        for (int dx = 0; dx < 2; dx++) {
            int xi = x0 + dx, yi = y0 + dy;
            if (xi < 0 || yi < 0 || xi >= W2 || yi >= H2) continue;
            const double *hq = hist + 12 * ((size_t)yi * W2 + xi);
            if (!(hq[6] + hq[7] > 0.0)) continue;
            double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy);
            for (int c = 0; c < nch; c++) acc[c] += w * hq[ch[c]];
            wsum += w;
        }
    return wsum;
}

static int camera_moved(const OrCamera *c) {
    for (int k = 0; k < 3; k++)
        if (c->O[k] != c->pO[k] || c->R[k] != c->pR[k] || c->U[k] != c->pU[k] || c->F[k] != c->pF[k])
            return 1;
    return 0;
}

/* Per half-resolution pixel with rays:
 *  - near field reprojected with the motion of the G-buffer surface (the pixel's
 *    depth through the current camera, projected by the previous one);
 *  - far field reprojected from the mean far-hit position of the pixel, else the
 *    mean over the 3x3 neighbours that have far hits, else the G-buffer position;
 *  - exponential moving average with blend alpha (0.95; alpha_motion when the
 *    camera moved, Section 5.3).  The history weight is scaled by the covered
 *    share W of the bilinear footprint (new = alpha * sum_k w_k H_k + (1 - alpha
 *    W) * current), which is the plain EMA when the footprint is fully covered and
 *    a restart when it is not covered at all (first frame, disocclusion);
 *  - near quantities (An, h, Bn, luminance moments) follow the near reprojection,
 *    far quantities (Af, g = 1 - h, Bf) the far one;
 *  - merge by lerp on the accumulated hit ratio (C = (An + Af) / (h + g)), or on
 *    the latest hit ratio when the camera moved (C = h Cn + (1-h) Cf with the
 *    normalised field colours); the CoC c_t is merged the same way;
 *  - luminance variance from the moments of the current merged ray colour
 *    (Schied et al. 2017): sigma^2 = max(0, mu2 - mu1^2).
 * Pixels without rays keep no history (all zero). */
void or_accumulate(const OrCamera *c, const OrParams *p, int W, int H, const double *z_h,
                   const double *rt, const int32_t *nrays, const double *hist_in, int has_history,
                   double *hist_out, double *crt, double *ct, double *var) {
    int W2 = W / 2, H2 = H / 2;
    int moved = camera_moved(c);
    int unchanged = !moved && c->jx == c->pjx && c->jy == c->pjy;
    double alpha = moved ? p->alpha_motion : p->alpha;
    static const int near_ch[7] = {0, 1, 2, 6, 8, 10, 11};
    static const int far_ch[5] = {3, 4, 5, 7, 9};
#pragma omp parallel for schedule(static)
    for (int j = 0; j < H2; j++)
        for (int i = 0; i < W2; i++) {
            size_t q = (size_t)j * W2 + i;
            double *ho = hist_out + 12 * q;
            if (nrays[q] <= 0) {
                for (int k = 0; k < 12; k++) ho[k] = 0.0;
                for (int k = 0; k < 4; k++) crt[4 * q + k] = 0.0;
                ct[q] = 0.0;
                var[q] = 0.0;
                continue;
            }
            const double *r = rt + 14 * q;
            double h = r[1], g = 1.0 - h;
            double cur[3] = {r[2] + r[5], r[3] + r[6], r[4] + r[7]};
            double L = luminance(cur);
            /* world positions */
            double dp[3], Xn[3], Xf[3];
            or_pixel_dir(c, W, H, 2.0 * i + 1.0, 2.0 * j + 1.0, dp);
            double s = z_h[q] / dot3(dp, c->F);
            for (int k = 0; k < 3; k++) Xn[k] = c->O[k] + s * dp[k];
            if (r[13] > 0.0) {
                for (int k = 0; k < 3; k++) Xf[k] = r[10 + k];
            } else {
                double acc[3] = {0, 0, 0};
                int cnt = 0;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        int x = i + dx, y = j + dy;
                        if (x < 0 || y < 0 || x >= W2 || y >= H2) continue;
                        const double *rn = rt + 14 * ((size_t)y * W2 + x);
                        if (nrays[(size_t)y * W2 + x] > 0 && rn[13] > 0.0) {
                            for (int k = 0; k < 3; k++) acc[k] += rn[10 + k];
                            cnt++;
                        }
                    }
                for (int k = 0; k < 3; k++) Xf[k] = cnt ? acc[k] / cnt : Xn[k];
            }
            double Hn[7] = {0}, Hf[5] = {0}, Wn = 0.0, Wf = 0.0, xh, yh;
            if (has_history) {
                if (project_prev(c, W, H, Xn, &xh, &yh)) Wn = fetch(hist_in, W2, H2, xh, yh, near_ch, 7, Hn);
                /* an unchanged camera (pose and jitter) maps every static point onto its own
                 * pixel: the far field keeps its pixel (the mean far position would move it by
                 * a fraction of a pixel every frame and smear the history) */
                if (unchanged) {
                    Wf = fetch(hist_in, W2, H2, (double)i, (double)j, far_ch, 5, Hf);
                } else if (project_prev(c, W, H, Xf, &xh, &yh)) {
                    Wf = fetch(hist_in, W2, H2, xh, yh, far_ch, 5, Hf);
                }
            }
            double kn = 1.0 - alpha * Wn, kf = 1.0 - alpha * Wf;
            double An[3], Af[3];
            for (int k = 0; k < 3; k++) {
                An[k] = alpha * Hn[k] + kn * r[2 + k];
                Af[k] = alpha * Hf[k] + kf * r[5 + k];
            }
            double ha = alpha * Hn[3] + kn * h;
            double ga = alpha * Hf[3] + kf * g;
            double Bn = alpha * Hn[4] + kn * r[8];
            double Bf = alpha * Hf[4] + kf * r[9];
            double m1 = alpha * Hn[5] + kn * L;
            double m2 = alpha * Hn[6] + kn * L * L;
            for (int k = 0; k < 3; k++) { ho[k] = An[k]; ho[3 + k] = Af[k]; }
            ho[6] = ha; ho[7] = ga; ho[8] = Bn; ho[9] = Bf; ho[10] = m1; ho[11] = m2;
            var[q] = fmax(0.0, m2 - m1 * m1);
            if (!moved) {
                double den = ha + ga;
                for (int k = 0; k < 3; k++) crt[4 * q + k] = (An[k] + Af[k]) / den;
                crt[4 * q + 3] = ha / den;
                ct[q] = (Bn + Bf) / den;
            } else {
                for (int k = 0; k < 3; k++) {
                    double cn = ha > 0.0 ? An[k] / ha : 0.0, cf = ga > 0.0 ? Af[k] / ga : 0.0;
                    crt[4 * q + k] = h * cn + (1.0 - h) * cf;
                }
                crt[4 * q + 3] = h;
                double bn = ha > 0.0 ? Bn / ha : 0.0, bf = ga > 0.0 ? Bf / ga : 0.0;
                ct[q] = h * bn + (1.0 - h) * bf;
            }
        }
}

/* Final temporal anti-aliasing of the composited image in the oracle (Section 3.4:
 * the final image is resolved with TAA after Karis 2014, reprojecting the previous
 * frame onto the newest).  Test infrastructure (see oracle.h).
 *
 * Per full-resolution pixel (x, y): the surface it shows (G-buffer depth along the
 * pixel's jittered ray) is projected into the previous frame (whose pixels sampled the
 * sensor at their position plus its jitter); the previous resolved image is sampled
 * there bilinearly (clamp to edge), clamped per channel to the min / max of the current
 * 3x3 neighbourhood, and blended with the current colour:
 *     out = h + taa_alpha (cur - h).
 * A point that projects outside the previous image takes the clamped edge texel (the
 * neighbourhood clamp bounds what it brings in); without a previous frame, or for a
 * point behind the previous camera, out = cur. */
#include "or_internal.h"

static double focal_px(const OrCamera *c, int W) {
    double v = c->f * c->d / (c->d - c->f);
    return (double)W * v / c->ws;
}

void or_taa(const OrCamera *c, const OrParams *p, int W, int H, const float *depth, const double *cur,
            const double *hist_in, int has_history, double *out) {
    double F = focal_px(c, W);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            size_t q = (size_t)y * W + x;
            const double *cq = cur + 4 * q;
            double *o = out + 4 * q;
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int xx = x + dx < 0 ? 0 : (x + dx >= W ? W - 1 : x + dx);
                    int yy = y + dy < 0 ? 0 : (y + dy >= H ? H - 1 : y + dy);
                    const double *n = cur + 4 * ((size_t)yy * W + xx);
                    for (int k = 0; k < 3; k++) {
                        lo[k] = fmin(lo[k], n[k]);
                        hi[k] = fmax(hi[k], n[k]);
                    }
                }
            for (int k = 0; k < 3; k++) o[k] = cq[k];
            o[3] = 1.0;
            if (!has_history) continue;
            double z = fmin((double)depth[q], p->z_far);
            double dir[3];
            or_pixel_dir(c, W, H, x + 0.5, y + 0.5, dir);
            double s = z / dot3(dir, c->F);
            double P[3] = {c->O[0] + s * dir[0], c->O[1] + s * dir[1], c->O[2] + s * dir[2]}, rel[3];
            sub3(P, c->pO, rel);
            double zc = dot3(rel, c->pF);
            if (!(zc > 0.0)) continue;
            double u = 0.5 * W + F * dot3(rel, c->pR) / zc - c->pjx;
            double v = 0.5 * H - F * dot3(rel, c->pU) / zc - c->pjy;
            /* texel centres at integers */
            double tx = u - 0.5, ty = v - 0.5;
            double x0f = floor(tx), y0f = floor(ty), fx = tx - x0f, fy = ty - y0f;
            int x0 = (int)x0f, y0 = (int)y0f;
            double h[3] = {0, 0, 0};
            for (int t = 0; t < 4; t++) {
                int ddx = t & 1, ddy = t >> 1;
                int xi = x0 + ddx < 0 ? 0 : (x0 + ddx >= W ? W - 1 : x0 + ddx);
                int yi = y0 + ddy < 0 ? 0 : (y0 + ddy >= H ? H - 1 : y0 + ddy);
                double w = (ddx ? fx : 1.0 - fx) * (ddy ? fy : 1.0 - fy);
                const double *hq = hist_in + 4 * ((size_t)yi * W + xi);
                for (int k = 0; k < 3; k++) h[k] += w * hq[k];
            }
            for (int k = 0; k < 3; k++) {
                double hc = fmin(fmax(h[k], lo[k]), hi[k]);
                o[k] = hc + p->taa_alpha * (cq[k] - hc);
            }
        }
}

/* Thin-lens camera of the oracle: circle of confusion, pixel rays, Philox lens
 * samples.  Test infrastructure (see oracle.h). */
#include "or_internal.h"

/* Signed CoC diameter in full-resolution pixels of a point at depth z (distance
 * along the optical axis from the lens plane).
 *
 * The paper gives the CoC only through its zone-of-focus bounds (Section 3.3,
 * Eq. 6): |CoC| <= sqrt(2) pixels exactly between those two depths.  The thin-lens
 * CoC of Potmesil and Chakravarty that reproduces both bounds is
 *     c(z) = a f (z - d) / (z (d - f)) * W / w_s,   a = f / N,
 * negative in front of the focus plane (near field) and positive behind it. */
double or_coc(const OrCamera *c, int W, double z) {
    double a = c->f / c->N;
    return a * c->f * (z - c->d) / (z * (c->d - c->f)) * ((double)W / c->ws);
}

/* Eq. 6: zone of focus [z_near, z_far] where |c| <= sqrt(2).  z_far is +inf when
 * the denominator is not positive (the zone reaches infinity). */
void or_zof_bounds(const OrCamera *c, int W, double *z_near, double *z_far) {
    double a = c->f / c->N;
    double k = sqrt(2.0) * (c->d - c->f) * (c->ws / (double)W);
    *z_near = a * c->f * c->d / (a * c->f + k);
    double den = a * c->f - k;
    *z_far = den > 0.0 ? a * c->f * c->d / den : INFINITY;
}

/* Image distance v = f d / (d - f); focal length in pixels F = W v / w_s.  The
 * field of view follows from the sensor at distance v behind the lens, which makes
 * the ray-traced blur agree with c(z) above. */
static double focal_px(const OrCamera *c, int W) {
    double v = c->f * c->d / (c->d - c->f);
    return (double)W * v / c->ws;
}

/* Direction through the sensor point (x, y) (full-resolution pixel units, y down)
 * and the lens centre; the frame's camera jitter (jx, jy) shifts every sampling
 * position by a sub-pixel offset (Section 3.1.2: the camera is jittered against
 * aliasing). */
void or_pixel_dir(const OrCamera *c, int W, int H, double x, double y, double dir[3]) {
    double F = focal_px(c, W);
    double sx = (x + c->jx - 0.5 * W) / F, sy = (y + c->jy - 0.5 * H) / F;
    for (int k = 0; k < 3; k++) dir[k] = c->F[k] + sx * c->R[k] - sy * c->U[k];
    normalize3(dir);
}

/* Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel Random Numbers: As Easy
 * as 1, 2, 3", SC 2011): ten rounds of two 64x64->128 multiplies with a Weyl
 * sequence key schedule. */
void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double or_poly_rho(int n, double th) {
    if (n <= 0) return 1.0;
    double sector = 2.0 * M_PI / n;
    double phi = fmod(th, sector);
    if (phi < 0.0) phi += sector;
    return cos(M_PI / n) / cos(phi - M_PI / n);
}

double or_poly_area(int n) {
    if (n <= 0) return M_PI;
    return 0.5 * n * sin(2.0 * M_PI / n);
}

void or_aperture_point(int n, double u1, double u2, double out[2]) {
    if (n <= 0) {
        double r = sqrt(u1), phi = 2.0 * M_PI * u2;
        out[0] = r * cos(phi);
        out[1] = r * sin(phi);
        return;
    }
    double a = u2 * n;
    int k = (int)floor(a);
    if (k > n - 1) k = n - 1;
    double t = a - k, r = sqrt(u1);
    double t0 = 2.0 * M_PI * k / n, t1 = 2.0 * M_PI * (k + 1) / n;
    out[0] = r * ((1.0 - t) * cos(t0) + t * cos(t1));
    out[1] = r * ((1.0 - t) * sin(t0) + t * sin(t1));
}

/* Distributed ray of Cook et al. for the half-resolution pixel (i, j) and lens
 * sample `sample` (Section 3.2.2): the pixel's direction through the lens centre
 * meets the focus plane z = d at P_f; a point L on the lens disk (radius a/2) is
 * drawn from Philox keyed on (seed, session) with counter (pixel, sample, frame, 0);
 * the ray runs from L towards P_f.  Lens point: (a/2) or_aperture_point of two 24-bit
 * uniforms, the polar map r = sqrt(u1), phi = 2 pi u2 for the circular aperture (the
 * paper only says "within a circle"). */
void or_lens_ray(const OrCamera *c, const OrParams *p, int W, int H, int i, int j, int sample,
                 double o[3], double d[3]) {
    int W2 = W / 2;
    double dp[3];
    or_pixel_dir(c, W, H, 2.0 * i + 1.0, 2.0 * j + 1.0, dp);
    double tf = c->d / dot3(dp, c->F);
    double Pf[3] = {c->O[0] + tf * dp[0], c->O[1] + tf * dp[1], c->O[2] + tf * dp[2]};
    uint64_t ctr[4] = {(uint64_t)j * (uint64_t)W2 + (uint64_t)i, (uint64_t)sample,
                       (uint64_t)c->frame, 0};
    uint64_t key[2] = {p->seed, p->session}, x[4];
    or_philox4x64(ctr, key, x);
    double u1 = (double)(x[0] >> 40) * (1.0 / 16777216.0);
    double u2 = (double)(x[1] >> 40) * (1.0 / 16777216.0);
    double a = c->f / c->N, pt[2];
    or_aperture_point((int)p->blades, u1, u2, pt);
    double lx = 0.5 * a * pt[0], ly = 0.5 * a * pt[1];
    for (int k = 0; k < 3; k++) o[k] = c->O[k] + lx * c->R[k] + ly * c->U[k];
    sub3(Pf, o, d);
    normalize3(d);
}

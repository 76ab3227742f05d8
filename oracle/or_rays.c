/* Ray mask (Section 3.2.1, Eq. 2-4) and the ray-traced layer (Section 3.2.2) of
 * the oracle.  Test infrastructure (see oracle.h). */
#include "or_internal.h"

void or_binomial5(const double *src, int w, int h, int C, double *dst);
void or_sobel5(const double *src, int w, int h, int C, int ci, double *gx, double *gy);

/* ---- A6: ray mask and ray count -------------------------------------------- */

/* Edge measure (Eq. 2, Eq. 3): the half-resolution depth and normals are blurred
 * (5x5 binomial, standing in for the Gaussian), then a 5x5 Sobel gives the depth
 * derivative delta_d (relative: |grad z| / z) and the normal derivative delta_n
 * (Frobenius norm over the three components); x = (delta_d + delta_n) s and
 * x_n = saturate(1 - 1/(x + 1)).  Ray count (Eq. 4): x_f = saturate(x_n +
 * sigma^2 * 1e5) * m, rounded up, at least one ray and at most m.
 *
 * Mask: a pixel gets rays when the dilated max near-CoC radius of its tile is at
 * least mask_near_hpx, i.e. when a blurred foreground object can reach it ("at
 * least one ray per pixel in the near field", scaled by the neighbourhood max CoC
 * as Section 5.3 proposes).  Fixed mode shoots spp rays per masked pixel. */
void or_mask(const OrParams *p, int W2, int H2, const double *z_h, const double *n_h,
             const double *dil, const double *var_prev, double *xn, double *xf, int32_t *nrays) {
    size_t N = (size_t)W2 * H2;
    double *gz = (double *)malloc(sizeof(double) * N);
    double *gn = (double *)malloc(sizeof(double) * N * 3);
    double *gx = (double *)malloc(sizeof(double) * N);
    double *gy = (double *)malloc(sizeof(double) * N);
    double *dn2 = (double *)calloc(N, sizeof(double));
    or_binomial5(z_h, W2, H2, 1, gz);
    or_binomial5(n_h, W2, H2, 3, gn);
    for (int c = 0; c < 3; c++) {
        or_sobel5(gn, W2, H2, 3, c, gx, gy);
        for (size_t q = 0; q < N; q++) dn2[q] += gx[q] * gx[q] + gy[q] * gy[q];
    }
    or_sobel5(gz, W2, H2, 1, 0, gx, gy);
    int T = p->tile, TW = (W2 + T - 1) / T;
    for (int j = 0; j < H2; j++)
        for (int i = 0; i < W2; i++) {
            size_t q = (size_t)j * W2 + i;
            double dd = sqrt(gx[q] * gx[q] + gy[q] * gy[q]) / gz[q];
            double x = (dd + sqrt(dn2[q])) * p->s;
            double x_n = saturate(1.0 - 1.0 / (x + 1.0));
            double sig2 = var_prev ? var_prev[q] : 0.0;
            double x_f = saturate(x_n + sig2 * p->var_w_mask) * p->m;
            xn[q] = x_n;
            xf[q] = x_f;
            double near_max = dil[2 * ((size_t)(j / T) * TW + (i / T))];
            int n = 0;
            if (near_max >= p->mask_near_hpx) {
                if (p->ray_mode == 0) n = p->spp;
                else n = (int)clampd(ceil(x_f), 1.0, p->m);
            }
            nrays[q] = n;
        }
    free(gz); free(gn); free(gx); free(gy); free(dn2);
}

/* ---- A8: rays, hits, shading, per-pixel near/far split --------------------- */

/* For each masked half-resolution pixel, its n rays (or_lens_ray) are traced to
 * the closest hit and shaded; a miss sees the sky at depth z_far.  Each ray's
 * colour is split between the fields by its distance to the focus plane
 * (Section 3.2.2) with the near weight w = saturate(-c(z_hit) / sqrt(2)): 1 for an
 * out-of-focus near hit, 0 behind the focus plane, a linear ramp across the near
 * half of the zone of focus.  Reduced over the pixel's rays in sample order:
 *   h  = sum w / n                                  (hit ratio)
 *   An = sum w col / n,  Af = sum (1-w) col / n     (premultiplied field colours)
 *   Bn = sum w |rho| / n, Bf = sum (1-w) |rho| / n  (premultiplied field CoCs)
 *   Pfar = sum (1-w) P / Fw, Fw = sum (1-w)  (mean far position: the hit point, or
 *   for a ray that hits nothing its point at depth z_far)
 * Layout of rt per pixel: n, h, An(3), Af(3), Bn, Bf, Pfar(3), Fw. */
void or_trace(const OrScene *s, const OrCamera *c, const OrParams *p, int W, int H,
              const int32_t *nrays, double *rt, int32_t *ray_prim, double *ray_c, int max_rays,
              const int32_t *hit_force) {
    int W2 = W / 2, H2 = H / 2;
    double rmax = 0.5 * p->max_coc_px;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < H2; j++)
        for (int i = 0; i < W2; i++) {
            size_t q = (size_t)j * W2 + i;
            double *o = rt + 14 * q;
            for (int k = 0; k < 14; k++) o[k] = 0.0;
            int n = nrays[q];
            if (n <= 0) continue;
            double Sw = 0, An[3] = {0, 0, 0}, Af[3] = {0, 0, 0}, Bn = 0, Bf = 0;
            double Pf[3] = {0, 0, 0}, Fw = 0;
            for (int smp = 0; smp < n; smp++) {
                double ro[3], rd[3], col[3], nrm[3], t = 0.0, z;
                or_lens_ray(c, p, W, H, i, j, smp, ro, rd);
                int forced = hit_force && smp < max_rays ? hit_force[q * max_rays + smp] : -2;
                int hit;
                if (forced >= -1 && forced < or_scene_ntris(s)) {
                    hit = forced;
                    if (hit >= 0) t = or_plane_t(s, hit, ro, rd);
                } else {
                    hit = or_closest(s, ro, rd, &t);
                }
                if (hit >= 0) {
                    or_shade(s, p, hit, ro, rd, t, col, nrm);
                    z = fmin(t * dot3(rd, c->F), p->z_far);
                } else {
                    for (int k = 0; k < 3; k++) col[k] = p->sky[k];
                    z = p->z_far;
                }
                double cz = or_coc(c, W, z);
                double rho = fabs(clampd(cz / 4.0, -rmax, rmax));
                double w = saturate(-cz / sqrt(2.0));
                if (ray_prim && smp < max_rays) ray_prim[q * max_rays + smp] = hit;
                if (ray_c && smp < max_rays) ray_c[q * max_rays + smp] = cz;
                Sw += w;
                for (int k = 0; k < 3; k++) {
                    An[k] += w * col[k];
                    Af[k] += (1.0 - w) * col[k];
                }
                Bn += w * rho;
                Bf += (1.0 - w) * rho;
                /* far position: the hit, or for a ray that escapes, its point at depth z_far
                 * (the sky is a finite depth, so its reprojection follows the ray) */
                double tf = hit >= 0 ? t : p->z_far / dot3(rd, c->F);
                for (int k = 0; k < 3; k++) Pf[k] += (1.0 - w) * (ro[k] + tf * rd[k]);
                Fw += 1.0 - w;
            }
            o[0] = n;
            o[1] = Sw / n;
            for (int k = 0; k < 3; k++) {
                o[2 + k] = An[k] / n;
                o[5 + k] = Af[k] / n;
                o[10 + k] = Fw > 0.0 ? Pf[k] / Fw : 0.0;
            }
            o[8] = Bn / n;
            o[9] = Bf / n;
            o[13] = Fw;
        }
}

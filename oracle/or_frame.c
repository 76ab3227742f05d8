/* One frame of the hybrid depth-of-field pass in the oracle, in the paper's order
 * (Fig. 1, Section 3): post-process chain, ray mask, ray tracing, accumulation,
 * variance blur, median, reconstruction, composite.  Test infrastructure (see
 * oracle.h). */
#include "or_internal.h"
#include <omp.h>

void or_downscale(const OrCamera *cam, const OrParams *p, int W, int H, const float *color4,
                  const float *depth, const float *normal4, double *pp_in, double *z_h,
                  double *n_h);
void or_tile_max(const OrParams *p, int W2, int H2, const double *pp_in, double *tiles);
void or_tile_dilate(const OrParams *p, int W2, int H2, const double *tiles, double *dil);
void or_prefilter(const OrParams *p, int W2, int H2, const double *pp_in, const double *dil,
                  double *pre);
void or_main_filter(const OrParams *p, int W2, int H2, const double *pre, const double *z_h,
                    const double *dil, double *out);
void or_median3x3(int W2, int H2, const double *src, double *dst);
void or_mask(const OrParams *p, int W2, int H2, const double *z_h, const double *n_h,
             const double *dil, const double *var_prev, double *xn, double *xf, int32_t *nrays);
void or_trace(const OrScene *s, const OrCamera *c, const OrParams *p, int W, int H,
              const int32_t *nrays, double *rt, int32_t *ray_prim, double *ray_c, int max_rays,
              const int32_t *hit_force);
void or_accumulate(const OrCamera *c, const OrParams *p, int W, int H, const double *z_h,
                   const double *rt, const int32_t *nrays, const double *hist_in, int has_history,
                   double *hist_out, double *crt, double *ct, double *var);
void or_median_rt(int W2, int H2, const double *crt, const int32_t *nrays, double *dst);
void or_recon(const OrParams *p, int W2, int H2, const double *med, const double *ct,
              const double *var_blur, const int32_t *nrays, double *out);
void or_composite(const OrCamera *cam, const OrParams *p, int W, int H, const float *color4,
                  const float *depth, const double *pp_med, const double *recon,
                  const int32_t *nrays, double *out);

/* returns 0, or -1 for an invalid size */
int or_frame(const OrScene *s, const OrCamera *c, const OrParams *p, int W, int H,
             const float *color4, const float *depth, const float *normal4, OrFrame *fr) {
    if (W < 2 || H < 2 || (W & 1) || (H & 1)) return -1;
    int W2 = W / 2, H2 = H / 2;
    /* post-process (Section 3.1) */
    or_downscale(c, p, W, H, color4, depth, normal4, fr->pp_in, fr->z_h, fr->n_h);
    or_tile_max(p, W2, H2, fr->pp_in, fr->tile_raw);
    or_tile_dilate(p, W2, H2, fr->tile_raw, fr->tile_dil);
    or_prefilter(p, W2, H2, fr->pp_in, fr->tile_dil, fr->pre);
    or_main_filter(p, W2, H2, fr->pre, fr->z_h, fr->tile_dil, fr->main_out);
    or_median3x3(W2, H2, fr->main_out, fr->pp_med);
    /* ray mask (Section 3.2.1) */
    or_mask(p, W2, H2, fr->z_h, fr->n_h, fr->tile_dil, fr->has_history ? fr->var_in : NULL,
            fr->xn, fr->xf, fr->nrays);
    if (fr->nrays_force) {
        int cap = p->ray_mode == 0 ? p->spp : (int)p->m;
        for (size_t q = 0; q < (size_t)W2 * H2; q++)
            if (fr->nrays_force[q] >= 0) fr->nrays[q] = fr->nrays_force[q] < cap ? fr->nrays_force[q] : cap;
    }
    /* ray tracing (Section 3.2.2) */
    or_trace(s, c, p, W, H, fr->nrays, fr->rt, fr->ray_prim, fr->ray_c, fr->max_rays, fr->ray_hit_force);
    /* accumulation, reprojection and variance (Section 3.2.3) */
    or_accumulate(c, p, W, H, fr->z_h, fr->rt, fr->nrays, fr->hist_in, fr->has_history,
                  fr->hist_out, fr->crt, fr->ct, fr->var);
    or_binomial5(fr->var, W2, H2, 1, fr->var_out);
    /* median and spatial reconstruction (Section 3.2.4) */
    or_median_rt(W2, H2, fr->crt, fr->nrays, fr->rt_med);
    or_recon(p, W2, H2, fr->rt_med, fr->ct, fr->var_out, fr->nrays, fr->recon);
    /* composite (Section 3.3) */
    or_composite(c, p, W, H, color4, depth, fr->pp_med, fr->recon, fr->nrays, fr->out);
    /* final TAA (Section 3.4) */
    if (p->taa_alpha > 0.0 && fr->taa_out)
        or_taa(c, p, W, H, depth, fr->out, fr->taa_in, fr->has_taa_history && fr->taa_in, fr->taa_out);
    return 0;
}

/* Threads of the OpenMP loops over image rows (results do not depend on it); returns
 * the previous count.  n <= 0 only queries. */
int or_set_threads(int n) {
    int prev = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return prev;
}

/*
 * FP64 CPU oracle of the hybrid depth-of-field pass (Tan et al., "A Hybrid System
 * for Real-Time Rendering of Depth of Field Effect in Games", arXiv 2210.06158).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA implementation;
 * only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code, header, table or constant with the CUDA path: every
 * step is restated here from the paper in plain, slow double-precision C, in the
 * order the paper describes it (Section 3, Fig. 1).  Where the paper is silent the
 * reading taken is stated beside the code.
 *
 * Conventions
 *   full-resolution image W x H (even), half resolution W2 x H2 = W/2 x H/2.
 *   Arrays are row-major, channel-interleaved doubles unless noted.
 *   Signed circle of confusion c: diameter in full-resolution pixels, negative in
 *   front of the focus plane (near field, Section 3 "Demarcation of near and far").
 *   rho: signed CoC radius in half-resolution pixels, clamped to +-max_coc_px/2.
 */
#ifndef DOF_ORACLE_H
#define DOF_ORACLE_H

#include <stdint.h>

typedef struct {
    double f, N, d, ws;                   /* focal length, f-number, focus distance, sensor width (m) */
    double O[3], R[3], U[3], F[3];        /* current lens centre and basis (right, up, forward) */
    double pO[3], pR[3], pU[3], pF[3];    /* previous frame's pose */
    int64_t frame;
    double jx, jy;                        /* this frame's sub-pixel jitter (full-res px) */
    double pjx, pjy;                      /* the previous frame's */
} OrCamera;

typedef struct {
    double s, var_w_mask, m;              /* Eq. 2 scale, Eq. 4 weight, ray budget m (Eq. 4) */
    int32_t spp, ray_mode;                /* fixed rays per masked pixel; 0 fixed / 1 adaptive */
    double depth_range;                   /* main-filter depth range (Section 4.2: 10 cm) */
    double alpha, alpha_motion;           /* EMA blend (Section 3.2.3) and its value in motion */
    double var_w_recon, b_max;            /* Eq. 5 */
    double h_edge;                        /* Eq. 7 */
    double lod_scale, lod_max;            /* Eq. 8 */
    double max_coc_px;                    /* CoC radius clamp, full-resolution px */
    double zof_ramp, cover_ramp;          /* continuous widths of the focus and coverage tests */
    double bright_lum, bright_ramp;       /* bright-bokeh luminance threshold and ramp */
    double mask_near_hpx;                 /* ray mask: dilated near radius threshold (hpx) */
    double z_far;                         /* depth that stands for "no geometry" */
    int32_t tile;                         /* tile size (hpx) of the max-CoC tiles */
    int32_t pad0;
    uint64_t seed, session;               /* Philox key */
    double light[3], k_a, k_d, sky[3], emit;
    uint32_t albedo_seed;
    int32_t pad1;
    double taa_alpha;                     /* final TAA blend of the current frame (0 = no TAA) */
    double blades;                        /* aperture: 0 = circle, n = 3..8 regular n-gon */
} OrParams;

typedef struct OrScene OrScene;

/* ---------------- polygonal aperture (or_camera.c) ----------------
 * Section 1.1: bokeh takes the aperture's shape, a polygon for an n-blade diaphragm;
 * Section 2.2: the method extends to such shapes by changing the shape of its
 * sampling kernel.  Reading: a regular n-gon inscribed in the circle the circular
 * aperture would have (circumradius 1 here, a vertex at angle 0); the lens samples
 * of the rays and the taps of the 81-tap kernels both take that shape, and
 * sampleAlpha divides by its area.  n = 0 is the circle. */
double or_poly_rho(int n, double th);     /* boundary radius in direction th (1 for n = 0) */
double or_poly_area(int n);               /* area (pi for n = 0) */
/* uniform point of the unit disk (n = 0: r = sqrt(u1), phi = 2 pi u2) or of the n-gon
 * (sector k = floor(n u2), position t = n u2 - k along its edge: sqrt(u1) ((1 - t) V_k
 * + t V_k+1), which is uniform over the triangle (0, V_k, V_k+1)) */
void or_aperture_point(int n, double u1, double u2, double out[2]);
/* tap t of the 81-tap kernel (centre, then rings k = 1..4 of 8k taps at angles
 * 2 pi m / (8k)): unit offset (x, y) on the circle (n = 0) or on the n-gon boundary
 * in the same direction, and the ring fraction k / 4 (or_post.c) */
void or_ring_tap(int n, int t, double out[3]);

/* ---------------- scene / rays (or_scene.c) ---------------- */
OrScene *or_scene_create(const float *xyz, int n_verts, const uint32_t *idx,
                         const uint32_t *mat, int n_tris);
void or_scene_destroy(OrScene *s);
int or_scene_depth(const OrScene *s);
int or_scene_ntris(const OrScene *s);
/* closest hit through the oracle's BVH; returns prim or -1; *t set on hit */
int or_closest(const OrScene *s, const double o[3], const double d[3], double *t);
/* closest hit by testing every triangle (no acceleration structure) */
int or_closest_brute(const OrScene *s, const double o[3], const double d[3], double *t);
/* Validity of a closest hit computed in lower precision (prim_k, -1 = none) against
 * the FP64 answer prim_o for the ray (o, d): 0 equal, 1..4 a valid rounding tie,
 * negative an invalid answer (codes in or_scene.c) */
int or_hit_check(const OrScene *s, const double o[3], const double d[3], int prim_k, int prim_o,
                 double rel_tol);
/* distance along (o, d) to the plane of triangle `prim` (+inf if parallel) */
double or_plane_t(const OrScene *s, int prim, const double o[3], const double d[3]);
void or_shade(const OrScene *s, const OrParams *p, int prim, const double o[3],
              const double d[3], double t, double col[3], double nrm[3]);
void or_albedo(uint32_t seed, int prim, double col[3]);
uint32_t or_fmix32(uint32_t h);

/* ---------------- camera / lens (or_camera.c) ---------------- */
double or_coc(const OrCamera *c, int W, double z);
void or_zof_bounds(const OrCamera *c, int W, double *z_near, double *z_far);
void or_pixel_dir(const OrCamera *c, int W, int H, double x, double y, double dir[3]);
void or_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
void or_lens_ray(const OrCamera *c, const OrParams *p, int W, int H, int i, int j, int sample,
                 double o[3], double d[3]);

/* ---------------- G-buffer producer (or_gbuffer.c) ---------------- */
void or_gbuffer(const OrScene *s, const OrCamera *c, const OrParams *p, int W, int H,
                double *color3, double *depth, double *normal3, int32_t *prim);

/* ---------------- one frame of the pass (or_frame.c) ---------------- */
typedef struct {
    /* half-resolution intermediates, W2*H2*channels */
    double *pp_in;      /* 4: rgb, rho      downscale (Section 3.1)            */
    double *z_h;        /* 1: depth (min of the 2x2, clamped to z_far)         */
    double *n_h;        /* 3: normal of the min-depth sample                    */
    double *tile_raw;   /* 2 per tile: max near radius, max |rho|              */
    double *tile_dil;   /* 2 per tile after neighbourhood dilation              */
    double *pre;        /* 4: prefiltered rgb, rho (Section 3.1.1)             */
    double *main_out;   /* 4: rgb, bright fraction (Eq. 1)                      */
    double *pp_med;     /* 4: median postfilter (Section 3.1.3)                 */
    double *xn;         /* 1: Eq. 3 edge measure                               */
    double *xf;         /* 1: Eq. 4 ray count before rounding                  */
    int32_t *nrays;     /* 1: rays shot for the pixel                          */
    int32_t *ray_prim;  /* W2*H2*max_rays, -1 = miss (optional)                */
    double *ray_c;      /* W2*H2*max_rays signed CoC of the ray's hit (optional) */
    double *rt;         /* 14: n, h, An(3), Af(3), Bn, Bf, Pfar(3), Fw         */
    double *crt;        /* 4: merged ray-traced rgb, hit ratio                  */
    double *ct;         /* 1: accumulated CoC radius (hpx)                      */
    double *var;        /* 1: luminance variance                                */
    double *rt_med;     /* 4: median of crt rgb, h copied                       */
    double *recon;      /* 4: reconstructed rgb, h (Eq. 5, Eq. 8)               */
    double *out;        /* W*H*4 final image (Eq. 6, Eq. 7)                    */
    const double *hist_in;  /* 12 per hpx: An(3) Af(3) h g Bn Bf mu1 mu2        */
    double *hist_out;
    const double *var_in;   /* blurred variance of the previous frame          */
    double *var_out;        /* blurred variance of this frame                  */
    int32_t has_history;
    int32_t max_rays;       /* stride of ray_prim / ray_c                       */
    /* optional (tests): per hpx, a ray count to use instead of the mask's where >= 0.
     * Where x_f (Eq. 4) lies on an integer, or a tile's dilated near radius on the
     * mask threshold, the count is decided by rounding and either neighbour is a valid
     * result; a test passes the other side's count there so the rest of the frame can
     * be compared.  NULL: the mask's counts. */
    const int32_t *nrays_force;
    /* optional (tests): per ray (W2*H2*max_rays), the triangle id to take as the ray's
     * hit where >= -1 (-1 = a miss), at the distance to its plane.  Where a ray passes
     * within rounding of a shared edge, or two triangles at equal depth, either answer
     * is a valid closest hit; a test passes the other side's answer there.  NULL: the
     * closest hit. */
    const int32_t *ray_hit_force;
    /* final TAA (Section 3.4), when taa_alpha > 0: W*H*4 resolved image of the previous
     * frame (history) and of this one */
    const double *taa_in;
    double *taa_out;
    int32_t has_taa_history;
    int32_t pad_taa;
} OrFrame;

/* OpenMP threads of the row loops (output independent of it); returns the previous
 * count, n <= 0 only queries */
int or_set_threads(int n);
int or_frame(const OrScene *s, const OrCamera *c, const OrParams *p, int W, int H,
             const float *color4, const float *depth, const float *normal4, OrFrame *fr);

/* Final TAA of the composited image (Section 3.4; Karis 2014) */
void or_taa(const OrCamera *c, const OrParams *p, int W, int H, const float *depth, const double *cur,
            const double *hist_in, int has_history, double *out);

/* individual steps, exposed for the pins */
void or_median9(const double v[9], int k, double *out);
void or_binomial5(const double *src, int w, int h, int C, double *dst);
void or_sobel5(const double *src, int w, int h, int C, int ci, double *gx, double *gy);

#endif

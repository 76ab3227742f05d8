/* G-buffer producer of the oracle (Section 3: deferred shading produces depth,
 * normals and the sharp all-in-focus image).  A pinhole primary ray through each
 * full-resolution pixel centre stands in for the rasteriser.  Test infrastructure
 * (see oracle.h). */
#include "or_internal.h"

/* Outputs per pixel: colour (3), linear depth along the optical axis (+inf on a
 * miss), the hit's face normal turned towards the camera (0 on a miss), and the
 * triangle id (-1 on a miss).  Misses see the constant sky colour. */
void or_gbuffer(const OrScene *s, const OrCamera *c, const OrParams *p, int W, int H,
                double *color3, double *depth, double *normal3, int32_t *prim) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < H; j++) {
        for (int i = 0; i < W; i++) {
            size_t q = (size_t)j * W + i;
            double d[3];
            or_pixel_dir(c, W, H, i + 0.5, j + 0.5, d);
            double t = 0.0;
            int hit = or_closest(s, c->O, d, &t);
            prim[q] = hit;
            if (hit < 0) {
                for (int k = 0; k < 3; k++) {
                    color3[3 * q + k] = p->sky[k];
                    normal3[3 * q + k] = 0.0;
                }
                depth[q] = INFINITY;
                continue;
            }
            double col[3], n[3];
            or_shade(s, p, hit, c->O, d, t, col, n);
            for (int k = 0; k < 3; k++) {
                color3[3 * q + k] = col[k];
                normal3[3 * q + k] = n[k];
            }
            depth[q] = t * dot3(d, c->F);
        }
    }
}

/* Small double-precision helpers shared by the oracle's translation units.
 * Test infrastructure: see oracle.h. */
#ifndef DOF_OR_INTERNAL_H
#define DOF_OR_INTERNAL_H

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static inline double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static inline void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline void sub3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static inline void normalize3(double v[3]) {
    double n = sqrt(dot3(v, v));
    v[0] /= n; v[1] /= n; v[2] /= n;
}
static inline double saturate(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }
static inline double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static inline int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }
static inline double lerp(double a, double b, double t) { return a + t * (b - a); }
/* textbook smoothstep: Hermite 3t^2 - 2t^3 on t = saturate((x-e0)/(e1-e0)) */
static inline double smoothstep(double e0, double e1, double x) {
    double t = saturate((x - e0) / (e1 - e0));
    return t * t * (3.0 - 2.0 * t);
}
/* Rec. 709 luminance */
static inline double luminance(const double c[3]) {
    return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2];
}

/* Bilinear sample of a w x h image with C interleaved channels at continuous
 * coordinates (x, y), where integer coordinates are texel centres.  Indices are
 * clamped to the image (clamp-to-edge).  Every channel gets the same weights. */
static inline void bilinear_clamped(const double *img, int w, int h, int C, double x, double y,
                                    double *out) {
    double x0f = floor(x), y0f = floor(y);
    double fx = x - x0f, fy = y - y0f;
    int x0 = (int)x0f, y0 = (int)y0f;
    for (int c = 0; c < C; c++) out[c] = 0.0;
    for (int dy = 0; dy < 2; dy++) {
        for (int dx = 0; dx < 2; dx++) {
            double wgt = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy);
            int xi = clampi(x0 + dx, 0, w - 1), yi = clampi(y0 + dy, 0, h - 1);
            const double *t = img + ((size_t)yi * w + xi) * C;
            for (int c = 0; c < C; c++) out[c] += wgt * t[c];
        }
    }
}

#endif

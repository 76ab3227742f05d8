/* Scene, closest-hit queries and shading of the oracle.  Test infrastructure (see
 * oracle.h).
 *
 * The oracle's acceleration structure is a plain top-down BVH (median split of the
 * centroids along the longest axis, leaves of at most 4 triangles), independent of
 * the device's LBVH.  Any valid BVH gives the same closest hit when no box with
 * an entry distance equal to the best hit is culled, which is checked against the
 * all-triangle loop `or_closest_brute`. */
#include "or_internal.h"

typedef struct {
    double lo[3], hi[3];
    int left, right;      /* children (internal), -1 for a leaf */
    int first, count;     /* leaf range in prim_order */
} OrNode;

struct OrScene {
    int n;
    double *v;            /* 9 per triangle */
    uint32_t *mat;
    int *order;           /* triangle ids in leaf order */
    OrNode *nodes;
    int n_nodes, depth;
};

typedef struct { double key; int id; } KeyId;

static int cmp_keyid(const void *a, const void *b) {
    const KeyId *x = (const KeyId *)a, *y = (const KeyId *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

static void tri_bounds(const OrScene *s, int t, double lo[3], double hi[3]) {
    const double *v = s->v + 9 * (size_t)t;
    for (int k = 0; k < 3; k++) {
        lo[k] = fmin(v[k], fmin(v[3 + k], v[6 + k]));
        hi[k] = fmax(v[k], fmax(v[3 + k], v[6 + k]));
    }
}

static int build(OrScene *s, KeyId *tmp, int first, int count, int depth) {
    int me = s->n_nodes++;
    OrNode *nd = &s->nodes[me];
    if (depth > s->depth) s->depth = depth;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = first; i < first + count; i++) {
        double a[3], b[3];
        tri_bounds(s, s->order[i], a, b);
        for (int k = 0; k < 3; k++) {
            lo[k] = fmin(lo[k], a[k]); hi[k] = fmax(hi[k], b[k]);
            double cen = 0.5 * (a[k] + b[k]);
            clo[k] = fmin(clo[k], cen); chi[k] = fmax(chi[k], cen);
        }
    }
    /* pad by a relative epsilon so that rounding in the slab test never culls a
     * triangle whose hit lies on the box surface */
    for (int k = 0; k < 3; k++) {
        double e = 1e-9 * (fabs(lo[k]) + fabs(hi[k]) + 1.0);
        nd->lo[k] = lo[k] - e; nd->hi[k] = hi[k] + e;
    }
    if (count <= 4) {
        nd->left = nd->right = -1; nd->first = first; nd->count = count;
        return me;
    }
    int axis = 0;
    for (int k = 1; k < 3; k++) if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
    for (int i = 0; i < count; i++) {
        double a[3], b[3];
        int t = s->order[first + i];
        tri_bounds(s, t, a, b);
        tmp[i].key = 0.5 * (a[axis] + b[axis]);
        tmp[i].id = t;
    }
    qsort(tmp, (size_t)count, sizeof(KeyId), cmp_keyid);
    for (int i = 0; i < count; i++) s->order[first + i] = tmp[i].id;
    int half = count / 2;
    nd->first = first; nd->count = 0;
    int l = build(s, tmp, first, half, depth + 1);
    int r = build(s, tmp, first + half, count - half, depth + 1);
    s->nodes[me].left = l; s->nodes[me].right = r;
    return me;
}

OrScene *or_scene_create(const float *xyz, int n_verts, const uint32_t *idx,
                         const uint32_t *mat, int n_tris) {
    (void)n_verts;
    OrScene *s = (OrScene *)calloc(1, sizeof(OrScene));
    s->n = n_tris;
    s->v = (double *)malloc(sizeof(double) * 9 * (size_t)(n_tris > 0 ? n_tris : 1));
    s->mat = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n_tris > 0 ? n_tris : 1));
    for (int t = 0; t < n_tris; t++) {
        for (int c = 0; c < 3; c++)
            for (int k = 0; k < 3; k++)
                s->v[9 * (size_t)t + 3 * c + k] = (double)xyz[3 * (size_t)idx[3 * (size_t)t + c] + k];
        s->mat[t] = mat[t];
    }
    s->order = (int *)malloc(sizeof(int) * (size_t)(n_tris > 0 ? n_tris : 1));
    for (int t = 0; t < n_tris; t++) s->order[t] = t;
    s->nodes = (OrNode *)malloc(sizeof(OrNode) * (size_t)(2 * n_tris + 1));
    s->n_nodes = 0;
    if (n_tris > 0) {
        KeyId *tmp = (KeyId *)malloc(sizeof(KeyId) * (size_t)n_tris);
        build(s, tmp, 0, n_tris, 1);
        free(tmp);
    }
    return s;
}

void or_scene_destroy(OrScene *s) {
    if (!s) return;
    free(s->v); free(s->mat); free(s->order); free(s->nodes); free(s);
}

int or_scene_depth(const OrScene *s) { return s->depth; }
int or_scene_ntris(const OrScene *s) { return s->n; }

/* Moller-Trumbore ray/triangle test in double precision; edges count as inside.
 * Returns 1 and the distance t > 0 on a hit. */
static int tri_hit(const double *v, const double o[3], const double d[3], double *t) {
    double e1[3], e2[3], pv[3], tv[3], qv[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(d, e2, pv);
    double det = dot3(e1, pv);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    sub3(o, v, tv);
    double u = dot3(tv, pv) * inv;
    if (u < 0.0 || u > 1.0) return 0;
    cross3(tv, e1, qv);
    double w = dot3(d, qv) * inv;
    if (w < 0.0 || u + w > 1.0) return 0;
    double tt = dot3(e2, qv) * inv;
    if (!(tt > 0.0)) return 0;
    *t = tt;
    return 1;
}

/* closest hit = lexicographic minimum of (t, triangle id) over t > 0 */
static void consider(const OrScene *s, int tri, const double o[3], const double d[3],
                     double *best_t, int *best) {
    double t;
    if (tri_hit(s->v + 9 * (size_t)tri, o, d, &t)) {
        if (t < *best_t || (t == *best_t && tri < *best)) { *best_t = t; *best = tri; }
    }
}

int or_closest_brute(const OrScene *s, const double o[3], const double d[3], double *t) {
    double best_t = INFINITY;
    int best = -1;
    for (int i = 0; i < s->n; i++) consider(s, i, o, d, &best_t, &best);
    if (best >= 0) *t = best_t;
    return best;
}

/* slab test; a box whose entry distance equals the best hit is still visited */
static int box_hit(const OrNode *nd, const double o[3], const double d[3], double best_t) {
    double tmin = 0.0, tmax = best_t;
    for (int k = 0; k < 3; k++) {
        if (d[k] == 0.0) {
            if (o[k] < nd->lo[k] || o[k] > nd->hi[k]) return 0;
            continue;
        }
        double t1 = (nd->lo[k] - o[k]) / d[k], t2 = (nd->hi[k] - o[k]) / d[k];
        tmin = fmax(tmin, fmin(t1, t2));
        tmax = fmin(tmax, fmax(t1, t2));
    }
    return tmin <= tmax;
}

int or_closest(const OrScene *s, const double o[3], const double d[3], double *t) {
    if (s->n == 0) return -1;
    double best_t = INFINITY;
    int best = -1;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const OrNode *nd = &s->nodes[stack[--sp]];
        if (!box_hit(nd, o, d, best_t)) continue;
        if (nd->left < 0) {
            for (int i = nd->first; i < nd->first + nd->count; i++)
                consider(s, s->order[i], o, d, &best_t, &best);
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    if (best >= 0) *t = best_t;
    return best;
}

double or_plane_t(const OrScene *s, int prim, const double o[3], const double d[3]) {
    const double *v = s->v + 9 * (size_t)prim;
    double e1[3], e2[3], n[3], tv[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(e1, e2, n);
    double dn = dot3(d, n);
    if (dn == 0.0) return INFINITY;
    sub3(v, o, tv);
    return dot3(tv, n) / dn;
}

/* ---- validity of a closest-hit answer computed in lower precision ------------
 *
 * A ray traced in FP32 may disagree with the FP64 closest hit only where rounding
 * can change the answer: where the ray passes within rounding distance of a
 * triangle's boundary (it may be counted inside or outside), or where two hits lie
 * at distances that rounding cannot order.  The rounding of a ray made in FP32 moves
 * it sideways by a distance proportional to |o| + s at ray parameter s, so "within
 * rounding" is measured as the distance between the ray and each edge segment of the
 * triangle, against rel_tol * (|o| + s).  The hit distance of a triangle the ray meets
 * at incidence cos = |d.n| is uncertain by that sideways tolerance over cos. */

enum { PROBE_MISS = 0, PROBE_GRAZED = 1, PROBE_CLEAN = 2 };
typedef struct { int state; double t, dt; } TriProbe;

/* Closest approach of the ray o + s d (s >= 0, |d| = 1) to the segment A + u e,
 * u in [0, 1]: returns the distance and the ray parameter s there. */
static double ray_segment(const double o[3], const double d[3], const double A[3], const double e[3],
                          double *s_out) {
    double w0[3];
    sub3(o, A, w0);
    double b = dot3(d, e), c = dot3(e, e), dd = dot3(d, w0), ee = dot3(e, w0);
    double u, sp;
    double den = c - b * b;            /* |e|^2 sin^2 of the angle between ray and edge */
    if (c <= 0.0) {
        u = 0.0;                        /* the edge is a point */
    } else if (den > 1e-14 * c) {
        u = (ee - dd * b) / den;
    } else {
        u = ee / c;                     /* parallel: the point of the edge nearest to o */
    }
    if (u < 0.0) u = 0.0;
    if (u > 1.0) u = 1.0;
    sp = u * b - dd;                    /* the ray's point nearest to A + u e */
    if (sp < 0.0) {                     /* behind the origin: nearest point of the edge to o */
        sp = 0.0;
        u = c > 0.0 ? ee / c : 0.0;     /* (o - A).e / |e|^2 */
        if (u < 0.0) u = 0.0;
        if (u > 1.0) u = 1.0;
    }
    double r[3];
    for (int k = 0; k < 3; k++) r[k] = w0[k] + sp * d[k] - u * e[k];
    *s_out = sp;
    return sqrt(dot3(r, r));
}

/* Classifies triangle prim for the ray (o, d), |d| = 1:
 *   CLEAN   the FP64 test hits it and the ray stays clear of its edges by more than
 *           the tolerance (a lower-precision test must hit it too);
 *   GRAZED  the ray passes within the tolerance of an edge segment, in front of the
 *           origin (a lower-precision test may hit or miss it);
 *   MISS    neither (no test within rounding hits it).
 * t is the hit distance (FP64 hit, else the plane's distance, else the ray parameter
 * of the closest approach to the edge) and dt its uncertainty. */
static TriProbe probe(const OrScene *s, int prim, const double o[3], const double d[3], double rel_tol) {
    const double *v = s->v + 9 * (size_t)prim;
    TriProbe r = {PROBE_MISS, INFINITY, 0.0};
    double on = sqrt(dot3(o, o));
    double best_gap = INFINITY, s_best = 0.0;
    int grazed = 0;
    for (int e = 0; e < 3; e++) {
        const double *A = v + 3 * e, *B = v + 3 * ((e + 1) % 3);
        double ab[3], se;
        sub3(B, A, ab);
        double dist = ray_segment(o, d, A, ab, &se);
        double tol = rel_tol * (on + se);
        if (dist <= tol) grazed = 1;
        if (dist - tol < best_gap) { best_gap = dist - tol; s_best = se; }
    }
    double e1[3], e2[3], n[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(e1, e2, n);
    double nn = sqrt(dot3(n, n));
    double cosi = nn > 0.0 ? fabs(dot3(d, n)) / nn : 0.0;
    double th;
    int hit = tri_hit(v, o, d, &th);
    double t;
    if (hit) t = th;
    else if (nn > 0.0 && cosi > 1e-9) t = or_plane_t(s, prim, o, d);
    else t = s_best;
    double tol_t = rel_tol * (on + fabs(t));
    double dt = tol_t / fmax(cosi, 1e-12) + tol_t;
    if (hit && !grazed) { r.state = PROBE_CLEAN; r.t = t; r.dt = dt; return r; }
    if (grazed && t > -dt) { r.state = PROBE_GRAZED; r.t = t; r.dt = dt; return r; }
    return r;
}

/* Is there a CLEAN hit whose whole uncertainty interval lies before t_lim? */
static int clean_hit_before(const OrScene *s, const double o[3], const double d[3], double t_lim,
                            double rel_tol) {
    if (s->n == 0 || !(t_lim > 0.0)) return 0;
    int stack[256], sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const OrNode *nd = &s->nodes[stack[--sp]];
        if (!box_hit(nd, o, d, t_lim)) continue;
        if (nd->left < 0) {
            for (int i = nd->first; i < nd->first + nd->count; i++) {
                TriProbe p = probe(s, s->order[i], o, d, rel_tol);
                if (p.state == PROBE_CLEAN && p.t + p.dt < t_lim) return 1;
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    return 0;
}

/* Is prim_k (a closest hit computed in lower precision; -1 = no hit) a valid answer
 * for the ray (o, d), given the FP64 answer prim_o?  The answer is valid when rounding
 * can explain the difference: the kernel's triangle is hit within rounding (CLEAN or
 * GRAZED), no CLEAN hit lies certainly in front of it, and, when it is CLEAN, the
 * FP64 answer does not lie certainly behind it.  Returns
 *    0  the ids agree
 *    1  depth tie: both hits clean, at distances rounding cannot order
 *    2  the FP64 hit is grazed (the kernel may miss it and see what lies behind)
 *    3  the kernel's triangle is grazed (it may count a hit the FP64 test misses)
 *    4  the kernel reports no hit and every hit along the ray is grazed
 *   -1  the kernel's triangle is not hit within rounding
 *   -2  a clean hit lies certainly in front of the kernel's answer
 *   -3  the kernel's hit is clean and the FP64 answer lies certainly behind it
 *       (or is a miss) */
int or_hit_check(const OrScene *s, const double o_in[3], const double d_in[3], int prim_k, int prim_o,
                 double rel_tol) {
    if (prim_k == prim_o) return 0;
    double o[3] = {o_in[0], o_in[1], o_in[2]}, d[3] = {d_in[0], d_in[1], d_in[2]};
    normalize3(d);
    TriProbe K = {PROBE_MISS, INFINITY, 0.0};
    if (prim_k >= 0) {
        if (prim_k >= s->n) return -1;
        K = probe(s, prim_k, o, d, rel_tol);
        if (K.state == PROBE_MISS) return -1;
    }
    double t_lim = prim_k >= 0 ? K.t - K.dt : INFINITY;
    if (clean_hit_before(s, o, d, t_lim, rel_tol)) return -2;
    if (prim_k < 0) return 4;
    if (K.state == PROBE_GRAZED) return 3;
    if (prim_o < 0 || prim_o >= s->n) return -3;
    TriProbe O = probe(s, prim_o, o, d, rel_tol);
    if (O.state == PROBE_MISS || O.t - O.dt > K.t + K.dt) return -3;
    return O.state == PROBE_CLEAN ? 1 : 2;
}

/* murmur3's 32-bit finaliser (Appleby): two xor-shift / multiply rounds and a last
 * xor-shift.  For an empty key, MurmurHash3_x86_32(seed) is exactly this of the seed. */
uint32_t or_fmix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85EBCA6BU; h ^= h >> 13; h *= 0xC2B2AE35U; h ^= h >> 16;
    return h;
}

/* Per-triangle albedo in [0.1, 0.9]^3 from an integer hash of (seed, triangle id):
 * the stand-in for the paper's scene materials. */
void or_albedo(uint32_t seed, int prim, double col[3]) {
    uint32_t base = or_fmix32(seed);
    for (int c = 0; c < 3; c++) {
        uint32_t h = or_fmix32(base ^ (uint32_t)(3 * prim + c));
        col[c] = 0.1 + 0.8 * ((double)(h >> 8) * (1.0 / 16777216.0));
    }
}

/* Deferred-shading colour of a hit (Section 3, Fig. 1): one directional light,
 * Lambert term on the face normal turned towards the ray, ambient k_a; material 1
 * is an emitter of radiance emit * albedo. */
void or_shade(const OrScene *s, const OrParams *p, int prim, const double o[3],
              const double d[3], double t, double col[3], double nrm[3]) {
    (void)o; (void)t;
    const double *v = s->v + 9 * (size_t)prim;
    double e1[3], e2[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(e1, e2, nrm);
    normalize3(nrm);
    if (dot3(nrm, d) > 0.0) { nrm[0] = -nrm[0]; nrm[1] = -nrm[1]; nrm[2] = -nrm[2]; }
    double alb[3];
    or_albedo(p->albedo_seed, prim, alb);
    if (s->mat[prim] == 1) {
        for (int c = 0; c < 3; c++) col[c] = p->emit * alb[c];
        return;
    }
    double l[3] = {p->light[0], p->light[1], p->light[2]};
    normalize3(l);
    double lam = -dot3(nrm, l);
    if (lam < 0.0) lam = 0.0;
    for (int c = 0; c < 3; c++) col[c] = alb[c] * (p->k_a + p->k_d * lam);
}

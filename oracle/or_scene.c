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

/* Is the disagreement "prim_a vs prim_b" for the ray (o, d) a floating-point near
 * tie?  Yes when the ray crosses the plane of either triangle within
 * rel_tol * (t + |o|) of that triangle's boundary (an edge graze, from inside or
 * outside) or runs nearly parallel to it, or when it passes inside both triangles
 * at relatively equal distance (a depth tie).  (The inner side of edge A->B is
 * where (B - A) x (P - A) points along the face normal.) */
static int graze(const OrScene *s, int prim, const double o[3], const double d[3], double rel_tol,
                 double *t_out, int *inside) {
    const double *v = s->v + 9 * (size_t)prim;
    double e1[3], e2[3], n[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(e1, e2, n);
    normalize3(n);
    double dn = dot3(d, n);
    *inside = 0;
    if (fabs(dn) < 1e-6) { *t_out = INFINITY; return 1; }
    double tv[3];
    sub3(v, o, tv);
    double t = dot3(tv, n) / dn;
    *t_out = t;
    double P[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
    double tol = rel_tol * (fabs(t) + sqrt(dot3(o, o)));
    int near_edge = 0, n_in = 0;
    for (int e = 0; e < 3; e++) {
        const double *A = v + 3 * e, *B = v + 3 * ((e + 1) % 3);
        double ab[3], ap[3], c[3];
        sub3(B, A, ab);
        sub3(P, A, ap);
        cross3(ab, ap, c);
        double sd = dot3(c, n) / sqrt(dot3(ab, ab));   /* > 0 on the inner side */
        if (fabs(sd) <= tol) near_edge = 1;
        if (sd >= 0.0) n_in++;
    }
    *inside = (n_in == 3) && t > 0.0;
    return near_edge;
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

int or_near_tie(const OrScene *s, const double o[3], const double d[3], int prim_a, int prim_b,
                double rel_tol) {
    if (prim_a == prim_b) return 1;
    double ta = INFINITY, tb = INFINITY;
    int ia = 0, ib = 0;
    int ga = prim_a >= 0 ? graze(s, prim_a, o, d, rel_tol, &ta, &ia) : 0;
    int gb = prim_b >= 0 ? graze(s, prim_b, o, d, rel_tol, &tb, &ib) : 0;
    if (ga || gb) return 1;
    if (ia && ib && fabs(ta - tb) <= rel_tol * fmax(fabs(ta), fabs(tb))) return 1;
    return 0;
}

/* murmur3's 32-bit finaliser (Appleby) */
static uint32_t fmix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85EBCA6BU; h ^= h >> 13; h *= 0xC2B2AE35U; h ^= h >> 16;
    return h;
}

/* Per-triangle albedo in [0.1, 0.9]^3 from an integer hash of (seed, triangle id):
 * the stand-in for the paper's scene materials. */
void or_albedo(uint32_t seed, int prim, double col[3]) {
    uint32_t base = fmix32(seed);
    for (int c = 0; c < 3; c++) {
        uint32_t h = fmix32(base ^ (uint32_t)(3 * prim + c));
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

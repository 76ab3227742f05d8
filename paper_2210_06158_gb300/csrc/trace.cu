// Ray side of libdof: G-buffer producer (pinhole primary visibility), ray mask with
// warp-aggregated compaction into a ray queue (Section 3.2.1, Eq. 2-4), and the
// persistent thin-lens ray kernels (Section 3.2.2): Philox lens samples, closest hit
// through the device BVH (one ray per lane, or the 32 rays of a warp as one packet),
// Lambert shading and the per-pixel near/far split.
#include "batch.cuh"
#include "geometry.cuh"

namespace {

constexpr int kStack = kTraversalStack;   // >= the tree depth (checked at upload)
constexpr int kTraceThreads = 128;        // threads of a tracer block (4 warps)

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC 2011); only the first two output words are used
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox2(unsigned long long c0, unsigned long long c1,
                                        unsigned long long c2, unsigned long long c3,
                                        unsigned long long k0, unsigned long long k1,
                                        unsigned long long &o0, unsigned long long &o1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += W0; k1 += W1; }
        unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        unsigned long long y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
        c0 = y0; c1 = lo1; c2 = y2; c3 = lo0;
    }
    o0 = c0; o1 = c1;
}

// slab test, one fused multiply-add per plane: the ray's outward-moved offsets cover
// the rounding of o * inv, and the relative slack on tmax the rest, so rounding never
// culls a hit on the surface
__device__ __forceinline__ bool box_hit(const Ray &r, float3 lo, float3 hi, float tbest, float &tent) {
    float tx0 = fmaf(lo.x, r.inv.x, -r.off0.x), tx1 = fmaf(hi.x, r.inv.x, -r.off1.x);
    float ty0 = fmaf(lo.y, r.inv.y, -r.off0.y), ty1 = fmaf(hi.y, r.inv.y, -r.off1.y);
    float tz0 = fmaf(lo.z, r.inv.z, -r.off0.z), tz1 = fmaf(hi.z, r.inv.z, -r.off1.z);
    float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tmax = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tbest));
    tent = tmin;
    return tmin <= tmax * 1.0000005f;
}

// The slab test for a ray of known octant: per axis the near plane is lo where inv >= 0
// and hi where inv < 0, so the near and far distances need no min/max.  With the
// offsets of make_ray (off0 for lo, off1 for hi) these are exactly the min and max
// that box_hit takes, so both tests give the same answer.
template <bool NX, bool NY, bool NZ>
__device__ __forceinline__ bool box_hit_o(const Ray &r, float3 lo, float3 hi, float tbest, float &tent) {
    const float nx = NX ? fmaf(hi.x, r.inv.x, -r.off1.x) : fmaf(lo.x, r.inv.x, -r.off0.x);
    const float fx = NX ? fmaf(lo.x, r.inv.x, -r.off0.x) : fmaf(hi.x, r.inv.x, -r.off1.x);
    const float ny = NY ? fmaf(hi.y, r.inv.y, -r.off1.y) : fmaf(lo.y, r.inv.y, -r.off0.y);
    const float fy = NY ? fmaf(lo.y, r.inv.y, -r.off0.y) : fmaf(hi.y, r.inv.y, -r.off1.y);
    const float nz = NZ ? fmaf(hi.z, r.inv.z, -r.off1.z) : fmaf(lo.z, r.inv.z, -r.off0.z);
    const float fz = NZ ? fmaf(lo.z, r.inv.z, -r.off0.z) : fmaf(hi.z, r.inv.z, -r.off1.z);
    const float tmin = fmaxf(fmaxf(nx, ny), fmaxf(nz, 0.f));
    const float tmax = fminf(fminf(fx, fy), fminf(fz, tbest));
    tent = tmin;
    return tmin <= tmax * 1.0000005f;
}

// both child boxes of a binary node, the octant's instance chosen by one multiway
// branch (uniform across a warp whose rays share the octant)
__device__ __forceinline__ void box_pair(const Ray &r, const float4 &a, const float4 &b, const float4 &c,
                                         float tbest, bool &h0, float &t0, bool &h1, float &t1) {
    const float3 lo0 = make_float3(a.x, a.y, a.z), hi0 = make_float3(a.w, b.x, b.y);
    const float3 lo1 = make_float3(b.z, b.w, c.x), hi1 = make_float3(c.y, c.z, c.w);
#define DOF_BOX_PAIR(X, Y, Z)                                   \
    {                                                           \
        h0 = box_hit_o<X, Y, Z>(r, lo0, hi0, tbest, t0);        \
        h1 = box_hit_o<X, Y, Z>(r, lo1, hi1, tbest, t1);        \
    }
    switch (r.oct & 7) {
    case 0: DOF_BOX_PAIR(false, false, false) break;
    case 1: DOF_BOX_PAIR(true, false, false) break;
    case 2: DOF_BOX_PAIR(false, true, false) break;
    case 3: DOF_BOX_PAIR(true, true, false) break;
    case 4: DOF_BOX_PAIR(false, false, true) break;
    case 5: DOF_BOX_PAIR(true, false, true) break;
    case 6: DOF_BOX_PAIR(false, true, true) break;
    default: DOF_BOX_PAIR(true, true, true) break;
    }
#undef DOF_BOX_PAIR
}

// the same slab test on one box of a 4-wide node (boxes stored per axis)
__device__ __forceinline__ bool box_hit_w(const Ray &r, float lx, float ly, float lz, float hx, float hy, float hz,
                                          float tbest, float &tent) {
    return box_hit(r, make_float3(lx, ly, lz), make_float3(hx, hy, hz), tbest, tent);
}



// ---------------------------------------------------------------------------
// 4-wide traversal step: the four child boxes of a node are tested at once and the
// children that are hit, internal nodes and leaves alike, are ordered by entry
// distance; the nearest is taken next and the others are pushed, farthest first.  A
// leaf reference taken from the stack is intersected.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cx_hit(float &ta, int &ra, float &tb, int &rb) {
    if (tb < ta) {
        float t = ta; ta = tb; tb = t;
        int r = ra; ra = rb; rb = r;
    }
}

__device__ __forceinline__ void tri_update(const Ray &ray, const float4 *__restrict__ tris, int k, HitRec &h) {
    const float4 *tp = tris + 3 * (size_t)k;
    float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
    float t = tri_hit(ray, v0, v1, v2, h.t);
    if (t > 0.f) {
        int prim = __float_as_int(v0.w);
        if (t < h.t || (t == h.t && prim < h.prim)) { h.t = t; h.prim = prim; h.k = k; }
    }
}

// tri_update against the bound tb, which is h.t for a lane of the packet's session and
// -1 for the others (no triangle passes, so their hit records stay as they are)
__device__ __forceinline__ void tri_update_bound(const Ray &ray, const float4 *__restrict__ tris, int k, float &tb,
                                                 HitRec &h) {
    const float4 *tp = tris + 3 * (size_t)k;
    float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
    float t = tri_hit(ray, v0, v1, v2, tb);
    if (t > 0.f) {
        int prim = __float_as_int(v0.w);
        if (t < tb || (t == tb && prim < h.prim)) { h.t = t; h.prim = prim; h.k = k; tb = t; }
    }
}

// Returns true when the query has ended (stack empty or a guard tripped).
template <int kCap>
__device__ __forceinline__ bool step4(const Ray &ray, const Bvh4Node *__restrict__ nodes4, int n4,
                                      const float4 *__restrict__ tris, int n_tree, int &node, int *stack, int &sp,
                                      HitRec &h, uint32_t &n_visit, uint32_t &n_tests, uint32_t *status) {
    if (node < 0) {
        const int k = ~node;
        if (k >= n_tree) {
            atomicOr(status, 2u);
            return true;
        }
        n_tests++;
        tri_update(ray, tris, k, h);
    } else {
        if (node >= n4) {
            atomicOr(status, 2u);
            return true;
        }
        n_visit++;
        const float4 *np = reinterpret_cast<const float4 *>(nodes4 + node);
        const float4 lx = __ldg(np), hx = __ldg(np + 1), ly = __ldg(np + 2), hy = __ldg(np + 3);
        const float4 lz = __ldg(np + 4), hz = __ldg(np + 5);
        const int4 rf = __ldg(reinterpret_cast<const int4 *>(np + 6));
        float t[4];
        int c[4] = {rf.x, rf.y, rf.z, rf.w};
        if (!box_hit_w(ray, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x, h.t, t[0]) || c[0] == kEmptyChild) {
            c[0] = kEmptyChild; t[0] = INFINITY;
        }
        if (!box_hit_w(ray, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y, h.t, t[1]) || c[1] == kEmptyChild) {
            c[1] = kEmptyChild; t[1] = INFINITY;
        }
        if (!box_hit_w(ray, lx.z, ly.z, lz.z, hx.z, hy.z, hz.z, h.t, t[2]) || c[2] == kEmptyChild) {
            c[2] = kEmptyChild; t[2] = INFINITY;
        }
        if (!box_hit_w(ray, lx.w, ly.w, lz.w, hx.w, hy.w, hz.w, h.t, t[3]) || c[3] == kEmptyChild) {
            c[3] = kEmptyChild; t[3] = INFINITY;
        }
        // an entry distance that overflowed to +inf still sorts before the misses
#pragma unroll
        for (int e = 0; e < 4; e++)
            if (c[e] != kEmptyChild) t[e] = fminf(t[e], 3.4e38f);
        cx_hit(t[0], c[0], t[1], c[1]);
        cx_hit(t[2], c[2], t[3], c[3]);
        cx_hit(t[0], c[0], t[2], c[2]);
        cx_hit(t[1], c[1], t[3], c[3]);
        cx_hit(t[1], c[1], t[2], c[2]);
#pragma unroll
        for (int e = 3; e >= 1; e--) {
            if (c[e] != kEmptyChild) {
                if (sp < kCap) stack[sp++] = c[e];
                else atomicOr(status, 1u);
            }
        }
        if (c[0] != kEmptyChild) {
            node = c[0];
            return false;
        }
    }
    if (sp == 0) return true;
    node = stack[--sp];
    return false;
}

// One step of the binary traversal: an internal node tests its two child boxes and
// descends into the nearer hit child (the farther one is pushed); a leaf is
// intersected.  Returns true when the query has ended (stack empty or a guard tripped).
template <int kCap>
__device__ __forceinline__ bool step2(const Ray &ray, const BvhNode *__restrict__ nodes, int n_nodes,
                                      const float4 *__restrict__ tris, int n_tree, int &node, int *stack, int &sp,
                                      HitRec &h, uint32_t &n_visit, uint32_t &n_tests, uint32_t *status) {
    if (node >= n_nodes || (node < 0 && ~node >= n_tree)) {
        atomicOr(status, 2u);
        return true;
    }
    if (node >= 0) {
        n_visit++;
        const float4 *np = reinterpret_cast<const float4 *>(nodes + node);
        float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
        int4 ref = __ldg(reinterpret_cast<const int4 *>(np + 3));
        float t0, t1;
        bool h0, h1;
        box_pair(ray, a, b, c, h.t, h0, t0, h1, t1);
        if (h0 && h1) {
            int nearc = t0 <= t1 ? ref.x : ref.y, farc = t0 <= t1 ? ref.y : ref.x;
            if (sp < kCap) stack[sp++] = farc;
            else atomicOr(status, 1u);
            node = nearc;
            return false;
        }
        if (h0) { node = ref.x; return false; }
        if (h1) { node = ref.y; return false; }
    } else {
        n_tests++;
        tri_update(ray, tris, ~node, h);
    }
    if (sp == 0) return true;
    node = stack[--sp];
    return false;
}

// closest hit = lexicographic min of (t, prim id); boxes with entry == best are kept.
// A reference outside the tree, a full stack or more steps than a valid tree can take
// set the status word and end the query (no fault, no endless loop).
__device__ HitRec closest_hit(const SceneDev &sc, const Ray &r, uint32_t *status, uint32_t &n_visit,
                              uint32_t &n_tests) {
    HitRec h{INFINITY, -1, -1};
    // large triangles first: their hits bound the tree traversal
    for (int k = sc.n_tris; k < sc.n_tris + sc.n_large; k++) {
        n_tests++;
        const float4 *tp = sc.tris + 3 * (size_t)k;
        float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
        float t = tri_hit(r, v0, v1, v2, h.t);
        if (t > 0.f) {
            int prim = __float_as_int(v0.w);
            if (t < h.t || (t == h.t && prim < h.prim)) { h.t = t; h.prim = prim; h.k = k; }
        }
    }
    if (sc.n_tris <= 0) return h;
    int stack[kStack];
    int sp = 0;
    if (sc.nodes4) {
        int node4 = sc.root4;
        const long long max4 = 4ll * sc.n_tris + 64;
        for (long long steps = 0;; steps++) {
            if (steps > max4) {
                atomicOr(status, 2u);
                break;
            }
            if (step4<kStack>(r, sc.nodes4, sc.n_nodes4, sc.tris, sc.n_tris, node4, stack, sp, h, n_visit, n_tests,
                              status))
                break;
        }
        return h;
    }
    int node = sc.root;
    const long long max_steps = 4ll * sc.n_tris + 64;
    for (long long steps = 0;; steps++) {
        if (steps > max_steps) {
            atomicOr(status, 2u);
            break;
        }
        if (step2<kStack>(r, sc.nodes, sc.n_tris - 1, sc.tris, sc.n_tris, node, stack, sp, h, n_visit, n_tests, status))
            break;
    }
    return h;
}

// ---------------------------------------------------------------------------
// A0: G-buffer producer
// ---------------------------------------------------------------------------
__global__ void k_primary(DevCam cam, DevParams p, SceneDev sc, float4 *color, float *depth, float4 *normal,
                          int32_t *prim, uint32_t *status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= cam.W || j >= cam.H) return;
    size_t q = (size_t)j * cam.W + i;
    float3 d = pixel_dir(cam, i + 0.5f, j + 0.5f);
    Ray r = make_ray(cam.O, d);
    uint32_t nv = 0, nt = 0;
    HitRec h = closest_hit(sc, r, status, nv, nt);
    if (prim) prim[q] = h.prim;
    if (h.prim < 0) {
        color[q] = make_float4(p.sky.x, p.sky.y, p.sky.z, 1.f);
        depth[q] = INFINITY;
        normal[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float3 n;
    float3 col = shade(p, sc, h, d, n);
    color[q] = make_float4(col.x, col.y, col.z, 1.f);
    depth[q] = h.t * dot(d, cam.F);
    normal[q] = make_float4(n.x, n.y, n.z, 0.f);
}

// ---------------------------------------------------------------------------
// A6: edge measure for the adaptive ray count (Eq. 2, Eq. 3)
// ---------------------------------------------------------------------------
// 5x5 binomial blur of (z, n.xyz) packed as float4, clamp-to-edge
template <class AS>
__global__ void k_blur_zn(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_HPX, i, j);
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const float *z_h = S.z_h;
    const float4 *n_h = S.n_h;
    float4 *out = S.zn;
    if (S.p.ray_mode != 1 || i >= W2 || j >= H2) return;
    const float b[5] = {1.f, 4.f, 6.f, 4.f, 1.f};
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int dy = -2; dy <= 2; dy++) {
        int y = min(max(j + dy, 0), H2 - 1);
        for (int dx = -2; dx <= 2; dx++) {
            int x = min(max(i + dx, 0), W2 - 1);
            size_t q = (size_t)y * W2 + x;
            float w = b[dx + 2] * b[dy + 2];
            float4 n = __ldg(&n_h[q]);
            acc = f4fma(w, make_float4(__ldg(&z_h[q]), n.x, n.y, n.z), acc);
        }
    }
    out[(size_t)j * W2 + i] = f4scale(1.f / 256.f, acc);
}

// 5x5 Sobel ([-1 -2 0 2 1] x [1 4 6 4 1] / 128) -> x_n (Eq. 2, 3) and x_f (Eq. 4)
template <class AS>
__global__ void k_edges(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_HPX, i, j);
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const DevParams &p = S.p;
    const float4 *zn = S.zn;
    const float *var_prev = S.var_in;
    const int has_prev = S.valid;
    float *xn = S.xn, *xf = S.xf;
    if (p.ray_mode != 1 || i >= W2 || j >= H2) return;
    const float sm[5] = {1.f, 4.f, 6.f, 4.f, 1.f}, dv[5] = {-1.f, -2.f, 0.f, 2.f, 1.f};
    float4 gx = make_float4(0.f, 0.f, 0.f, 0.f), gy = gx;
    for (int dy = -2; dy <= 2; dy++) {
        int y = min(max(j + dy, 0), H2 - 1);
        for (int dx = -2; dx <= 2; dx++) {
            int x = min(max(i + dx, 0), W2 - 1);
            float4 v = __ldg(&zn[(size_t)y * W2 + x]);
            gx = f4fma(dv[dx + 2] * sm[dy + 2], v, gx);
            gy = f4fma(sm[dx + 2] * dv[dy + 2], v, gy);
        }
    }
    gx = f4scale(1.f / 128.f, gx);
    gy = f4scale(1.f / 128.f, gy);
    size_t q = (size_t)j * W2 + i;
    float zc = __ldg(&zn[q]).x;
    float dd = sqrtf(gx.x * gx.x + gy.x * gy.x) / zc;
    float dn = sqrtf(gx.y * gx.y + gx.z * gx.z + gx.w * gx.w + gy.y * gy.y + gy.z * gy.z + gy.w * gy.w);
    float x = (dd + dn) * p.s;
    float x_n = sat(1.f - 1.f / (x + 1.f));
    float s2 = has_prev ? __ldg(&var_prev[q]) : 0.f;
    xn[q] = x_n;
    xf[q] = sat(x_n + s2 * p.var_w_mask) * p.m;
}

// ---------------------------------------------------------------------------
// A6: mask, ray count, and compaction into a pixel queue and a flat ray list
// ---------------------------------------------------------------------------
// Per block (32 x 8 pixels, one warp per 8 x 4 tile) one atomic reserves room for the
// block's masked pixels (queue) and their rays.  A pixel's rays own the consecutive
// slots first_ray[q] + s (s = sample index): the tracer writes each ray and its hit
// there and the shader reduces them in sample order.  The order in which the tracer
// takes the rays is a separate list (ray_pix: work items q << 6 | s over the same
// range): inside the block the rays are grouped by the cell of their lens point on a
// g x g grid over the aperture's bounding square (g = BatchArgs::lens_grid; 1 keeps
// pixel order), cells taken in Morton order, so the 32 rays a tracer warp takes leave
// nearby lens points for nearby pixels and stay close together through the blurred near
// field.  The grouping changes no result: every ray is traced independently.
constexpr int kMaxLensGrid = 16, kMaxLensCells = kMaxLensGrid * kMaxLensGrid;

__device__ __forceinline__ int morton2(int x, int y) {
    int m = 0;
#pragma unroll
    for (int b = 0; b < 4; b++) m |= (((x >> b) & 1) << (2 * b)) | (((y >> b) & 1) << (2 * b + 1));
    return m;
}

// Lens cell of the ray (q, s) on a g x g grid: its lens sample (the same Philox draw as
// lens_ray) on the unit disk; the cell's Morton index (< 256 for g <= 16).  Only a
// scheduling key.
__device__ __forceinline__ int lens_cell(const DevCam &cam, const DevParams &p, uint32_t q, int s, int g) {
    unsigned long long x0, x1;
    philox2(q, (unsigned long long)s, cam.frame, 0ull, p.seed, p.session, x0, x1);
    const float u1 = (float)(x0 >> 40) * 5.9604644775390625e-8f;
    const float u2 = (float)(x1 >> 40) * 5.9604644775390625e-8f;
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    const float r = sqrtf(u1), half_g = 0.5f * (float)g;
    const int cx = min(max((int)((r * cs + 1.f) * half_g), 0), g - 1);
    const int cy = min(max((int)((r * sn + 1.f) * half_g), 0), g - 1);
    return morton2(cx, cy);
}
static_assert(DOF_MAX_RAYS <= 64, "work items keep the sample index in 6 bits");

template <class AS>
__global__ void __launch_bounds__(256) k_mask_compact(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_HPX, i, j);
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const DevParams &p = S.p;
    const float *xf = S.xf;
    int32_t *nrays = S.nrays;
    uint32_t *queue = S.queue, *first_ray = S.first_ray, *ray_pix = S.ray_pix, *counters = S.counters;
    const unsigned lane = threadIdx.x, warp = threadIdx.y;
    // the dilated max-CoC of the block's four tiles (A2; the prefilter computes the same
    // values on the other stream and writes them out)
    __shared__ float2 dil_s[4];
    dilate_block_tiles(S, i - (int)threadIdx.x, j - (int)threadIdx.y, dil_s);
    __syncthreads();
    // each warp takes an 8x4 tile of the block's 32x8 pixels, lanes in Morton order, so
    // that the 32 consecutive rays a tracer warp takes come from a compact patch
    i = i - (int)threadIdx.x + (int)((warp & 3u) * 8u + (lane & 1u) + ((lane >> 1) & 2u) + ((lane >> 2) & 4u));
    j = j - (int)threadIdx.y + (int)((warp >> 2) * 4u + ((lane >> 1) & 1u) + ((lane >> 2) & 2u));
    int n = 0;
    uint32_t q = 0;
    if (i < W2 && j < H2) {
        q = (uint32_t)j * W2 + i;
        float near_max = dil_s[warp & 3u].x;
        if (near_max >= p.mask_near_hpx) {
            if (p.ray_mode == 0) n = p.spp;
            else n = (int)fminf(fmaxf(ceilf(__ldg(&xf[q])), 1.f), p.m);
        }
        nrays[q] = n;
    }
    // warp: inclusive prefix of the ray counts, ballot of the masked pixels
    int incl = n;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += v;
    }
    unsigned ball = __ballot_sync(0xffffffffu, n > 0);
    __shared__ uint32_t w_pix[8], w_ray[8], b_pix, b_ray;
    if (lane == 31) { w_pix[warp] = __popc(ball); w_ray[warp] = (uint32_t)incl; }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        uint32_t tp = 0, tr = 0;
        for (int w = 0; w < 8; w++) {
            uint32_t a = w_pix[w], b = w_ray[w];
            w_pix[w] = tp; w_ray[w] = tr;
            tp += a; tr += b;
        }
        // queue length and ray count share one 64-bit word (rays < 2^32 by the size limits)
        unsigned long long old = 0;
        if (tp) old = atomicAdd(reinterpret_cast<unsigned long long *>(counters),
                                ((unsigned long long)tr << 32) | tp);
        b_pix = (uint32_t)old;
        b_ray = (uint32_t)(old >> 32);
    }
    __syncthreads();     // b_pix, b_ray and the warp offsets are read by every thread below
    const int grid = A.lens_grid;
    if (grid <= 1) {
        // pixel order: the work items follow the pixels' own slots
        if (n > 0) {
            queue[b_pix + w_pix[warp] + __popc(ball & ((1u << lane) - 1u))] = q;
            const uint32_t f = b_ray + w_ray[warp] + (uint32_t)(incl - n);
            first_ray[q] = f;
            for (int s = 0; s < n; s++) ray_pix[f + s] = (q << 6) | (uint32_t)s;
        }
        return;
    }
    // lens cells of the block's rays (Morton indices below the power-of-two square that
    // holds the g x g grid), and how many rays fall in each
    __shared__ uint32_t cell_n[kMaxLensCells], cell_at[kMaxLensCells];
    __shared__ uint8_t cell_of[DOF_MAX_RAYS][256];
    const int tid = (int)(warp * 32u + lane);
    cell_n[tid] = 0u;                       // 256 threads, 256 cells
    __syncthreads();
    for (int s = 0; s < n; s++) {
        const int c = lens_cell(S.cam, p, q, s, grid);
        cell_of[s][tid] = (uint8_t)c;
        atomicAdd(&cell_n[c], 1u);
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive prefix over the 256 cells: 8 per lane, then across the warp
        uint32_t v[8], acc = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) { v[k] = acc; acc += cell_n[lane * 8 + k]; }
        uint32_t incl_c = acc;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl_c, o);
            if ((int)lane >= o) incl_c += u;
        }
        const uint32_t base = incl_c - acc;
#pragma unroll
        for (int k = 0; k < 8; k++) cell_at[lane * 8 + k] = base + v[k];
    }
    __syncthreads();
    if (n > 0) {
        queue[b_pix + w_pix[warp] + __popc(ball & ((1u << lane) - 1u))] = q;
        first_ray[q] = b_ray + w_ray[warp] + (uint32_t)(incl - n);
        for (int s = 0; s < n; s++) {
            const uint32_t at = atomicAdd(&cell_at[cell_of[s][tid]], 1u);
            ray_pix[b_ray + at] = (q << 6) | (uint32_t)s;
        }
    }
}

// ---------------------------------------------------------------------------
// A8: thin-lens rays (Section 3.2.2)
// ---------------------------------------------------------------------------
// The ray of half-resolution pixel q and lens sample s: direction through the pixel
// and the lens centre meets the focus plane at Pf; Philox(counter = (q, s, frame, 0),
// key = (seed, session)) gives the lens point.  The tracer makes each ray once and keeps
// it (origin, direction) for the shader.
__device__ __forceinline__ void lens_ray(const DevCam &cam, const DevParams &p, uint32_t q, int s, float3 &L,
                                      float3 &dir) {
    int i = (int)(q % (uint32_t)cam.W2), j = (int)(q / (uint32_t)cam.W2);
    float3 dp = pixel_dir(cam, 2.f * i + 1.f, 2.f * j + 1.f);
    float tf = cam.d / dot(dp, cam.F);
    float3 Pf = cam.O + tf * dp;
    unsigned long long x0, x1;
    philox2(q, (unsigned long long)s, cam.frame, 0ull, p.seed, p.session, x0, x1);
    float u1 = (float)(x0 >> 40) * 5.9604644775390625e-8f;
    float u2 = (float)(x1 >> 40) * 5.9604644775390625e-8f;
    float rr = cam.lens_r * sqrtf(u1), lx, ly;
    if (p.blades == 0) {
        float sn, cs;
        sincospif(2.f * u2, &sn, &cs);
        lx = rr * cs; ly = rr * sn;
    } else {
        // regular n-gon (vertex k at angle 2 pi k / n): sector k = floor(n u2), position
        // t = n u2 - k along its edge; sqrt(u1) (lerp of the edge's vertices) is uniform
        // over the triangle (centre, V_k, V_k+1)
        const float a = u2 * (float)p.blades;
        const int k = min((int)a, p.blades - 1);
        const float t = a - (float)k;
        float s0, c0, s1, c1;
        sincospif(2.f * (float)k / (float)p.blades, &s0, &c0);
        sincospif(2.f * (float)(k + 1) / (float)p.blades, &s1, &c1);
        lx = rr * ((1.f - t) * c0 + t * c1);
        ly = rr * ((1.f - t) * s0 + t * s1);
    }
    L = cam.O + lx * cam.R + ly * cam.U;
    dir = normalize(Pf - L);
}


// Persistent tracer, one ray per lane (Aila and Laine 2009, persistent threads with
// dynamic fetch): lanes whose ray has finished take new rays from the ray list when
// enough of the warp is idle, so divergent rays do not hold the warp.  Writes the
// closest hit of each ray: (sorted triangle index or -1, t).  kWide: every session of
// the batch traverses its 4-wide tree, else every session its binary tree.
template <bool kWide, int kCap, class AS>
__global__ void __launch_bounds__(kTraceThreads, 7) k_trace_rays(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    // inclusive prefix of the sessions' ray counts (the batch's concatenated ray list)
    __shared__ uint32_t pre[kMaxBatch];
    if (threadIdx.x < 32) {
        uint32_t c = lane < (unsigned)A.ns ? *((volatile uint32_t *)&A.s[lane].counters[1]) : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, c, o);
            if ((int)lane >= o) c += v;
        }
        pre[lane] = c;
    }
    __syncthreads();
    const uint32_t total = pre[A.ns - 1];
    const int refill_idle = A.refill_idle, steps_per_round = A.steps_per_round;
    uint32_t n_visit = 0, n_tests = 0;
    bool have = false, exhausted = false;
    uint32_t r = 0;
    int si = 0;
    Ray ray;
    HitRec h{INFINITY, -1, -1};
    int node = 0, sp = 0, n_tree = 0, n_nodes = 0;
    const BvhNode *nodes = nullptr;
    const Bvh4Node *nodes4 = nullptr;
    const float4 *tris = nullptr;
    uint32_t steps = 0, max_steps = 0;
    int stack[kCap];
    while (true) {
        unsigned idle = __ballot_sync(0xffffffffu, !have);
        if (idle == 0xffffffffu || (!exhausted && __popc(idle) >= refill_idle)) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(A.cursor, (uint32_t)__popc(idle));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (base >= total) exhausted = true;
            if (!have) {
                uint32_t g = base + __popc(idle & lt);
                if (g < total) {
                    // session of global ray g: the first s with pre[s] > g
                    int lo = 0, hi = A.ns - 1;
                    while (lo < hi) {
                        int mid = (lo + hi) >> 1;
                        if (pre[mid] > g) hi = mid;
                        else lo = mid + 1;
                    }
                    si = lo;
                    const SessDesc &S = A.s[si];
                    // work item (pixel q, sample sm) -> the ray's own slot r
                    const uint32_t wq = __ldg(&S.ray_pix[g - (si > 0 ? pre[si - 1] : 0u)]);
                    const uint32_t q = wq >> 6;
                    const int sm = (int)(wq & 63u);
                    if (q >= (uint32_t)S.N || sm >= S.max_rays) {
                        // a work item outside the session: flag it, the lane stays idle
                        atomicOr(&A.s[si].counters[3], 2u);
                    } else {
                        r = __ldg(&S.first_ray[q]) + (uint32_t)sm;
                        float3 L, dir;
                        lens_ray(S.cam, S.p, q, sm, L, dir);
                        // kept for the shader, which takes the ray as made here
                        S.ray_a[r] = make_float4(L.x, L.y, L.z, dir.x);
                        S.ray_b[r] = make_float2(dir.y, dir.z);
                        ray = make_ray(L, dir);
                        if (kWide) {
                            nodes4 = S.sc.nodes4;
                            n_nodes = S.sc.n_nodes4;
                        } else {
                            nodes = S.sc.nodes;
                            n_nodes = S.sc.n_tris - 1;
                        }
                        tris = S.sc.tris;
                        n_tree = S.sc.n_tris;
                        h = HitRec{INFINITY, -1, -1};
                        for (int k = n_tree; k < n_tree + S.sc.n_large; k++) {
                            n_tests++;
                            const float4 *tp = tris + 3 * (size_t)k;
                            float t = tri_hit(ray, __ldg(tp), __ldg(tp + 1), __ldg(tp + 2), h.t);
                            if (t > 0.f) {
                                int prim = __float_as_int(__ldg(tp).w);
                                if (t < h.t || (t == h.t && prim < h.prim)) { h.t = t; h.prim = prim; h.k = k; }
                            }
                        }
                        node = kWide ? S.sc.root4 : S.sc.root;
                        sp = 0;
                        steps = 0;
                        max_steps = (uint32_t)min(4ll * n_tree + 64, 4294967295ll);
                        have = n_tree > 0;
                        if (!have) S.hits[r] = make_int2(h.k, __float_as_int(h.t));
                    }
                }
            }
            if (__ballot_sync(0xffffffffu, have) == 0 && exhausted) break;
        }
        if (!have) continue;
        for (int it = 0; it < steps_per_round; it++) {
            bool done;
            if (++steps > max_steps) {
                atomicOr(&A.s[si].counters[3], 2u);
                done = true;
            } else if (kWide) {
                done = step4<kCap>(ray, nodes4, n_nodes, tris, n_tree, node, stack, sp, h, n_visit, n_tests,
                             &A.s[si].counters[3]);
            } else {
                done = step2<kCap>(ray, nodes, n_nodes, tris, n_tree, node, stack, sp, h, n_visit, n_tests,
                             &A.s[si].counters[3]);
            }
            if (done) {
                A.s[si].hits[r] = make_int2(h.k, __float_as_int(h.t));
                have = false;
                break;
            }
        }
    }
    // traversal work (node visits, triangle tests), one atomic per warp, booked on the
    // first session of the batch
    unsigned long long a = n_visit, b = n_tests;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.s[0].counters[4]), a);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.s[0].counters[6]), b);
    }
}

// Packet tracer over the binary tree: the 32 rays a warp takes traverse it together,
// one node sequence for the warp held in a warp-uniform stack.  A child is entered
// when the ray of any lane enters its box, and the two children go in the order that
// most of the lanes entering both prefer.  Each lane tests boxes and triangles with
// its own ray and its own best hit (inclusive cull), so every ray ends with the closest
// hit that the per-ray traversal finds.  A warp's rays come from a compact patch of
// pixels (pixel order: with several rays per pixel, the cones of a few pixels through
// their focus points) or of pixels and aperture (lens-cell order, close to a pinhole
// frustum): the warp then steps with all its lanes and one broadcast load per node, at
// the price of the nodes that only some of its rays need.  Lanes of a warp that
// straddles two sessions of a batch trace one session's packet after the other.
template <int kCap, bool kStats, class AS>
__global__ void __launch_bounds__(kTraceThreads, 8) k_trace_packets(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    const unsigned lane = threadIdx.x & 31;
    __shared__ uint32_t pre[kMaxBatch];
    if (threadIdx.x < 32) {
        uint32_t c = lane < (unsigned)A.ns ? *((volatile uint32_t *)&A.s[lane].counters[1]) : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, c, o);
            if ((int)lane >= o) c += v;
        }
        pre[lane] = c;
    }
    __syncthreads();
    const uint32_t total = pre[A.ns - 1];
    uint32_t n_visit = 0, n_tests = 0;
    // the warp's stack: one copy in shared memory (every lane writes the same entry and
    // reads it back, so no lane waits on another's store)
    __shared__ int stacks[kTraceThreads / 32][kCap];
    int *stack = stacks[threadIdx.x >> 5];
    while (true) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(A.cursor, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total) break;
        const uint32_t g = base + lane;
        bool pending = false;           // the lane holds a ray not yet traced
        int si = 0;
        uint32_t r = 0;
        Ray ray = make_ray(make_float3(0.f, 0.f, 0.f), make_float3(0.f, 0.f, 1.f));
        HitRec h{INFINITY, -1, -1};
        if (g < total) {
            int lo = 0, hi = A.ns - 1;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (pre[mid] > g) hi = mid;
                else lo = mid + 1;
            }
            si = lo;
            const SessDesc &S = A.s[si];
            const uint32_t wq = __ldg(&S.ray_pix[g - (si > 0 ? pre[si - 1] : 0u)]);
            const uint32_t q = wq >> 6;
            const int sm = (int)(wq & 63u);
            if (q >= (uint32_t)S.N || sm >= S.max_rays) {
                atomicOr(&A.s[si].counters[3], 2u);
            } else {
                r = __ldg(&S.first_ray[q]) + (uint32_t)sm;
                float3 L, dir;
                lens_ray(S.cam, S.p, q, sm, L, dir);
                S.ray_a[r] = make_float4(L.x, L.y, L.z, dir.x);
                S.ray_b[r] = make_float2(dir.y, dir.z);
                ray = make_ray(L, dir);
                const float4 *__restrict__ tris = S.sc.tris;
                const int n_tree = S.sc.n_tris;
                for (int k = n_tree; k < n_tree + S.sc.n_large; k++) {
                    n_tests++;
                    tri_update(ray, tris, k, h);
                }
                pending = true;
            }
        }
        while (true) {
            const unsigned pm = __ballot_sync(0xffffffffu, pending);
            if (pm == 0) break;
            const int lead = __shfl_sync(0xffffffffu, si, __ffs(pm) - 1);
            const bool act = pending && si == lead;
            const SessDesc &S = A.s[lead];
            const int n_tree = S.sc.n_tris;
            if (n_tree > 0) {
                const BvhNode *__restrict__ nodes = S.sc.nodes;
                const float4 *__restrict__ tris = S.sc.tris;
                int node = S.sc.root, sp = 0;
                // the best distance the lane tests boxes and triangles against: its own
                // for a lane of this session, -1 (nothing passes) for the others
                float tb = act ? h.t : -1.f;
                // no per-step guard: the tree passed the structure check at upload (every
                // reference in range, every node but the root referenced once), so the
                // packet enters each node at most once and ends within the tree's size;
                // the stack holds one entry per level at most, and the launch's capacity
                // covers the depth measured on those references
                for (;;) {
                    if (node >= 0) {
                        const float4 *np = reinterpret_cast<const float4 *>(nodes + node);
                        const float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
                        const int4 ref = __ldg(reinterpret_cast<const int4 *>(np + 3));
                        float t0, t1;
                        bool h0, h1;
                        box_pair(ray, a, b, c, tb, h0, t0, h1, t1);
                        if (kStats) n_visit += act ? 1u : 0u;
                        const unsigned m0 = __ballot_sync(0xffffffffu, h0), m1 = __ballot_sync(0xffffffffu, h1);
                        if (m0 && m1) {
                            const unsigned right_first = __ballot_sync(0xffffffffu, h0 && h1 && t1 < t0);
                            const bool rf = 2 * __popc(right_first) > __popc(m0 & m1);
                            // at most one entry per level above the node: sp < depth <= kCap
                            stack[sp++] = rf ? ref.x : ref.y;
                            node = rf ? ref.y : ref.x;
                            continue;
                        }
                        if (m0) { node = ref.x; continue; }
                        if (m1) { node = ref.y; continue; }
                    } else {
                        if (kStats && act) n_tests++;
                        tri_update_bound(ray, tris, ~node, tb, h);
                    }
                    if (sp == 0) break;
                    node = stack[--sp];
                }
            }
            if (act) {
                S.hits[r] = make_int2(h.k, __float_as_int(h.t));
                pending = false;
            }
        }
    }
    if (!kStats) return;
    unsigned long long a = n_visit, b = n_tests;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.s[0].counters[4]), a);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.s[0].counters[6]), b);
    }
}

// Shading and the per-pixel near/far split of the masked pixel queue[e]: its rays, as
// the tracer made and kept them, are shaded at their recorded hits and reduced in
// sample order.
template <class AS>
__global__ void __launch_bounds__(128) k_shade(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int lb;
    const SessDesc &S = A.s[find_session(A, SH_SHADE, blockIdx.x, lb)];
    const DevCam &cam = S.cam;
    const DevParams &p = S.p;
    const SceneDev &sc = S.sc;
    const uint32_t *queue = S.queue, *first_ray = S.first_ray;
    const int32_t *nrays = S.nrays;
    const int2 *hits = S.hits;
    float4 *rt = S.rt;
    int32_t *ray_prim = S.record_rays ? S.ray_prim : nullptr;
    const int max_rays = S.max_rays;
    const uint32_t e = lb * blockDim.x + threadIdx.x;
    const uint32_t count = *((volatile const uint32_t *)&S.counters[0]);
    if (e >= count) return;
    const size_t N = (size_t)cam.W2 * cam.H2;
    const float inv_sqrt2 = 0.70710678118654752f;
    uint32_t q = queue[e];
    int n = nrays[q];
    uint32_t f = first_ray[q];
    float Sw = 0.f, Bn = 0.f, Bf = 0.f, Fw = 0.f;
    float3 An = make_float3(0.f, 0.f, 0.f), Af = An, Pfar = An;
    const float4 *__restrict__ ray_a = S.ray_a;
    const float2 *__restrict__ ray_b = S.ray_b;
    for (int s = 0; s < n; s++) {
        // the ray as the tracer made it (lens_ray): origin on the lens and direction
        const float4 ra = __ldg(&ray_a[f + s]);
        const float2 rb = __ldg(&ray_b[f + s]);
        const float3 L = make_float3(ra.x, ra.y, ra.z), dir = make_float3(ra.w, rb.x, rb.y);
        int2 hh = __ldg(&hits[f + s]);
        HitRec h{__int_as_float(hh.y), -1, hh.x};
        float3 col;
        float z;
        if (h.k >= 0) {
            h.prim = __float_as_int(__ldg(&sc.tris[3 * (size_t)h.k]).w);
            float3 nrm;
            col = shade(p, sc, h, dir, nrm);
            z = fminf(h.t * dot(dir, cam.F), p.z_far);
        } else {
            col = p.sky;
            z = p.z_far;
        }
        float c = coc_of(cam, z);
        float rho = fabsf(fminf(fmaxf(0.25f * c, -p.rmax_hpx), p.rmax_hpx));
        float w = sat(-c * inv_sqrt2);
        if (ray_prim && s < max_rays) ray_prim[(size_t)q * max_rays + s] = h.prim;
        Sw += w;
        An = An + w * col;
        Af = Af + (1.f - w) * col;
        Bn += w * rho;
        Bf += (1.f - w) * rho;
        // far position: the hit, or for a ray that escapes, its point at depth z_far
        // (the sky is a finite depth, so its reprojection follows the ray's direction)
        const float tf = h.k >= 0 ? h.t : p.z_far / dot(dir, cam.F);
        Pfar = Pfar + (1.f - w) * (L + tf * dir);
        Fw += 1.f - w;
    }
    float inv_n = 1.f / (float)n;
    float invF = Fw > 0.f ? 1.f / Fw : 0.f;
    rt[q] = make_float4(An.x * inv_n, An.y * inv_n, An.z * inv_n, Sw * inv_n);
    rt[N + q] = make_float4(Af.x * inv_n, Af.y * inv_n, Af.z * inv_n, (float)n);
    rt[2 * N + q] = make_float4(Bn * inv_n, Bf * inv_n, Fw, 0.f);
    rt[3 * N + q] = make_float4(Pfar.x * invF, Pfar.y * invF, Pfar.z * invF, 0.f);
}

}  // namespace

void launch_primary(const DevCam &cam, const DevParams &p, SceneDev sc, float4 *color, float *depth,
                    float4 *normal, int32_t *prim, uint32_t *status, cudaStream_t st) {
    dim3 b(16, 8), g((cam.W + 15) / 16, (cam.H + 7) / 8);
    k_primary<<<g, b, 0, st>>>(cam, p, sc, color, depth, normal, prim, status);
    count_launches(1);
}

template <class AS>
void launch_mask_b(const BatchArgs &A, const AS &as, bool any_adaptive, cudaStream_t st, DofHistory *tm) {
    const int n = A.ns;
    if (any_adaptive) {
        k_blur_zn<AS><<<A.start[SH_HPX][n], dim3(32, 8), 0, st>>>(as);
        k_edges<AS><<<A.start[SH_HPX][n], dim3(32, 8), 0, st>>>(as);
    }
    tmark(tm, DOF_K_EDGES, st);
    k_mask_compact<AS><<<A.start[SH_HPX][n], dim3(32, 8), 0, st>>>(as);
    count_launches(any_adaptive ? 3 : 1);
    tmark(tm, DOF_K_MASK, st);
}

template <class AS>
void launch_trace_b(const BatchArgs &A, const AS &as, int blocks, cudaStream_t st, DofHistory *tm) {
    // the 4-wide kernel when every session of the batch has its 4-wide tree in use
    bool wide = A.ns > 0;
    for (int i = 0; i < A.ns; i++) wide = wide && A.s[i].sc.nodes4 != nullptr;
    // the stack capacity: the smallest compiled one that holds the requested depth and
    // what every session's tree can need
    int need = A.stack_depth;
    for (int i = 0; i < A.ns; i++) need = max(need, A.s[i].sc.stack_need);
    if (A.packets && !wide && A.stats) {
        if (need <= 32) k_trace_packets<32, true, AS><<<blocks, kTraceThreads, 0, st>>>(as);
        else if (need <= 64) k_trace_packets<64, true, AS><<<blocks, kTraceThreads, 0, st>>>(as);
        else k_trace_packets<kStack, true, AS><<<blocks, kTraceThreads, 0, st>>>(as);
    } else if (A.packets && !wide) {
        if (need <= 32) k_trace_packets<32, false, AS><<<blocks, kTraceThreads, 0, st>>>(as);
        else if (need <= 64) k_trace_packets<64, false, AS><<<blocks, kTraceThreads, 0, st>>>(as);
        else k_trace_packets<kStack, false, AS><<<blocks, kTraceThreads, 0, st>>>(as);
    } else if (wide) {
        if (need <= 32) k_trace_rays<true, 32, AS><<<blocks, kTraceThreads, 0, st>>>(as);
        else if (need <= 64) k_trace_rays<true, 64, AS><<<blocks, kTraceThreads, 0, st>>>(as);
        else k_trace_rays<true, kStack, AS><<<blocks, kTraceThreads, 0, st>>>(as);
    } else {
        if (need <= 32) k_trace_rays<false, 32, AS><<<blocks, kTraceThreads, 0, st>>>(as);
        else if (need <= 64) k_trace_rays<false, 64, AS><<<blocks, kTraceThreads, 0, st>>>(as);
        else k_trace_rays<false, kStack, AS><<<blocks, kTraceThreads, 0, st>>>(as);
    }
    tmark(tm, DOF_K_TRACE, st);
    k_shade<AS><<<A.start[SH_SHADE][A.ns], 128, 0, st>>>(as);
    count_launches(2);
    tmark(tm, DOF_K_SHADE, st);
}

// the two argument forms: by value (a kernel parameter) and from device memory (graphs)
template void launch_mask_b<BatchArgs>(const BatchArgs &, const BatchArgs &, bool, cudaStream_t, DofHistory *);
template void launch_mask_b<const BatchArgs *>(const BatchArgs &, const BatchArgs *const &, bool, cudaStream_t, DofHistory *);
// Every tracer instance and the adaptive-mode kernels loaded on the current device now
// (with lazy module loading a kernel is otherwise loaded at its first launch: a batch
// whose trees need another stack capacity, or the first adaptive session, would stall a
// frame on the load).
void preload_trace_kernels() {
    cudaFuncAttributes a;
#define DOF_PRELOAD(AS)                                                        \
    cudaFuncGetAttributes(&a, k_trace_packets<32, true, AS>);                  \
    cudaFuncGetAttributes(&a, k_trace_packets<64, true, AS>);                  \
    cudaFuncGetAttributes(&a, k_trace_packets<kStack, true, AS>);              \
    cudaFuncGetAttributes(&a, k_trace_packets<32, false, AS>);                 \
    cudaFuncGetAttributes(&a, k_trace_packets<64, false, AS>);                 \
    cudaFuncGetAttributes(&a, k_trace_packets<kStack, false, AS>);             \
    cudaFuncGetAttributes(&a, k_trace_rays<true, 32, AS>);                     \
    cudaFuncGetAttributes(&a, k_trace_rays<true, 64, AS>);                     \
    cudaFuncGetAttributes(&a, k_trace_rays<true, kStack, AS>);                 \
    cudaFuncGetAttributes(&a, k_trace_rays<false, 32, AS>);                    \
    cudaFuncGetAttributes(&a, k_trace_rays<false, 64, AS>);                    \
    cudaFuncGetAttributes(&a, k_trace_rays<false, kStack, AS>);                \
    cudaFuncGetAttributes(&a, k_blur_zn<AS>);                                  \
    cudaFuncGetAttributes(&a, k_edges<AS>);
    DOF_PRELOAD(BatchArgs)
    DOF_PRELOAD(const BatchArgs *)
#undef DOF_PRELOAD
    cudaGetLastError();
}

template void launch_trace_b<BatchArgs>(const BatchArgs &, const BatchArgs &, int, cudaStream_t, DofHistory *);
template void launch_trace_b<const BatchArgs *>(const BatchArgs &, const BatchArgs *const &, int, cudaStream_t, DofHistory *);

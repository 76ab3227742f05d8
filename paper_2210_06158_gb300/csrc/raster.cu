// Object-order G-buffer producer (Section 3: the method shades a rasterised G-buffer).
//
// Visibility is resolved triangle by triangle instead of pixel by pixel: each triangle
// is set up once (its three edge planes through the lens centre give three half-planes
// of the image whose intersection holds every pixel centre whose primary ray can hit
// it), the pixels of that conservative region are enumerated, and each candidate pixel
// runs the same watertight ray/triangle test as the ray-cast producer.  The closest hit
// per pixel is the minimum of the 64-bit key (t bits, triangle id), which orders hits by
// distance and breaks exact ties on the smaller id, as the ray-cast producer does; a
// resolve pass shades it.  The two producers therefore give the same bits.
//
// Work distribution: triangles whose candidate box holds at most kSmallPx pixels are
// rasterised by the warp that set them up (the warp's 32 boxes are enumerated as one
// list, so a warp's lanes stay busy whatever the box sizes); larger ones are queued and
// cut into chunks of kChunkPx pixels that persistent blocks claim from a counter.
//
// Occlusion culling: the triangles are taken nearest first, in batches of growing size
// (sorted by a lower bound of their distance from the lens centre).  After each batch a
// two-level depth pyramid holds, per 16 x 16 and 128 x 128 pixel tile, the farthest
// closest hit so far; a triangle whose bound is beyond it on every tile of its candidate
// box is dropped whole, and a candidate pixel skips the ray test when the bound is beyond
// the pixel's own closest hit.  Keys only decrease, so a stale read or an older pyramid
// culls less, never wrongly; see near_bound for the margin.
#include "geometry.cuh"

#include <algorithm>

namespace {

constexpr int kSmallPx = 4096;       // candidate pixels above which a triangle is queued
constexpr int kChunkPx = 2048;       // pixels of one chunk of a queued triangle
constexpr int kRastThreads = 256;
constexpr int kHizShift1 = 4, kHizShift2 = 7;   // depth-pyramid tiles: 16 and 128 pixels
constexpr int kHizMaxTiles1 = 16;               // boxes over more fine tiles use the coarse level

// Edge functions of the image plane, scaled so that |a| + |b| = 1 (values in pixels)
// and oriented so that a pixel centre (x, y) can see the triangle only where
// a x + b y + c >= 0 for all three (after the safety margin added to c).
struct TriSetup {
    float e[9];                 // (a, b, c) per edge
    int i0, j0, i1, j1;         // candidate pixel box (inclusive)
};

// queued (large) triangle: setup and vertices
struct BigTri {
    float4 e0, e1, e2;          // (a, b, c, -) per edge
    int4 box;                   // i0, j0, box width, candidate pixels
    int k;                      // sorted triangle index
    float tn;                   // its distance bound (near_bound)
    int pad[2];
};

__device__ __forceinline__ float3 xyz(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float vlen(float3 v) { return sqrtf(dot(v, v)); }

__device__ __forceinline__ float edge_at(const float *e, float x, float y) { return fmaf(e[0], x, fmaf(e[1], y, e[2])); }

__device__ __forceinline__ bool edges_pass(const float *e, float x, float y) {
    return edge_at(e, x, y) >= 0.f && edge_at(e + 3, x, y) >= 0.f && edge_at(e + 6, x, y) >= 0.f;
}

// Conservative candidate region of one triangle.  Returns false when no pixel centre can
// see it.  Pixel (i, j) has its centre at (i + 1/2, j + 1/2); the primary ray direction
// of image point (x, y) is proportional to F + sx R - sy U with sx = (x + jx - W/2) / f,
// sy = (y + jy - H/2) / f (f the focal length in pixels).
//
// The ray with direction d hits the triangle at t > 0 exactly when d is a non-negative
// combination of the vertex offsets r_i = p_i - O, i.e. when e_k . d has the sign of
// D = det(r_0, r_1, r_2) for the three edge-plane normals e_k (e_0 = r_1 x r_2 ...).
// Each e_k . d is affine in (x, y) up to the positive factor of the normalisation, so
// the candidate region is an intersection of three half-planes; each is widened by
// half a pixel (far more than the rounding of either side), and its bounding box is
// found by clipping the image rectangle (its vertices are rectangle corners, line /
// rectangle-side crossings and line / line crossings).
__device__ bool tri_setup(const DevCam &cam, float4 v0, float4 v1, float4 v2, TriSetup &S) {
    const float3 p0 = xyz(v0), p1 = xyz(v1), p2 = xyz(v2);
    const float3 r0 = p0 - cam.O, r1 = p1 - cam.O, r2 = p2 - cam.O;
    const float3 g01 = p1 - p0, g12 = p2 - p1, g20 = p0 - p2;
    // a long vector times a short one: no cancellation for small, distant triangles
    const float3 e[3] = {cross(r1, g12), cross(r2, g20), cross(r0, g01)};
    const float D = -dot(g01, e[0]);     // (p0 - p1) . e0 = det(r0, r1, r2)
    const float Wf = (float)cam.W, Hf = (float)cam.H;
    const float xl = 0.5f, xh = Wf - 0.5f, yl = 0.5f, yh = Hf - 0.5f;
    // a plane through (or nearly through) the lens centre, an edge pointing at it, or a
    // degenerate triangle: the orientation is not reliable, so no edge is used and the
    // box is that of the projected vertices (the whole image if one is not in front)
    bool deg = !(fabsf(D) > 1e-5f * vlen(g01) * vlen(e[0]));
    deg = deg || !(vlen(e[0]) > 1e-5f * vlen(r1) * vlen(g12)) || !(vlen(e[1]) > 1e-5f * vlen(r2) * vlen(g20)) ||
          !(vlen(e[2]) > 1e-5f * vlen(r0) * vlen(g01));
    float xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    if (deg) {
#pragma unroll
        for (int k = 0; k < 9; k++) S.e[k] = (k % 3 == 2) ? 1.f : 0.f;
        const float3 r[3] = {r0, r1, r2};
        bool front = true;
#pragma unroll
        for (int v = 0; v < 3; v++) {
            const float zc = dot(r[v], cam.F);
            if (!(zc > 0.f)) { front = false; continue; }
            const float x = cam.halfW - cam.jx + cam.Fpx * dot(r[v], cam.R) / zc;
            const float y = cam.halfH - cam.jy - cam.Fpx * dot(r[v], cam.U) / zc;
            xmin = fminf(xmin, x - 1.f); xmax = fmaxf(xmax, x + 1.f);
            ymin = fminf(ymin, y - 1.f); ymax = fmaxf(ymax, y + 1.f);
        }
        if (!front) { xmin = xl; xmax = xh; ymin = yl; ymax = yh; }
        if (!(xmin <= xmax) || !(ymin <= ymax)) return false;   // NaN vertices
    } else {
        const float s = D > 0.f ? 1.f : -1.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float a = dot(e[k], cam.R), b = -dot(e[k], cam.U);
            float c = dot(e[k], cam.F) * cam.Fpx + a * (cam.jx - cam.halfW) + b * (cam.jy - cam.halfH);
            if (c != c) return false;            // non-finite vertices: nothing to hit
            const float n = fabsf(a) + fabsf(b);
            const float sn = s / n, cn = c * sn;
            if (n > 0.f && fabsf(cn) < INFINITY) {
                a *= sn; b *= sn;
                c = cn + 0.5f + 1e-5f * (fabsf(cn) + Wf + Hf);
            } else {
                // the edge plane holds no image direction (or its line lies beyond float
                // range): one side of it sees the whole image, the other nothing
                c = (s * c >= 0.f) ? 1.f : -1.f;
                a = b = 0.f;
            }
            S.e[3 * k] = a; S.e[3 * k + 1] = b; S.e[3 * k + 2] = c;
        }
        // vertices of the clipped image rectangle; a candidate lying on a line is tested
        // only against the other lines, with a small tolerance
        const float tol = 1e-2f;
        auto inside_other = [&](float x, float y, int skip_a, int skip_b) {
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 3; k++)
                if (k != skip_a && k != skip_b) ok = ok && edge_at(S.e + 3 * k, x, y) >= -tol;
            return ok;
        };
        auto add = [&](float x, float y) {
            xmin = fminf(xmin, x); xmax = fmaxf(xmax, x);
            ymin = fminf(ymin, y); ymax = fmaxf(ymax, y);
        };
        const float cx[2] = {xl, xh}, cy[2] = {yl, yh};
#pragma unroll
        for (int u = 0; u < 2; u++)
#pragma unroll
            for (int v = 0; v < 2; v++)
                if (inside_other(cx[u], cy[v], -1, -1)) add(cx[u], cy[v]);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float a = S.e[3 * k], b = S.e[3 * k + 1], c = S.e[3 * k + 2];
            if (b != 0.f) {
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const float y = -(a * cx[u] + c) / b;
                    if (y >= yl - tol && y <= yh + tol && inside_other(cx[u], y, k, -1))
                        add(cx[u], fminf(fmaxf(y, yl), yh));
                }
            }
            if (a != 0.f) {
#pragma unroll
                for (int v = 0; v < 2; v++) {
                    const float x = -(b * cy[v] + c) / a;
                    if (x >= xl - tol && x <= xh + tol && inside_other(x, cy[v], k, -1))
                        add(fminf(fmaxf(x, xl), xh), cy[v]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int l = (k + 1) % 3;
            const float ak = S.e[3 * k], bk = S.e[3 * k + 1], ck = S.e[3 * k + 2];
            const float al = S.e[3 * l], bl = S.e[3 * l + 1], cl = S.e[3 * l + 2];
            const float det = ak * bl - al * bk;
            if (det == 0.f) continue;
            const float x = (bk * cl - bl * ck) / det, y = (al * ck - ak * cl) / det;
            if (x >= xl - tol && x <= xh + tol && y >= yl - tol && y <= yh + tol && inside_other(x, y, k, l))
                add(fminf(fmaxf(x, xl), xh), fminf(fmaxf(y, yl), yh));
        }
        if (!(xmin <= xmax)) return false;
    }
    // pixel centres x = i + 1/2 in [xmin, xmax]
    S.i0 = max(0, (int)ceilf(fmaxf(xmin, 0.f) - 0.5f));
    S.i1 = min(cam.W - 1, (int)floorf(fminf(xmax, Wf) - 0.5f));
    S.j0 = max(0, (int)ceilf(fmaxf(ymin, 0.f) - 0.5f));
    S.j1 = min(cam.H - 1, (int)floorf(fminf(ymax, Hf) - 0.5f));
    return S.i0 <= S.i1 && S.j0 <= S.j1;
}

// q = idx / w, r = idx % w for idx < 2^22 through a float estimate and one correction
__device__ __forceinline__ void divmod(int idx, int w, float rw, int &q, int &r) {
    q = (int)(((float)idx + 0.5f) * rw);
    r = idx - q * w;
    if (r < 0) { q--; r += w; }
    else if (r >= w) { q++; r -= w; }
}

// the ray test of one candidate pixel, written to its closest-hit key
__device__ __forceinline__ void test_pixel(const DevCam &cam, unsigned long long *keys, int i, int j, float4 v0,
                                           float4 v1, float4 v2) {
    const float3 d = pixel_dir(cam, i + 0.5f, j + 0.5f);
    const Ray r = make_ray(cam.O, d);
    const float t = tri_hit(r, v0, v1, v2);
    if (t > 0.f && t < INFINITY) {
        const unsigned long long key =
            ((unsigned long long)__float_as_uint(t) << 32) | (unsigned long long)(uint32_t)__float_as_int(v0.w);
        atomicMin(&keys[(size_t)j * cam.W + i], key);
    }
}

struct SmallSlot {               // one triangle of a warp's list (112 bytes)
    float e[9];
    int i0, j0, bw;
    float rbw;
    float tn;                   // its distance bound (near_bound)
    int pad[2];
    float4 v0, v1, v2;
};

// Lower bound of the ray-test distance t of any primary ray to the triangle, for the
// occlusion test.  The directions are unit vectors, so t is the distance from the lens
// centre to the hit point, at least the distance to the triangle's bounding box, which
// is evaluated with every operation rounded down.  The test's t is a convex combination
// of the vertices' depths along the ray (barycentric weights), evaluated in FP32; the
// bound is shrunk by 2^-7 to stay below it.  A triangle with a vertex direction more than
// 60 degrees off the view axis (within 30 degrees of the lens plane) gets 0 and is never
// culled: near the lens plane those depths can cancel.
__device__ __forceinline__ float near_bound(const DevCam &cam, float4 v0, float4 v1, float4 v2) {
    const float4 v[3] = {v0, v1, v2};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float3 r = make_float3(v[k].x - cam.O.x, v[k].y - cam.O.y, v[k].z - cam.O.z);
        if (!(dot(r, cam.F) >= 0.5f * sqrtf(dot(r, r)))) return 0.f;
    }
    auto gap = [](float o, float a, float b, float c) {
        const float lo = fminf(a, fminf(b, c)), hi = fmaxf(a, fmaxf(b, c));
        return fmaxf(fmaxf(__fsub_rd(lo, o), __fsub_rd(o, hi)), 0.f);
    };
    const float gx = gap(cam.O.x, v0.x, v1.x, v2.x), gy = gap(cam.O.y, v0.y, v1.y, v2.y);
    const float gz = gap(cam.O.z, v0.z, v1.z, v2.z);
    const float s = __fadd_rd(__fadd_rd(__fmul_rd(gx, gx), __fmul_rd(gy, gy)), __fmul_rd(gz, gz));
    const float d = __fmul_rd(__fsqrt_rd(s), 0.9921875f);
    return d >= 0.f ? d : 0.f;
}

// the pixel's closest hit so far (from L2: the atomics update it there); +inf bits are
// 0xFFFFFFFF, a NaN, so an untouched pixel never culls
__device__ __forceinline__ bool occluded(const unsigned long long *keys, size_t q, float tn) {
    const unsigned long long key = __ldcg(&keys[q]);
    return tn > __uint_as_float((uint32_t)(key >> 32));
}

// Depth pyramid: hiz1 per 16 x 16 tile (tw1 x th1), hiz2 per 128 x 128 tile (tw2 x th2),
// each the largest closest-hit distance of its pixels (+inf while a pixel has none).
struct Hiz {
    const float *l1, *l2;
    int tw1, th1, tw2, th2;
};

// true when every tile of the pixel box [i0, i1] x [j0, j1] has all its pixels' closest
// hits nearer than tn (fine tiles when the box spans few of them, else coarse ones)
__device__ bool hiz_occluded(const Hiz &z, int i0, int j0, int i1, int j1, float tn) {
    if (!(tn > 0.f)) return false;
    int x0 = i0 >> kHizShift1, x1 = i1 >> kHizShift1, y0 = j0 >> kHizShift1, y1 = j1 >> kHizShift1;
    const float *lv = z.l1;
    int tw = z.tw1;
    if ((x1 - x0 + 1) * (y1 - y0 + 1) > kHizMaxTiles1) {
        x0 = i0 >> kHizShift2; x1 = i1 >> kHizShift2; y0 = j0 >> kHizShift2; y1 = j1 >> kHizShift2;
        lv = z.l2;
        tw = z.tw2;
    }
    for (int y = y0; y <= y1; y++)
        for (int x = x0; x <= x1; x++)
            if (!(tn > __ldcg(&lv[y * tw + x]))) return false;
    return true;
}

// one 16 x 16 block per fine tile: the largest closest hit of its pixels
__global__ void __launch_bounds__(256) k_hiz1(const unsigned long long *keys, int W, int H, float *hiz1, int tw1) {
    __shared__ float wmax[8];
    const int i = blockIdx.x * 16 + (threadIdx.x & 15), j = blockIdx.y * 16 + (threadIdx.x >> 4);
    float t = -INFINITY;
    if (i < W && j < H) {
        const float v = __uint_as_float((uint32_t)(__ldcg(&keys[(size_t)j * W + i]) >> 32));
        t = v == v ? v : INFINITY;       // no hit yet: +inf
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(0xffffffffu, t, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = wmax[0];
#pragma unroll
        for (int k = 1; k < 8; k++) m = fmaxf(m, wmax[k]);
        hiz1[blockIdx.y * tw1 + blockIdx.x] = m;
    }
}

// coarse tiles: the largest of their 8 x 8 fine tiles
__global__ void k_hiz2(const float *hiz1, int tw1, int th1, float *hiz2, int tw2, int th2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= tw2 || y >= th2) return;
    float m = -INFINITY;
    for (int b = 0; b < 8; b++)
        for (int a = 0; a < 8; a++) {
            const int fx = 8 * x + a, fy = 8 * y + b;
            if (fx < tw1 && fy < th1) m = fmaxf(m, hiz1[fy * tw1 + fx]);
        }
    hiz2[y * tw2 + x] = m;
}

// Setup of every triangle; the small ones are rasterised here, the others queued.
// `split` warps serve each group of 32 triangles (each sets the group up and takes every
// split-th stretch of 32 of its candidate pixels), so that scenes with few triangles
// still occupy the GPU.
__global__ void __launch_bounds__(kRastThreads) k_rast_small(DevCam cam, SceneDev sc, const uint32_t *order,
                                                              int count, int split, const float *tnear, Hiz hiz,
                                                              bool use_hiz, unsigned long long *keys, BigTri *big,
                                                              uint32_t *n_big) {
    __shared__ SmallSlot slot[kRastThreads];
    __shared__ int excl[kRastThreads];
    const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
    const int gw = blockIdx.x * (kRastThreads / 32) + (threadIdx.x >> 5);
    const int part = gw % split;
    const int idx = (gw / split) * 32 + lane;
    const int k = idx < count ? (int)__ldg(&order[idx]) : 0;
    int npx = 0;
    if (idx < count) {
        const float4 *tp = sc.tris + 3 * (size_t)k;
        const float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
        TriSetup S;
        const float tn = __ldg(&tnear[k]);
        if (tri_setup(cam, v0, v1, v2, S) && !(use_hiz && hiz_occluded(hiz, S.i0, S.j0, S.i1, S.j1, tn))) {
            const int bw = S.i1 - S.i0 + 1, bh = S.j1 - S.j0 + 1;
            const long long n = (long long)bw * bh;
            if (n > kSmallPx) {
                if (part == 0) {                     // the group's first warp queues it
                    const uint32_t b = atomicAdd(n_big, 1u);
                    BigTri B;
                    B.e0 = make_float4(S.e[0], S.e[1], S.e[2], 0.f);
                    B.e1 = make_float4(S.e[3], S.e[4], S.e[5], 0.f);
                    B.e2 = make_float4(S.e[6], S.e[7], S.e[8], 0.f);
                    B.box = make_int4(S.i0, S.j0, bw, (int)n);
                    B.k = k;
                    B.tn = tn;
                    B.pad[0] = B.pad[1] = 0;
                    big[b] = B;
                }
            } else {
                npx = (int)n;
                SmallSlot &o = slot[threadIdx.x];
#pragma unroll
                for (int q = 0; q < 9; q++) o.e[q] = S.e[q];
                o.i0 = S.i0; o.j0 = S.j0; o.bw = bw; o.rbw = 1.f / (float)bw;
                o.tn = tn;
                o.v0 = v0; o.v1 = v1; o.v2 = v2;
            }
        }
    }
    // the warp's candidate pixels as one list
    int incl = npx;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    excl[threadIdx.x] = incl - npx;
    __syncwarp();
    for (int w = lane + 32 * part; w < total; w += 32 * split) {
        // owner: the last triangle whose list starts at or before w (it has pixels)
        int l = 0;
#pragma unroll
        for (int step = 16; step; step >>= 1)
            if (excl[wbase + l + step] <= w) l += step;
        const SmallSlot &o = slot[wbase + l];
        int q, r;
        divmod(w - excl[wbase + l], o.bw, o.rbw, q, r);
        const int i = o.i0 + r, j = o.j0 + q;
        if (edges_pass(o.e, i + 0.5f, j + 0.5f) && !occluded(keys, (size_t)j * cam.W + i, o.tn))
            test_pixel(cam, keys, i, j, o.v0, o.v1, o.v2);
    }
}

// exclusive prefix of the queued triangles' chunk counts (one block)
__global__ void __launch_bounds__(1024) k_big_chunks(const BigTri *big, const uint32_t *n_big,
                                                     uint32_t *chunk_start, uint32_t *n_chunks) {
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    const int n = (int)*n_big;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int b = base + threadIdx.x;
        const uint32_t c = b < n ? (uint32_t)((big[b].box.w + kChunkPx - 1) / kChunkPx) : 0u;
        uint32_t incl = c;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = warp_sum[lane], si = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o) si += v;
            }
            warp_sum[lane] = si - s;
        }
        __syncthreads();
        const uint32_t off = carry + warp_sum[warp] + incl - c;
        if (b < n) chunk_start[b] = off;
        __syncthreads();
        if (threadIdx.x == 1023) carry = off + c;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        chunk_start[n] = carry;
        *n_chunks = carry;
    }
}

// queued triangles: persistent blocks claim chunks of kChunkPx candidate pixels
__global__ void __launch_bounds__(kRastThreads) k_rast_big(DevCam cam, SceneDev sc, unsigned long long *keys,
                                                            const BigTri *big, const uint32_t *n_big,
                                                            const uint32_t *chunk_start, const uint32_t *n_chunks,
                                                            uint32_t *cursor) {
    __shared__ float e[9];
    __shared__ float4 v[3];
    __shared__ int box[4];
    __shared__ float tn;
    __shared__ uint32_t claim[2];
    const uint32_t total = *n_chunks;
    const int nb = (int)*n_big;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t c = atomicAdd(cursor, 1u);
            int b = 0;
            if (c < total) {
                // last triangle whose chunks start at or before c
                int lo = 0, hi = nb - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (chunk_start[mid] <= c) lo = mid; else hi = mid - 1;
                }
                b = lo;
                const BigTri &B = big[b];
                e[0] = B.e0.x; e[1] = B.e0.y; e[2] = B.e0.z;
                e[3] = B.e1.x; e[4] = B.e1.y; e[5] = B.e1.z;
                e[6] = B.e2.x; e[7] = B.e2.y; e[8] = B.e2.z;
                box[0] = B.box.x; box[1] = B.box.y; box[2] = B.box.z; box[3] = B.box.w;
                tn = B.tn;
                const float4 *tp = sc.tris + 3 * (size_t)B.k;
                v[0] = __ldg(tp); v[1] = __ldg(tp + 1); v[2] = __ldg(tp + 2);
            }
            claim[0] = c;
            claim[1] = c < total ? c - chunk_start[b] : 0u;
        }
        __syncthreads();
        const uint32_t c = claim[0];
        if (c >= total) break;
        const int bw = box[2], npx = box[3];
        const int first = (int)claim[1] * kChunkPx;
        const int last = min(npx, first + kChunkPx);
        for (int w = first + threadIdx.x; w < last; w += kRastThreads) {
            const int q = w / bw, r = w - q * bw;
            const int i = box[0] + r, j = box[1] + q;
            if (edges_pass(e, i + 0.5f, j + 0.5f) && !occluded(keys, (size_t)j * cam.W + i, tn))
                test_pixel(cam, keys, i, j, v[0], v[1], v[2]);
        }
        __syncthreads();
    }
}

// closest hit per pixel -> colour, depth, normal, id (as the ray-cast producer writes them)
__global__ void __launch_bounds__(kRastThreads) k_rast_resolve(DevCam cam, DevParams p, SceneDev sc,
                                                                const unsigned long long *keys,
                                                                const int32_t *prim_k, float4 *color, float *depth,
                                                                float4 *normal, int32_t *prim) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= cam.W || j >= cam.H) return;
    const size_t q = (size_t)j * cam.W + i;
    const unsigned long long key = keys[q];
    if (key == ~0ull) {
        if (prim) prim[q] = -1;
        color[q] = make_float4(p.sky.x, p.sky.y, p.sky.z, 1.f);
        depth[q] = INFINITY;
        normal[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    HitRec h;
    h.t = __uint_as_float((uint32_t)(key >> 32));
    h.prim = (int)(uint32_t)key;
    h.k = __ldg(&prim_k[h.prim]);
    const float3 d = pixel_dir(cam, i + 0.5f, j + 0.5f);
    float3 n;
    const float3 col = shade(p, sc, h, d, n);
    if (prim) prim[q] = h.prim;
    color[q] = make_float4(col.x, col.y, col.z, 1.f);
    depth[q] = h.t * dot(d, cam.F);
    normal[q] = make_float4(n.x, n.y, n.z, 0.f);
}

// per triangle: its distance bound, and the sort key (the bound's bits: non-negative
// floats order as unsigned integers) with its index
__global__ void k_tri_near(DevCam cam, SceneDev sc, int n_tot, float *tnear, unsigned long long *skeys,
                           uint32_t *svals) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_tot) return;
    const float4 *tp = sc.tris + 3 * (size_t)k;
    const float tn = near_bound(cam, __ldg(tp), __ldg(tp + 1), __ldg(tp + 2));
    tnear[k] = tn;
    skeys[k] = (unsigned long long)__float_as_uint(tn);
    svals[k] = (uint32_t)k;
}

// inverse of the tree order: triangle id -> sorted index
__global__ void k_prim_index(const float4 *tris, int n, int32_t *prim_k) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) prim_k[__float_as_int(__ldg(&tris[3 * (size_t)k]).w)] = k;
}

}  // namespace

void launch_prim_index(const float4 *tris, int n, int32_t *prim_k, cudaStream_t st) {
    if (n > 0) {
        k_prim_index<<<(n + 255) / 256, 256, 0, st>>>(tris, n, prim_k);
        count_launches(1);
    }
}

// triangles of the depth-ordered batches: the nearest 1/32, then 1/32, 1/16, 1/8, 1/4
// and the farthest half; scenes under kSortedMin triangles run as one batch in scene
// order (the sort and the launches would cost more than they save)
constexpr int kBatches = 6;
constexpr int kSortedMin = 65536;
__host__ inline int batch_end(int b, int nb, int n) { return b + 1 >= nb ? n : (int)((long long)n >> (nb - 1 - b)); }

// Scratch of one call, from the context's stream-ordered pool.
size_t raster_scratch_bytes(int W, int H, int n_tot) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t n = (size_t)n_tot;
    const size_t t1 = (size_t)((W + 15) >> kHizShift1) * ((H + 15) >> kHizShift1);
    const size_t t2 = (size_t)((W + 127) >> kHizShift2) * ((H + 127) >> kHizShift2);
    return up(8 * (size_t)W * H) + up(sizeof(BigTri) * n) + up(4 * (n + 1)) + up(16 * kBatches) +
           up(4 * n) + 2 * up(8 * n) + 2 * up(4 * n) + up(4 * sort_pairs_scratch_ints(n_tot)) + up(4 * t1) +
           up(4 * t2);
}

cudaError_t launch_raster(const DevCam &cam, const DevParams &p, const SceneDev &sc, const int32_t *prim_k,
                          void *scratch, int sm_count, float4 *color, float *depth, float4 *normal, int32_t *prim,
                          cudaStream_t st) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int n_tot = sc.n_tris + sc.n_large;
    char *base = static_cast<char *>(scratch);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(base);
    base += up(8 * (size_t)cam.W * cam.H);
    BigTri *big = reinterpret_cast<BigTri *>(base);
    base += up(sizeof(BigTri) * (size_t)n_tot);
    uint32_t *chunk_start = reinterpret_cast<uint32_t *>(base);
    base += up(4 * ((size_t)n_tot + 1));
    uint32_t *counters = reinterpret_cast<uint32_t *>(base);   // per batch: n_big, n_chunks, cursor
    base += up(16 * kBatches);
    const size_t n = (size_t)n_tot;
    float *tnear = reinterpret_cast<float *>(base);
    base += up(4 * n);
    unsigned long long *skeys = reinterpret_cast<unsigned long long *>(base);
    base += up(8 * n);
    unsigned long long *skeys2 = reinterpret_cast<unsigned long long *>(base);
    base += up(8 * n);
    uint32_t *order = reinterpret_cast<uint32_t *>(base);
    base += up(4 * n);
    uint32_t *order2 = reinterpret_cast<uint32_t *>(base);
    base += up(4 * n);
    int *sort_scratch = reinterpret_cast<int *>(base);
    base += up(4 * sort_pairs_scratch_ints(n_tot));
    Hiz hiz;
    hiz.tw1 = (cam.W + 15) >> kHizShift1; hiz.th1 = (cam.H + 15) >> kHizShift1;
    hiz.tw2 = (cam.W + 127) >> kHizShift2; hiz.th2 = (cam.H + 127) >> kHizShift2;
    float *hiz1 = reinterpret_cast<float *>(base);
    base += up(4 * (size_t)hiz.tw1 * hiz.th1);
    float *hiz2 = reinterpret_cast<float *>(base);
    hiz.l1 = hiz1;
    hiz.l2 = hiz2;
    cudaError_t e = cudaMemsetAsync(keys, 0xFF, 8 * (size_t)cam.W * cam.H, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 16 * kBatches, st);
    if (e != cudaSuccess) return e;
    if (n_tot > 0) {
        // the triangles nearest first
        const int nbat = n_tot >= kSortedMin ? kBatches : 1;
        k_tri_near<<<(n_tot + 255) / 256, 256, 0, st>>>(cam, sc, n_tot, tnear, skeys, order);
        if (nbat > 1) sort_pairs_by_low_bits(skeys, order, skeys2, order2, n_tot, 32, sort_scratch, st);
        for (int bt = 0, b0 = 0; bt < nbat; bt++) {
            const int b1 = batch_end(bt, nbat, n_tot);
            if (b1 <= b0) continue;
            uint32_t *cb = counters + 4 * bt;
            // at least 32 warps per SM: groups of 32 triangles are split over several warps
            const int groups = (b1 - b0 + 31) / 32;
            const int split = std::min(16, std::max(1, (32 * sm_count + groups - 1) / groups));
            const int warps = groups * split;
            k_rast_small<<<(warps + kRastThreads / 32 - 1) / (kRastThreads / 32), kRastThreads, 0, st>>>(
                cam, sc, order + b0, b1 - b0, split, tnear, hiz, b0 > 0, keys, big, cb);
            k_big_chunks<<<1, 1024, 0, st>>>(big, cb, chunk_start, cb + 1);
            k_rast_big<<<4 * sm_count, kRastThreads, 0, st>>>(cam, sc, keys, big, cb, chunk_start, cb + 1, cb + 2);
            count_launches(3);
            b0 = b1;
            if (b0 < n_tot) {
                // the depth pyramid for the next batch
                k_hiz1<<<dim3(hiz.tw1, hiz.th1), 256, 0, st>>>(keys, cam.W, cam.H, hiz1, hiz.tw1);
                k_hiz2<<<dim3((hiz.tw2 + 15) / 16, (hiz.th2 + 15) / 16), dim3(16, 16), 0, st>>>(
                    hiz1, hiz.tw1, hiz.th1, hiz2, hiz.tw2, hiz.th2);
                count_launches(2);
            }
        }
        count_launches(1);
    }
    dim3 b(32, 8), g((cam.W + 31) / 32, (cam.H + 7) / 8);
    k_rast_resolve<<<g, b, 0, st>>>(cam, p, sc, keys, prim_k, color, depth, normal, prim);
    count_launches(1);
    return cudaGetLastError();
}

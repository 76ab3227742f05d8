// Device-built BVH of libdof (the acceleration structure whose build the paper
// counts in its ray-trace time, Section 4.2).
//
// LBVH after Karras, "Maximizing Parallelism in the Construction of BVHs, Octrees,
// and k-d Trees" (HPG 2012): 63-bit Morton codes of triangle centroids (21 bits per
// axis: scenes with a ground plane hundreds of metres wide still resolve centimetre
// detail), a stable LSD radix sort written here (8-bit digits, warp-matched ranks), one
// thread per internal node to find its key range and
// split (ties between equal codes broken by the sorted index), then a
// bottom-up box refit in which the second thread to reach a node merges its two
// children (atomic arrival counter, no waiting).  Nodes hold both child boxes so that
// traversal fetches one node per step.

#include "dof_internal.cuh"

namespace {

__device__ __forceinline__ int ord_of(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float float_of(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

__device__ __forceinline__ float3 vtx(const float *xyz, uint32_t i) {
    return make_float3(xyz[3 * (size_t)i], xyz[3 * (size_t)i + 1], xyz[3 * (size_t)i + 2]);
}

// centroids and their bounds (order-preserving int atomics); flags bad indices
__global__ void k_centroids(const float *xyz, uint32_t n_verts, const uint32_t *idx, uint32_t n,
                            float4 *cen, int *bounds, int *bad) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float3 c = make_float3(0.f, 0.f, 0.f);
    bool ok = t < n;
    if (ok) {
        uint32_t i0 = idx[3 * (size_t)t], i1 = idx[3 * (size_t)t + 1], i2 = idx[3 * (size_t)t + 2];
        if (i0 >= n_verts || i1 >= n_verts || i2 >= n_verts) {
            atomicExch(bad, 1);
            i0 = i1 = i2 = 0;
        }
        float3 a = vtx(xyz, i0), b = vtx(xyz, i1), d = vtx(xyz, i2);
        float3 lo = make_float3(fminf(a.x, fminf(b.x, d.x)), fminf(a.y, fminf(b.y, d.y)), fminf(a.z, fminf(b.z, d.z)));
        float3 hi = make_float3(fmaxf(a.x, fmaxf(b.x, d.x)), fmaxf(a.y, fmaxf(b.y, d.y)), fmaxf(a.z, fmaxf(b.z, d.z)));
        c = make_float3(0.5f * (lo.x + hi.x), 0.5f * (lo.y + hi.y), 0.5f * (lo.z + hi.z));
        cen[t] = make_float4(c.x, c.y, c.z, fmaxf(hi.x - lo.x, fmaxf(hi.y - lo.y, hi.z - lo.z)));
    }
    // block reduction of min/max through warp shuffles
    float v[6] = {c.x, c.y, c.z, c.x, c.y, c.z};
    if (!ok) { v[0] = v[1] = v[2] = INFINITY; v[3] = v[4] = v[5] = -INFINITY; }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 6; k++) {
            float w = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = k < 3 ? fminf(v[k], w) : fmaxf(v[k], w);
        }
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; k++) atomicMin(&bounds[k], ord_of(v[k]));
        for (int k = 3; k < 6; k++) atomicMax(&bounds[k], ord_of(v[k]));
    }
}

// threshold of a "large" triangle: its largest box extent above 1/16 of the largest
// centroid extent of the scene (a ground plane, a wall spanning the scene)
__device__ __forceinline__ float big_threshold(const int *bounds) {
    float e = 0.f;
    for (int k = 0; k < 3; k++) e = fmaxf(e, float_of(bounds[3 + k]) - float_of(bounds[k]));
    return e * (1.f / 16.f);
}

// count the large triangles and the centroid bounds of the others
__global__ void k_classify(const float4 *cen, uint32_t n, const int *bounds, int *n_big, int *small_bounds) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float thr = big_threshold(bounds);
    bool ok = t < n;
    float4 c = ok ? cen[t] : make_float4(0.f, 0.f, 0.f, 0.f);
    bool big = ok && c.w > thr;
    bool small = ok && !big;
    unsigned nb = __popc(__ballot_sync(0xffffffffu, big));
    float v[6] = {c.x, c.y, c.z, c.x, c.y, c.z};
    if (!small) { v[0] = v[1] = v[2] = INFINITY; v[3] = v[4] = v[5] = -INFINITY; }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 6; k++) {
            float w = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = k < 3 ? fminf(v[k], w) : fmaxf(v[k], w);
        }
    if ((threadIdx.x & 31) == 0) {
        if (nb) atomicAdd(n_big, (int)nb);
        for (int k = 0; k < 3; k++) atomicMin(&small_bounds[k], ord_of(v[k]));
        for (int k = 3; k < 6; k++) atomicMax(&small_bounds[k], ord_of(v[k]));
    }
}

// spread the low 21 bits of v to every third bit
__device__ __forceinline__ unsigned long long expand21(uint32_t v) {
    unsigned long long x = v & 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

// Morton keys over the centroid bounds `bounds`; with separate_big, large triangles
// (classified against `all_bounds`) get the key ~0 and sort after every other one
__global__ void k_morton(const float4 *cen, uint32_t n, const int *bounds, const int *all_bounds, int separate_big,
                         unsigned long long *keys, uint32_t *vals) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    vals[t] = t;
    if (separate_big && cen[t].w > big_threshold(all_bounds)) {
        keys[t] = ~0ull;
        return;
    }
    float lo[3], ext[3];
    for (int k = 0; k < 3; k++) {
        lo[k] = float_of(bounds[k]);
        ext[k] = float_of(bounds[3 + k]) - lo[k];
    }
    float4 c = cen[t];
    float p[3] = {c.x, c.y, c.z};
    uint32_t q[3];
    for (int k = 0; k < 3; k++) {
        float u = ext[k] > 0.f ? (p[k] - lo[k]) / ext[k] : 0.f;
        q[k] = (uint32_t)fminf(fmaxf(u * 2097152.f, 0.f), 2097151.f);
    }
    keys[t] = (expand21(q[0]) << 2) | (expand21(q[1]) << 1) | expand21(q[2]);
}

// sorted triangles: v0 (w = original id), v1, v2 (w = material)
__global__ void k_sorted_tris(const float *xyz, const uint32_t *idx, const uint32_t *mat, uint32_t n,
                              uint32_t n_verts, const uint32_t *order, float4 *tris) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t t = order[k];
    uint32_t i0 = idx[3 * (size_t)t], i1 = idx[3 * (size_t)t + 1], i2 = idx[3 * (size_t)t + 2];
    if (i0 >= n_verts || i1 >= n_verts || i2 >= n_verts) i0 = i1 = i2 = 0;
    float3 a = vtx(xyz, i0), b = vtx(xyz, i1), c = vtx(xyz, i2);
    tris[3 * (size_t)k] = make_float4(a.x, a.y, a.z, __int_as_float((int)t));
    tris[3 * (size_t)k + 1] = make_float4(b.x, b.y, b.z, 0.f);
    tris[3 * (size_t)k + 2] = make_float4(c.x, c.y, c.z, __int_as_float(mat ? (int)mat[t] : 0));
}

// common-prefix length of sorted keys i and j, ties broken by index (Karras 2012)
__device__ __forceinline__ int delta(const unsigned long long *keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    unsigned long long a = keys[i], b = keys[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz(i ^ j);
}

// one thread per internal node: its range, split and children; parent links.
// child refs: >= 0 internal, < 0 leaf ~k
__global__ void k_karras(const unsigned long long *keys, int n, int4 *child, int *parent_node, int *parent_leaf, int *bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(keys, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int g = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    if (lo < 0 || hi > n - 1 || g < lo || g + 1 > hi) {   // cannot happen for a valid key order
        atomicExch(bad, 2);
        child[i] = make_int4(~0, ~0, 0, 0);
        return;
    }
    int left = (lo == g) ? ~g : g;
    int right = (hi == g + 1) ? ~(g + 1) : g + 1;
    child[i] = make_int4(left, right, 0, 0);
    if (left < 0) parent_leaf[~left] = i; else parent_node[left] = i;
    if (right < 0) parent_leaf[~right] = i; else parent_node[right] = i;
    if (i == 0) parent_node[0] = -1;
}

__device__ __forceinline__ void tri_box(const float4 *tris, int k, float3 &lo, float3 &hi) {
    float4 a = tris[3 * (size_t)k], b = tris[3 * (size_t)k + 1], c = tris[3 * (size_t)k + 2];
    lo = make_float3(fminf(a.x, fminf(b.x, c.x)), fminf(a.y, fminf(b.y, c.y)), fminf(a.z, fminf(b.z, c.z)));
    hi = make_float3(fmaxf(a.x, fmaxf(b.x, c.x)), fmaxf(a.y, fmaxf(b.y, c.y)), fmaxf(a.z, fmaxf(b.z, c.z)));
}

// bottom-up refit: each leaf walks towards the root; the second arrival at a node
// merges both children's boxes (written before the first arrival's fence).
__global__ void k_refit(const float4 *tris, int n, const int4 *child, const int *parent_node,
                        const int *parent_leaf, float4 *box_lo, float4 *box_hi, int *arrivals,
                        BvhNode *nodes, int *bad) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float3 lo, hi;
    tri_box(tris, k, lo, hi);
    // leaf boxes are stored after the n-1 internal ones
    box_lo[n - 1 + k] = make_float4(lo.x, lo.y, lo.z, 0.f);
    box_hi[n - 1 + k] = make_float4(hi.x, hi.y, hi.z, 0.f);
    __threadfence();
    int p = parent_leaf[k];
    for (int level = 0; p >= 0; level++) {
        if (p >= n - 1 || level > 160) { atomicExch(bad, 3); return; }
        if (atomicAdd(&arrivals[p], 1) == 0) return;   // the sibling finishes this node
        __threadfence();
        int4 ch = child[p];
        if (ch.x >= n - 1 || ch.y >= n - 1 || (ch.x < 0 && ~ch.x >= n) || (ch.y < 0 && ~ch.y >= n)) {
            atomicExch(bad, 3);
            return;
        }
        int s0 = ch.x >= 0 ? ch.x : n - 1 + ~ch.x;
        int s1 = ch.y >= 0 ? ch.y : n - 1 + ~ch.y;
        float4 l0 = __ldcg(&box_lo[s0]), h0 = __ldcg(&box_hi[s0]);
        float4 l1 = __ldcg(&box_lo[s1]), h1 = __ldcg(&box_hi[s1]);
        BvhNode nd;
        nd.a = make_float4(l0.x, l0.y, l0.z, h0.x);
        nd.b = make_float4(h0.y, h0.z, l1.x, l1.y);
        nd.c = make_float4(l1.z, h1.x, h1.y, h1.z);
        nd.r = make_int4(ch.x, ch.y, 0, 0);
        nodes[p] = nd;
        box_lo[p] = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f);
        box_hi[p] = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f);
        __threadfence();
        p = parent_node[p];
    }
}

// half the surface area of a box
__device__ __forceinline__ float half_area(float4 lo, float4 hi) {
    float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

// Tree rotations (Kensler, "Tree Rotations for Improving Bounding Volume Hierarchies",
// 2008), one bottom-up pass synchronised like the refit: at each internal node p with
// children L and R, swapping R with a child of L (or L with a child of R) changes the
// box of one child only, so the swap that shrinks that child's surface area the most is
// made, when it shrinks it by more than 2^-16 of p's area.  Every subtree keeps its
// leaves and every box is the exact union of its children's, so the closest hit of a ray
// is unchanged; the parents of the two moved subtrees are updated.
__device__ __forceinline__ void node_child(const BvhNode &nd, int c, float4 &lo, float4 &hi, int &ref) {
    if (c == 0) {
        lo = make_float4(nd.a.x, nd.a.y, nd.a.z, 0.f); hi = make_float4(nd.a.w, nd.b.x, nd.b.y, 0.f); ref = nd.r.x;
    } else {
        lo = make_float4(nd.b.z, nd.b.w, nd.c.x, 0.f); hi = make_float4(nd.c.y, nd.c.z, nd.c.w, 0.f); ref = nd.r.y;
    }
}

__device__ __forceinline__ BvhNode make_node(float4 l0, float4 h0, int r0, float4 l1, float4 h1, int r1) {
    BvhNode nd;
    nd.a = make_float4(l0.x, l0.y, l0.z, h0.x);
    nd.b = make_float4(h0.y, h0.z, l1.x, l1.y);
    nd.c = make_float4(l1.z, h1.x, h1.y, h1.z);
    nd.r = make_int4(r0, r1, 0, 0);
    return nd;
}

__device__ __forceinline__ float union_area(float4 l0, float4 h0, float4 l1, float4 h1) {
    return half_area(make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f),
                     make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f));
}

__device__ __forceinline__ void set_parent(int ref, int p, int n, int *parent_node, int *parent_leaf, int *bad) {
    if (ref < 0 ? ~ref >= n : ref >= n - 1) { atomicExch(bad, 7); return; }
    if (ref < 0) parent_leaf[~ref] = p;
    else parent_node[ref] = p;
}

// a node as other threads of the pass last wrote it (from L2, not a stale L1 line)
__device__ __forceinline__ BvhNode ld_node_cg(const BvhNode *nd) {
    const float4 *q = reinterpret_cast<const float4 *>(nd);
    BvhNode o;
    o.a = __ldcg(q);
    o.b = __ldcg(q + 1);
    o.c = __ldcg(q + 2);
    o.r = __ldcg(reinterpret_cast<const int4 *>(q + 3));
    return o;
}

__global__ void k_rotate(int n, BvhNode *nodes, int *parent_node, int *parent_leaf, int *arrivals, int *bad) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int p = __ldcg(&parent_leaf[k]);
    for (int level = 0; p >= 0; level++) {
        if (p >= n - 1 || level > 160) { atomicExch(bad, 7); return; }
        __threadfence();
        if (atomicAdd(&arrivals[p], 1) == 0) return;   // the sibling finishes this node
        __threadfence();
        const BvhNode np = ld_node_cg(&nodes[p]);
        float4 lL, hL, lR, hR;
        int L, R;
        node_child(np, 0, lL, hL, L);
        node_child(np, 1, lR, hR, R);
        const float areaL = half_area(lL, hL), areaR = half_area(lR, hR);
        const float thresh = union_area(lL, hL, lR, hR) * (1.f / 65536.f);
        float best = thresh;
        int kind = -1;                      // 0, 1: R with a child of L; 2, 3: L with a child of R
        BvhNode nL, nR;
        float4 la, ha, lb, hb, lc, hc, ld, hd;
        int ra = 0, rb = 0, rc = 0, rd = 0;
        if (L >= 0) {
            if (L >= n - 1) { atomicExch(bad, 7); return; }
            nL = ld_node_cg(&nodes[L]);
            node_child(nL, 0, la, ha, ra);
            node_child(nL, 1, lb, hb, rb);
            const float g0 = areaL - union_area(lR, hR, lb, hb);   // R <-> LL: L = (R, LR)
            const float g1 = areaL - union_area(la, ha, lR, hR);   // R <-> LR: L = (LL, R)
            if (g0 > best) { best = g0; kind = 0; }
            if (g1 > best) { best = g1; kind = 1; }
        }
        if (R >= 0) {
            if (R >= n - 1) { atomicExch(bad, 7); return; }
            nR = ld_node_cg(&nodes[R]);
            node_child(nR, 0, lc, hc, rc);
            node_child(nR, 1, ld, hd, rd);
            const float g2 = areaR - union_area(lL, hL, ld, hd);   // L <-> RL: R = (L, RR)
            const float g3 = areaR - union_area(lc, hc, lL, hL);   // L <-> RR: R = (RL, L)
            if (g2 > best) { best = g2; kind = 2; }
            if (g3 > best) { best = g3; kind = 3; }
        }
        if (kind == 0 || kind == 1) {
            // the child of L that moves up to p (m) and the one that stays with R
            const float4 lm = kind == 0 ? la : lb, hm = kind == 0 ? ha : hb;
            const int rm = kind == 0 ? ra : rb;
            const float4 ls = kind == 0 ? lb : la, hs = kind == 0 ? hb : ha;
            const int rs = kind == 0 ? rb : ra;
            const BvhNode newL = kind == 0 ? make_node(lR, hR, R, ls, hs, rs) : make_node(ls, hs, rs, lR, hR, R);
            float4 lN, hN;
            int dummy;
            node_child(newL, 0, lN, hN, dummy);
            float4 l2, h2;
            node_child(newL, 1, l2, h2, dummy);
            lN = make_float4(fminf(lN.x, l2.x), fminf(lN.y, l2.y), fminf(lN.z, l2.z), 0.f);
            hN = make_float4(fmaxf(hN.x, h2.x), fmaxf(hN.y, h2.y), fmaxf(hN.z, h2.z), 0.f);
            nodes[L] = newL;
            nodes[p] = make_node(lN, hN, L, lm, hm, rm);
            set_parent(R, L, n, parent_node, parent_leaf, bad);
            set_parent(rm, p, n, parent_node, parent_leaf, bad);
        } else if (kind == 2 || kind == 3) {
            const float4 lm = kind == 2 ? lc : ld, hm = kind == 2 ? hc : hd;
            const int rm = kind == 2 ? rc : rd;
            const float4 ls = kind == 2 ? ld : lc, hs = kind == 2 ? hd : hc;
            const int rs = kind == 2 ? rd : rc;
            const BvhNode newR = kind == 2 ? make_node(lL, hL, L, ls, hs, rs) : make_node(ls, hs, rs, lL, hL, L);
            float4 lN, hN, l2, h2;
            int dummy;
            node_child(newR, 0, lN, hN, dummy);
            node_child(newR, 1, l2, h2, dummy);
            lN = make_float4(fminf(lN.x, l2.x), fminf(lN.y, l2.y), fminf(lN.z, l2.z), 0.f);
            hN = make_float4(fmaxf(hN.x, h2.x), fmaxf(hN.y, h2.y), fmaxf(hN.z, h2.z), 0.f);
            nodes[R] = newR;
            nodes[p] = make_node(lm, hm, rm, lN, hN, R);
            set_parent(L, R, n, parent_node, parent_leaf, bad);
            set_parent(rm, p, n, parent_node, parent_leaf, bad);
        }
        __threadfence();
        p = __ldcg(&parent_node[p]);
    }
}

// Structure check of the finished binary tree, before any traversal relies on it: every
// child reference in range (internal nodes 0 .. n_nodes - 1, leaves ~0 .. ~(n_tree - 1)),
// and every internal node except the root, and every leaf, referenced by exactly one
// internal node, the root by none.  Nodes on a cycle would take their one reference from
// inside the cycle, so none is reachable from the root: a traversal from the root visits
// each node at most once and reads only in-range nodes and triangles.  The parents are
// recorded from the same references (parent_node / parent_leaf, -1 beforehand), so the
// depth that k_depth then walks up from every leaf is the depth of the tree the traversal
// reads: a leaf below a cycle walks to k_depth's cap, which the traversal stack rejects.
__global__ void k_tree_refs(const BvhNode *nodes, int n_nodes, int n_tree, int *ref_node, int *ref_leaf,
                            int *parent_node, int *parent_leaf, int *bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_nodes) return;
    const int4 r = nodes[i].r;
    const int c[2] = {r.x, r.y};
#pragma unroll
    for (int e = 0; e < 2; e++) {
        if (c[e] >= 0 ? c[e] >= n_nodes : ~c[e] >= n_tree) { atomicExch(bad, 8); continue; }
        atomicAdd(c[e] >= 0 ? &ref_node[c[e]] : &ref_leaf[~c[e]], 1);
        if (c[e] >= 0) parent_node[c[e]] = i;
        else parent_leaf[~c[e]] = i;
    }
}
__global__ void k_tree_counts(int n_nodes, int n_tree, int root, const int *ref_node, const int *ref_leaf, int *bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (root < 0 || root >= n_nodes)) atomicExch(bad, 9);
    if (i < n_nodes && ref_node[i] != (i == root ? 0 : 1)) atomicExch(bad, 9);
    if (i < n_tree && ref_leaf[i] != 1) atomicExch(bad, 9);
}

// tree depth (levels from the root to the deepest leaf, root = 1)
__global__ void k_depth(int n, const int *parent_node, const int *parent_leaf, int *depth) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int d = 1, p = parent_leaf[k];
    while (p >= 0 && d < 1000) { d++; p = parent_node[p]; }
    atomicMax(depth, d);
}


// ---------------------------------------------------------------------------
// PLOC (Meister and Bittner, "Parallel Locally-Ordered Clustering for Bounding
// Volume Hierarchy Construction", TVCG 2018): clusters start as the Morton-sorted
// leaves; each finds its nearest neighbour within +-kPlocRadius positions by the
// surface area of the merged box; mutual nearest neighbours merge into a new node;
// the cluster array is compacted (order preserved) and the steps repeat.
// ---------------------------------------------------------------------------

__global__ void k_ploc_init(const float4 *tris, int m, int *cid, float4 *clo, float4 *chi) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    float3 lo, hi;
    tri_box(tris, k, lo, hi);
    cid[k] = ~k;
    clo[k] = make_float4(lo.x, lo.y, lo.z, 0.f);
    chi[k] = make_float4(hi.x, hi.y, hi.z, 0.f);
}

// nearest neighbour by merged area; ties to the smaller index (symmetric cost, so the
// globally cheapest pair is always mutual and every round merges at least once)
__global__ void k_ploc_nn(int count, int radius, const float4 *clo, const float4 *chi, int *nn) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float4 lo = clo[i], hi = chi[i];
    float best = INFINITY;
    int bj = -1;
    int j0 = max(0, i - radius), j1 = min(count - 1, i + radius);
    for (int j = j0; j <= j1; j++) {
        if (j == i) continue;
        float4 l2 = clo[j], h2 = chi[j];
        float a = half_area(make_float4(fminf(lo.x, l2.x), fminf(lo.y, l2.y), fminf(lo.z, l2.z), 0.f),
                            make_float4(fmaxf(hi.x, h2.x), fmaxf(hi.y, h2.y), fmaxf(hi.z, h2.z), 0.f));
        if (a < best) { best = a; bj = j; }
    }
    nn[i] = bj;
}

// mutual pairs merge: the lower position creates the node and keeps the merged
// cluster, the higher one drops out
__global__ void k_ploc_merge(int count, int *cid, float4 *clo, float4 *chi, const int *nn, int *keep,
                             int *node_count, BvhNode *nodes, int *parent_node, int *parent_leaf, int n_nodes,
                             int *bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    int j = nn[i];
    bool mutual = j >= 0 && nn[j] == i;
    if (!mutual) { keep[i] = 1; return; }
    if (i > j) { keep[i] = 0; return; }
    int id = atomicAdd(node_count, 1);
    if (id >= n_nodes) { atomicExch(bad, 4); keep[i] = 1; return; }
    int a = cid[i], b = cid[j];
    float4 l0 = clo[i], h0 = chi[i], l1 = clo[j], h1 = chi[j];
    BvhNode nd;
    nd.a = make_float4(l0.x, l0.y, l0.z, h0.x);
    nd.b = make_float4(h0.y, h0.z, l1.x, l1.y);
    nd.c = make_float4(l1.z, h1.x, h1.y, h1.z);
    nd.r = make_int4(a, b, 0, 0);
    nodes[id] = nd;
    if (a < 0) parent_leaf[~a] = id; else parent_node[a] = id;
    if (b < 0) parent_leaf[~b] = id; else parent_node[b] = id;
    cid[i] = id;
    clo[i] = make_float4(fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z), 0.f);
    chi[i] = make_float4(fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z), 0.f);
    keep[i] = 1;
}

__global__ void k_ploc_scatter(int count, const int *keep, const int *pos, const int *cid, const float4 *clo,
                               const float4 *chi, int *cid2, float4 *clo2, float4 *chi2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count || !keep[i]) return;
    int o = pos[i];
    cid2[o] = cid[i];
    clo2[o] = clo[i];
    chi2[o] = chi[i];
}


// ---------------------------------------------------------------------------
// Collapse of the binary tree into 4-wide nodes, top-down one level per launch:
// a 4-wide node starts from the two children of its binary node and opens its
// largest-area internal child until it holds four children (or only leaves).  The
// child boxes are stored as the binary tree holds them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bin_child(const BvhNode &nd, int c, float3 &lo, float3 &hi, int &ref) {
    if (c == 0) {
        lo = make_float3(nd.a.x, nd.a.y, nd.a.z); hi = make_float3(nd.a.w, nd.b.x, nd.b.y); ref = nd.r.x;
    } else {
        lo = make_float3(nd.b.z, nd.b.w, nd.c.x); hi = make_float3(nd.c.y, nd.c.z, nd.c.w); ref = nd.r.y;
    }
}

__global__ void k_collapse(const BvhNode *nodes, int n_bin, const int2 *fin, int n_in, Bvh4Node *out4, int max4,
                           int *n4, int2 *fout, int *n_out, int *bad) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_in) return;
    int w4 = fin[t].x, b = fin[t].y;
    if (b < 0 || b >= n_bin || w4 < 0 || w4 >= max4) { atomicExch(bad, 5); return; }
    float3 lo[4], hi[4];
    int ref[4], cnt = 2;
    BvhNode nd = nodes[b];
    bin_child(nd, 0, lo[0], hi[0], ref[0]);
    bin_child(nd, 1, lo[1], hi[1], ref[1]);
    while (cnt < 4) {
        int best = -1;
        float ba = -1.f;
        for (int e = 0; e < cnt; e++) {
            if (ref[e] < 0) continue;
            float dx = hi[e].x - lo[e].x, dy = hi[e].y - lo[e].y, dz = hi[e].z - lo[e].z;
            float a = dx * dy + dy * dz + dz * dx;
            if (a > ba) { ba = a; best = e; }
        }
        if (best < 0) break;
        if (ref[best] >= n_bin) { atomicExch(bad, 5); return; }
        BvhNode c = nodes[ref[best]];
        bin_child(c, 0, lo[best], hi[best], ref[best]);
        bin_child(c, 1, lo[cnt], hi[cnt], ref[cnt]);
        cnt++;
    }
    int nint = 0;
    for (int e = 0; e < cnt; e++) nint += ref[e] >= 0;
    int base = nint ? atomicAdd(n4, nint) : 0;
    if (base + nint > max4) { atomicExch(bad, 6); return; }
    int fo = nint ? atomicAdd(n_out, nint) : 0;
    if (fo + nint > max4) { atomicExch(bad, 6); return; }
    float L[3][4], Hh[3][4];
    int R[4];
    int k = 0;
    for (int e = 0; e < 4; e++) {
        if (e < cnt) {
            L[0][e] = lo[e].x;
            L[1][e] = lo[e].y;
            L[2][e] = lo[e].z;
            Hh[0][e] = hi[e].x;
            Hh[1][e] = hi[e].y;
            Hh[2][e] = hi[e].z;
            if (ref[e] >= 0) {
                R[e] = base + k;
                fout[fo + k] = make_int2(base + k, ref[e]);
                k++;
            } else {
                R[e] = ref[e];
            }
        } else {
            L[0][e] = L[1][e] = L[2][e] = 0.f;
            Hh[0][e] = Hh[1][e] = Hh[2][e] = 0.f;
            R[e] = kEmptyChild;
        }
    }
    Bvh4Node o;
    o.lox = make_float4(L[0][0], L[0][1], L[0][2], L[0][3]);
    o.hix = make_float4(Hh[0][0], Hh[0][1], Hh[0][2], Hh[0][3]);
    o.loy = make_float4(L[1][0], L[1][1], L[1][2], L[1][3]);
    o.hiy = make_float4(Hh[1][0], Hh[1][1], Hh[1][2], Hh[1][3]);
    o.loz = make_float4(L[2][0], L[2][1], L[2][2], L[2][3]);
    o.hiz = make_float4(Hh[2][0], Hh[2][1], Hh[2][2], Hh[2][3]);
    o.ref = make_int4(R[0], R[1], R[2], R[3]);
    o.pad = make_int4(0, 0, 0, 0);
    out4[w4] = o;
}

// ---------------------------------------------------------------------------
// device exclusive scan (int) and stable LSD radix sort (64-bit keys, 32-bit values)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

// exclusive prefix of v over the 256 threads of the block; *total = the block's sum
__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_sums, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    int wpre = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < kScanThreads / 32; k++) {
        const int s = warp_sums[k];
        if (k < w) wpre += s;
        tot += s;
    }
    __syncthreads();
    total = tot;
    return wpre + incl - v;
}

// tile-local exclusive prefix of in[0..n) into out, and each tile's sum into sums
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int *in, int *out, int n, int *sums) {
    __shared__ int ws[kScanThreads / 32];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int tot;
    int pre = block_exclusive_scan(s, ws, tot);
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < n) out[base + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// exclusive prefix of sums[0..nb) in place, one block (each thread a consecutive chunk)
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int *sums, int nb) {
    __shared__ int ws[kScanThreads / 32];
    const int chunk = (nb + kScanThreads - 1) / kScanThreads;
    const int b0 = threadIdx.x * chunk;
    int s = 0;
    for (int k = 0; k < chunk; k++)
        if (b0 + k < nb) s += sums[b0 + k];
    int tot;
    int pre = block_exclusive_scan(s, ws, tot);
    for (int k = 0; k < chunk; k++)
        if (b0 + k < nb) {
            const int v = sums[b0 + k];
            sums[b0 + k] = pre;
            pre += v;
        }
}

__global__ void k_scan_add(int *out, int n, const int *sums) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / kScanTile];
}

// out[i] = in[0] + ... + in[i-1]; sums holds ceil(n / 2048) ints
void device_exclusive_scan(const int *in, int *out, int n, int *sums, cudaStream_t st) {
    if (n <= 0) return;
    const int nb = (n + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<nb, kScanThreads, 0, st>>>(in, out, n, sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, nb);
    k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(out, n, sums);
}

constexpr int kSortThreads = 256, kSortRounds = 8, kSortTile = kSortThreads * kSortRounds, kSortBins = 256;

// per block of 2048 keys: the count of each 8-bit digit at `shift`, digit-major
__global__ void __launch_bounds__(kSortThreads) k_rs_hist(const unsigned long long *keys, int n, int shift, int *hist,
                                                          int nblocks) {
    __shared__ int h[kSortBins];
    h[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortRounds; r++) {
        const long long idx = (long long)blockIdx.x * kSortTile + r * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(int)((keys[idx] >> shift) & 255ull)], 1);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of a block's 2048 keys by their digit: offs[d * nblocks + b] is where
// digit d of block b starts (exclusive scan of the histograms).  The block takes its keys
// in 8 rounds of 256 in index order; within a round a key's place among equal digits is
// its rank in its warp (lanes with the same digit, __match_any_sync) plus the counts of
// the lower warps, and the digit's running offset carries across rounds.
__global__ void __launch_bounds__(kSortThreads) k_rs_scatter(const unsigned long long *keys, const uint32_t *vals,
                                                             unsigned long long *keys_out, uint32_t *vals_out, int n,
                                                             int shift, const int *offs, int nblocks) {
    __shared__ int run[kSortBins];
    __shared__ int wcount[kSortThreads / 32][kSortBins];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    run[tid] = offs[tid * nblocks + blockIdx.x];
    for (int r = 0; r < kSortRounds; r++) {
        const long long idx = (long long)blockIdx.x * kSortTile + r * kSortThreads + tid;
        const bool valid = idx < n;
        const unsigned long long key = valid ? keys[idx] : 0ull;
        const uint32_t val = valid ? vals[idx] : 0u;
        const int d = valid ? (int)((key >> shift) & 255ull) : kSortBins;
#pragma unroll
        for (int k = 0; k < kSortBins / 32; k++) wcount[w][lane + 32 * k] = 0;
        __syncwarp();
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt);
        if (valid && lane == __ffs(peers) - 1) wcount[w][d] = __popc(peers);
        __syncthreads();
        // per digit (thread tid = digit tid): exclusive prefix of the warps' counts
        int acc = 0;
#pragma unroll
        for (int k = 0; k < kSortThreads / 32; k++) {
            const int c = wcount[k][tid];
            wcount[k][tid] = acc;
            acc += c;
        }
        __syncthreads();
        if (valid) {
            const int pos = run[d] + wcount[w][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
        run[tid] += acc;
        __syncthreads();
    }
}

// Stable sort of (keys, vals) by the key's low `bits` bits (a multiple of 16: an even
// number of 8-bit passes); the result ends in (keys, vals), (keys2, vals2) and hist are
// scratch (hist: 256 * ceil(n / 2048) ints, sums: ceil(256 * ceil(n / 2048) / 2048) ints).
void device_radix_sort_pairs(unsigned long long *keys, uint32_t *vals, unsigned long long *keys2, uint32_t *vals2,
                             int n, int *hist, int *sums, cudaStream_t st, int bits = 64) {
    if (n <= 1) return;
    const int nb = (n + kSortTile - 1) / kSortTile;
    unsigned long long *ki = keys, *ko = keys2;
    uint32_t *vi = vals, *vo = vals2;
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<nb, kSortThreads, 0, st>>>(ki, n, shift, hist, nb);
        device_exclusive_scan(hist, hist, kSortBins * nb, sums, st);
        k_rs_scatter<<<nb, kSortThreads, 0, st>>>(ki, vi, ko, vo, n, shift, hist, nb);
        unsigned long long *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
    }
    // an even number of passes: the sorted data are back in (keys, vals)
}

}  // namespace

size_t sort_pairs_scratch_ints(int n) {
    const size_t nbk = (size_t)(n + kSortTile - 1) / kSortTile;
    const size_t nh = (size_t)kSortBins * nbk;
    return nh + (nh + kScanTile - 1) / kScanTile + 1;
}

void sort_pairs_by_low_bits(unsigned long long *keys, uint32_t *vals, unsigned long long *keys2, uint32_t *vals2,
                            int n, int bits, int *scratch, cudaStream_t st) {
    const size_t nh = (size_t)kSortBins * ((n + kSortTile - 1) / kSortTile);
    device_radix_sort_pairs(keys, vals, keys2, vals2, n, scratch, scratch + nh, st, bits);
}

static inline unsigned blocks_for(size_t n, int b) { return (unsigned)((n + b - 1) / b); }

// PLOC hierarchy over the m sorted tree triangles; writes nodes, parents, *root
static int ploc_build(DofScene *s, int m, int radius, int *pnode, int *pleaf, int *ibuf, int *root, cudaStream_t st) {
    const int B = 256;
    int rc = DOF_OK;
    int *cid[2] = {nullptr, nullptr}, *nn = nullptr, *keep = nullptr, *pos = nullptr, *cnt = nullptr;
    float4 *clo[2] = {nullptr, nullptr}, *chi[2] = {nullptr, nullptr};
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    auto ck = [&](cudaError_t e, const char *w) { if (rc == DOF_OK && e != cudaSuccess) rc = dof_cuda_check(e, w); };
    for (int k = 0; k < 2; k++) {
        ck(cudaMalloc(&cid[k], sizeof(int) * m), "ploc");
        ck(cudaMalloc(&clo[k], sizeof(float4) * m), "ploc");
        ck(cudaMalloc(&chi[k], sizeof(float4) * m), "ploc");
    }
    ck(cudaMalloc(&nn, sizeof(int) * m), "ploc");
    ck(cudaMalloc(&keep, sizeof(int) * m), "ploc");
    ck(cudaMalloc(&pos, sizeof(int) * m), "ploc");
    ck(cudaMalloc(&cnt, sizeof(int)), "ploc");
    tmp_bytes = sizeof(int) * (size_t)((m + kScanTile - 1) / kScanTile + 1);
    ck(cudaMalloc(&tmp, tmp_bytes), "ploc scan temp");
    if (rc == DOF_OK) {
        ck(cudaMemsetAsync(cnt, 0, sizeof(int), st), "ploc");
        k_ploc_init<<<blocks_for(m, B), B, 0, st>>>(s->tris, m, cid[0], clo[0], chi[0]);
        int count = m, cur = 0;
        for (int round = 0; count > 1 && rc == DOF_OK; round++) {
            if (round > 100000) { rc = dof_set_error(DOF_ERR_DEVICE_CHECK, "PLOC made no progress"); break; }
            k_ploc_nn<<<blocks_for(count, B), B, 0, st>>>(count, radius, clo[cur], chi[cur], nn);
            k_ploc_merge<<<blocks_for(count, B), B, 0, st>>>(count, cid[cur], clo[cur], chi[cur], nn, keep, cnt,
                                                            s->nodes, pnode, pleaf, m - 1, ibuf + 6);
            device_exclusive_scan(keep, pos, count, static_cast<int *>(tmp), st);
            k_ploc_scatter<<<blocks_for(count, B), B, 0, st>>>(count, keep, pos, cid[cur], clo[cur], chi[cur],
                                                              cid[cur ^ 1], clo[cur ^ 1], chi[cur ^ 1]);
            int last[2];
            ck(cudaMemcpyAsync(&last[0], pos + count - 1, sizeof(int), cudaMemcpyDeviceToHost, st), "ploc count");
            ck(cudaMemcpyAsync(&last[1], keep + count - 1, sizeof(int), cudaMemcpyDeviceToHost, st), "ploc count");
            ck(cudaStreamSynchronize(st), "ploc round");
            int next = last[0] + last[1];
            if (rc == DOF_OK && next >= count) { rc = dof_set_error(DOF_ERR_DEVICE_CHECK, "PLOC round merged nothing"); break; }
            count = next;
            cur ^= 1;
        }
        if (rc == DOF_OK) {
            ck(cudaMemcpyAsync(root, cid[cur], sizeof(int), cudaMemcpyDeviceToHost, st), "ploc root");
            ck(cudaStreamSynchronize(st), "ploc root");
            if (rc == DOF_OK && *root >= 0) {
                int minus1 = -1;
                ck(cudaMemcpy(pnode + *root, &minus1, sizeof(int), cudaMemcpyHostToDevice), "ploc root parent");
            }
        }
    }
    for (int k = 0; k < 2; k++) { cudaFree(cid[k]); cudaFree(clo[k]); cudaFree(chi[k]); }
    cudaFree(nn); cudaFree(keep); cudaFree(pos); cudaFree(cnt); cudaFree(tmp);
    return rc;
}

// 4-wide tree from the binary one (root `root`, n_bin internal nodes); sets
// s->nodes4 / root4 / n_nodes4 / depth4 (nodes4 stays null for a one-leaf tree)
static int collapse4(DofScene *s, int root, int n_bin, int *ibuf, cudaStream_t st) {
    const int B = 256;
    int rc = DOF_OK;
    s->root4 = root;
    s->n_nodes4 = 0;
    s->depth4 = 0;
    if (root < 0 || n_bin < 1) return DOF_OK;
    Bvh4Node *big = nullptr;
    int2 *fr[2] = {nullptr, nullptr};
    int *cnt = nullptr;
    auto ck = [&](cudaError_t e, const char *w) { if (rc == DOF_OK && e != cudaSuccess) rc = dof_cuda_check(e, w); };
    ck(cudaMalloc(&big, sizeof(Bvh4Node) * n_bin), "collapse");
    ck(cudaMalloc(&fr[0], sizeof(int2) * n_bin), "collapse");
    ck(cudaMalloc(&fr[1], sizeof(int2) * n_bin), "collapse");
    ck(cudaMalloc(&cnt, sizeof(int) * 2), "collapse");
    if (rc == DOF_OK) {
        int2 first = make_int2(0, root);
        int init[2] = {1, 0};   // [0] 4-wide nodes allocated (the root), [1] next frontier size
        ck(cudaMemcpy(fr[0], &first, sizeof(int2), cudaMemcpyHostToDevice), "collapse");
        ck(cudaMemcpy(cnt, init, sizeof(init), cudaMemcpyHostToDevice), "collapse");
        int n_in = 1, cur = 0, level = 0;
        while (n_in > 0 && rc == DOF_OK) {
            if (++level > 200) { rc = dof_set_error(DOF_ERR_DEVICE_CHECK, "BVH collapse did not terminate"); break; }
            ck(cudaMemsetAsync(cnt + 1, 0, sizeof(int), st), "collapse");
            k_collapse<<<blocks_for(n_in, B), B, 0, st>>>(s->nodes, n_bin, fr[cur], n_in, big, n_bin, cnt, fr[cur ^ 1],
                                                         cnt + 1, ibuf + 6);
            int h[2];
            ck(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st), "collapse");
            ck(cudaStreamSynchronize(st), "collapse");
            n_in = h[1];
            s->n_nodes4 = h[0];
            cur ^= 1;
        }
        s->depth4 = level;
    }
    if (rc == DOF_OK) {
        s->nodes4_bytes = sizeof(Bvh4Node) * (size_t)s->n_nodes4;
        rc = dof_alloc(s->ctx, s->nodes4_bytes, (void **)&s->nodes4, &s->bytes);
        if (rc == DOF_OK)
            ck(cudaMemcpy(s->nodes4, big, s->nodes4_bytes, cudaMemcpyDeviceToDevice), "collapse copy");
        s->root4 = 0;
    }
    cudaFree(big); cudaFree(fr[0]); cudaFree(fr[1]); cudaFree(cnt);
    return rc;
}

int launch_bvh_build(DofScene *s, const float *d_xyz, uint32_t n_verts, const uint32_t *d_idx,
                     const uint32_t *d_mat, int builder, int ploc_radius, int rotations, cudaStream_t st) {
    const int n = (int)s->n_tris;
    const int B = 256;
    int rc = DOF_OK;
    float4 *cen = nullptr;
    int *ibuf = nullptr;                    // bounds[6], bad, depth
    unsigned long long *keys = nullptr, *keys2 = nullptr;
    uint32_t *vals = nullptr, *vals2 = nullptr;
    int4 *child = nullptr;
    int *pnode = nullptr, *pleaf = nullptr, *arr = nullptr;
    float4 *blo = nullptr, *bhi = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    int hbuf[16];
    int n_small = n, n_big = 0;
    auto ck = [&](cudaError_t e, const char *w) { if (rc == DOF_OK && e != cudaSuccess) rc = dof_cuda_check(e, w); };
    ck(cudaMalloc(&cen, sizeof(float4) * n), "bvh centroids");
    ck(cudaMalloc(&ibuf, sizeof(int) * 16), "bvh scalars");
    ck(cudaMalloc(&keys, sizeof(unsigned long long) * n), "bvh keys");
    ck(cudaMalloc(&vals, sizeof(uint32_t) * n), "bvh vals");
    ck(cudaMalloc(&keys2, sizeof(unsigned long long) * n), "bvh keys2");
    ck(cudaMalloc(&vals2, sizeof(uint32_t) * n), "bvh vals2");
    ck(cudaMalloc(&child, sizeof(int4) * (n > 1 ? n - 1 : 1)), "bvh children");
    ck(cudaMalloc(&pnode, sizeof(int) * (n > 1 ? n - 1 : 1)), "bvh parents");
    ck(cudaMalloc(&pleaf, sizeof(int) * n), "bvh leaf parents");
    ck(cudaMalloc(&arr, sizeof(int) * (n > 1 ? n - 1 : 1)), "bvh flags");
    ck(cudaMalloc(&blo, sizeof(float4) * (2 * n)), "bvh boxes");
    ck(cudaMalloc(&bhi, sizeof(float4) * (2 * n)), "bvh boxes");
    if (rc != DOF_OK) goto done;
    {
        // ibuf: [0..5] centroid bounds, [6] bad, [7] depth, [8] large count, [9..14] small bounds
        const int lo_i = 0x7FFFFFFF, hi_i = (int)0x80000000;
        int init[16] = {lo_i, lo_i, lo_i, hi_i, hi_i, hi_i, 0, 0, 0, lo_i, lo_i, lo_i, hi_i, hi_i, hi_i, 0};
        ck(cudaMemcpyAsync(ibuf, init, sizeof(init), cudaMemcpyHostToDevice, st), "bvh init");
        k_centroids<<<blocks_for(n, B), B, 0, st>>>(d_xyz, n_verts, d_idx, (uint32_t)n, cen, ibuf, ibuf + 6);
        k_classify<<<blocks_for(n, B), B, 0, st>>>(cen, (uint32_t)n, ibuf, ibuf + 8, ibuf + 9);
        ck(cudaMemcpyAsync(hbuf, ibuf, sizeof(hbuf), cudaMemcpyDeviceToHost, st), "bvh readback");
        ck(cudaStreamSynchronize(st), "bvh classify");
        if (rc != DOF_OK) goto done;
        // large triangles stay out of the tree (tested directly by every ray) when there
        // are few of them and at least one other triangle
        int separate = hbuf[8] > 0 && hbuf[8] <= kMaxLargeTris && hbuf[8] < n;
        n_big = separate ? hbuf[8] : 0;
        n_small = n - n_big;
        k_morton<<<blocks_for(n, B), B, 0, st>>>(cen, (uint32_t)n, separate ? ibuf + 9 : ibuf, ibuf, separate, keys,
                                                 vals);
        {
            // scratch of the sort: the digit histograms and the scan's tile sums
            const size_t nbk = (size_t)(n + kSortTile - 1) / kSortTile;
            const size_t nh = (size_t)kSortBins * nbk, ns = (nh + kScanTile - 1) / kScanTile + 1;
            tmp_bytes = sizeof(int) * (nh + ns);
            ck(cudaMalloc(&tmp, tmp_bytes), "sort temp");
            if (rc != DOF_OK) goto done;
            int *hist = static_cast<int *>(tmp);
            device_radix_sort_pairs(keys, vals, keys2, vals2, n, hist, hist + nh, st);
            ck(cudaGetLastError(), "sort");
        }
        // sorted (key, triangle) pairs are in (keys, vals)
        k_sorted_tris<<<blocks_for(n, B), B, 0, st>>>(d_xyz, d_idx, d_mat, (uint32_t)n, n_verts, vals, s->tris);
        const int m = n_small;
        int root = m >= 2 ? 0 : ~0;
        if (m >= 2) {
            ck(cudaMemsetAsync(pleaf, 0xFF, sizeof(int) * m, st), "memset");
            ck(cudaMemsetAsync(arr, 0, sizeof(int) * (m - 1), st), "memset");
            ck(cudaMemsetAsync(s->nodes, 0xFF, sizeof(BvhNode) * (m - 1), st), "memset");
            if (builder == DOF_BVH_PLOC) {
                if (rc == DOF_OK) rc = ploc_build(s, m, ploc_radius, pnode, pleaf, ibuf, &root, st);
                if (rc != DOF_OK) goto done;
            } else {
                k_karras<<<blocks_for(m - 1, B), B, 0, st>>>(keys, m, child, pnode, pleaf, ibuf + 6);
                k_refit<<<blocks_for(m, B), B, 0, st>>>(s->tris, m, child, pnode, pleaf, blo, bhi, arr, s->nodes,
                                                        ibuf + 6);
            }
            for (int pass = 0; pass < rotations; pass++) {
                ck(cudaMemsetAsync(arr, 0, sizeof(int) * (m - 1), st), "memset");
                k_rotate<<<blocks_for(m, B), B, 0, st>>>(m, s->nodes, pnode, pleaf, arr, ibuf + 6);
            }
            // the structure the packet tracer relies on (k_tree_refs), then the depth of
            // that structure; the sort's second buffers count the leaves' references
            ck(cudaMemsetAsync(arr, 0, sizeof(int) * (m - 1), st), "memset");
            ck(cudaMemsetAsync(vals2, 0, sizeof(int) * m, st), "memset");
            ck(cudaMemsetAsync(pnode, 0xFF, sizeof(int) * (m - 1), st), "memset");
            ck(cudaMemsetAsync(pleaf, 0xFF, sizeof(int) * m, st), "memset");
            int *ref_leaf = reinterpret_cast<int *>(vals2);
            k_tree_refs<<<blocks_for(m - 1, B), B, 0, st>>>(s->nodes, m - 1, m, arr, ref_leaf, pnode, pleaf, ibuf + 6);
            k_tree_counts<<<blocks_for(m, B), B, 0, st>>>(m - 1, m, root, arr, ref_leaf, ibuf + 6);
            k_depth<<<blocks_for(m, B), B, 0, st>>>(m, pnode, pleaf, ibuf + 7);
        }
        s->root = root;
        ck(cudaGetLastError(), "bvh kernels");
        ck(cudaMemcpyAsync(hbuf, ibuf, sizeof(hbuf), cudaMemcpyDeviceToHost, st), "bvh readback");
        ck(cudaStreamSynchronize(st), "bvh build");
        if (rc != DOF_OK) goto done;
        if (hbuf[6] == 1) { rc = dof_set_error(DOF_ERR_INVALID_ARG, "dof_scene_upload: vertex index out of range"); goto done; }
        if (hbuf[6]) { rc = dof_set_error(DOF_ERR_DEVICE_CHECK, "dof_scene_upload: BVH hierarchy check failed (%d)", hbuf[6]); goto done; }
        s->depth = m >= 2 ? (uint32_t)hbuf[7] : 1;
        s->n_tree = (uint32_t)m;
        s->n_large = (uint32_t)n_big;
        s->n_nodes = m >= 2 ? (uint32_t)(m - 1) : 0;
        if (s->depth > kTraversalStack) {
            rc = dof_set_error(DOF_ERR_DEVICE_CHECK, "BVH depth %u exceeds the traversal stack", s->depth);
            goto done;
        }
        if (m >= 2) {
            rc = collapse4(s, root, m - 1, ibuf, st);
            if (rc != DOF_OK) goto done;
            ck(cudaMemcpyAsync(hbuf, ibuf, sizeof(hbuf), cudaMemcpyDeviceToHost, st), "bvh readback");
            ck(cudaStreamSynchronize(st), "bvh collapse");
            if (rc != DOF_OK) goto done;
            if (hbuf[6]) { rc = dof_set_error(DOF_ERR_DEVICE_CHECK, "dof_scene_upload: BVH collapse check failed (%d)", hbuf[6]); goto done; }
        }
        // bounds of the tree's triangles: union of the root's child boxes
        if (m >= 2 && root >= 0) {
            BvhNode nd;
            ck(cudaMemcpy(&nd, s->nodes + root, sizeof(BvhNode), cudaMemcpyDeviceToHost), "bounds");
            s->lo[0] = fminf(nd.a.x, nd.b.z); s->lo[1] = fminf(nd.a.y, nd.b.w); s->lo[2] = fminf(nd.a.z, nd.c.x);
            s->hi[0] = fmaxf(nd.a.w, nd.c.y); s->hi[1] = fmaxf(nd.b.x, nd.c.z); s->hi[2] = fmaxf(nd.b.y, nd.c.w);
        }
    }
done:
    cudaFree(cen); cudaFree(ibuf); cudaFree(keys); cudaFree(vals); cudaFree(keys2); cudaFree(vals2);
    cudaFree(child); cudaFree(pnode); cudaFree(pleaf); cudaFree(arr); cudaFree(blo); cudaFree(bhi); cudaFree(tmp);
    return rc;
}

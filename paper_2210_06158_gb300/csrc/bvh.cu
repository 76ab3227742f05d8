// Device-built BVH of libdof (the acceleration structure whose build the paper
// counts in its ray-trace time, Section 4.2).
//
// LBVH after Karras, "Maximizing Parallelism in the Construction of BVHs, Octrees,
// and k-d Trees" (HPG 2012): 30-bit Morton codes of triangle centroids, a radix sort,
// one thread per internal node to find its key range and split (ties between equal
// codes broken by the sorted index, so the tree depth is at most 62), then a
// bottom-up box refit in which the second thread to reach a node merges its two
// children (atomic arrival counter, no waiting).  Nodes hold both child boxes so that
// traversal fetches one node per step.
#include <cub/cub.cuh>

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
        cen[t] = make_float4(c.x, c.y, c.z, 0.f);
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

__device__ __forceinline__ uint32_t expand10(uint32_t v) {
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__global__ void k_morton(const float4 *cen, uint32_t n, const int *bounds, uint32_t *keys, uint32_t *vals) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
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
        q[k] = (uint32_t)fminf(fmaxf(u * 1024.f, 0.f), 1023.f);
    }
    keys[t] = (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
    vals[t] = t;
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
__device__ __forceinline__ int delta(const uint32_t *keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    uint32_t a = keys[i], b = keys[j];
    if (a != b) return __clz(a ^ b);
    return 32 + __clz(i ^ j);
}

// one thread per internal node: its range, split and children; parent links.
// child refs: >= 0 internal, < 0 leaf ~k
__global__ void k_karras(const uint32_t *keys, int n, int4 *child, int *parent_node, int *parent_leaf, int *bad) {
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
        if (p >= n - 1 || level > 128) { atomicExch(bad, 3); return; }
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

// tree depth (levels from the root to the deepest leaf, root = 1)
__global__ void k_depth(int n, const int *parent_node, const int *parent_leaf, int *depth) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int d = 1, p = parent_leaf[k];
    while (p >= 0 && d < 1000) { d++; p = parent_node[p]; }
    atomicMax(depth, d);
}

}  // namespace

static inline unsigned blocks_for(size_t n, int b) { return (unsigned)((n + b - 1) / b); }

int launch_bvh_build(DofScene *s, const float *d_xyz, uint32_t n_verts, const uint32_t *d_idx,
                     const uint32_t *d_mat, cudaStream_t st) {
    const int n = (int)s->n_tris;
    const int B = 256;
    int rc = DOF_OK;
    float4 *cen = nullptr;
    int *ibuf = nullptr;                    // bounds[6], bad, depth
    uint32_t *keys = nullptr, *vals = nullptr, *keys2 = nullptr, *vals2 = nullptr;
    int4 *child = nullptr;
    int *pnode = nullptr, *pleaf = nullptr, *arr = nullptr;
    float4 *blo = nullptr, *bhi = nullptr;
    void *tmp = nullptr;
    size_t tmp_bytes = 0;
    int hbuf[8];
    auto ck = [&](cudaError_t e, const char *w) { if (rc == DOF_OK && e != cudaSuccess) rc = dof_cuda_check(e, w); };
    ck(cudaMalloc(&cen, sizeof(float4) * n), "bvh centroids");
    ck(cudaMalloc(&ibuf, sizeof(int) * 8), "bvh scalars");
    ck(cudaMalloc(&keys, sizeof(uint32_t) * n), "bvh keys");
    ck(cudaMalloc(&vals, sizeof(uint32_t) * n), "bvh vals");
    ck(cudaMalloc(&keys2, sizeof(uint32_t) * n), "bvh keys2");
    ck(cudaMalloc(&vals2, sizeof(uint32_t) * n), "bvh vals2");
    ck(cudaMalloc(&child, sizeof(int4) * (n > 1 ? n - 1 : 1)), "bvh children");
    ck(cudaMalloc(&pnode, sizeof(int) * (n > 1 ? n - 1 : 1)), "bvh parents");
    ck(cudaMalloc(&pleaf, sizeof(int) * n), "bvh leaf parents");
    ck(cudaMalloc(&arr, sizeof(int) * (n > 1 ? n - 1 : 1)), "bvh flags");
    ck(cudaMalloc(&blo, sizeof(float4) * (2 * n)), "bvh boxes");
    ck(cudaMalloc(&bhi, sizeof(float4) * (2 * n)), "bvh boxes");
    if (rc != DOF_OK) goto done;
    {
        int init[8] = {0x7FFFFFFF, 0x7FFFFFFF, 0x7FFFFFFF, (int)0x80000000, (int)0x80000000, (int)0x80000000, 0, 0};
        ck(cudaMemcpyAsync(ibuf, init, sizeof(init), cudaMemcpyHostToDevice, st), "bvh init");
        k_centroids<<<blocks_for(n, B), B, 0, st>>>(d_xyz, n_verts, d_idx, (uint32_t)n, cen, ibuf, ibuf + 6);
        k_morton<<<blocks_for(n, B), B, 0, st>>>(cen, (uint32_t)n, ibuf, keys, vals);
        ck(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, keys, keys2, vals, vals2, n, 0, 30, st), "sort size");
        ck(cudaMalloc(&tmp, tmp_bytes ? tmp_bytes : 16), "sort temp");
        if (rc != DOF_OK) goto done;
        ck(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys, keys2, vals, vals2, n, 0, 30, st), "sort");
        k_sorted_tris<<<blocks_for(n, B), B, 0, st>>>(d_xyz, d_idx, d_mat, (uint32_t)n, n_verts, vals2, s->tris);
        if (n >= 2) {
            ck(cudaMemsetAsync(pleaf, 0xFF, sizeof(int) * n, st), "memset");
            ck(cudaMemsetAsync(arr, 0, sizeof(int) * (n - 1), st), "memset");
            ck(cudaMemsetAsync(s->nodes, 0xFF, sizeof(BvhNode) * (n - 1), st), "memset");
            k_karras<<<blocks_for(n - 1, B), B, 0, st>>>(keys2, n, child, pnode, pleaf, ibuf + 5 + 1);
            k_refit<<<blocks_for(n, B), B, 0, st>>>(s->tris, n, child, pnode, pleaf, blo, bhi, arr, s->nodes,
                                                    ibuf + 6);
            k_depth<<<blocks_for(n, B), B, 0, st>>>(n, pnode, pleaf, ibuf + 7);
        }
        ck(cudaGetLastError(), "bvh kernels");
        ck(cudaMemcpyAsync(hbuf, ibuf, sizeof(hbuf), cudaMemcpyDeviceToHost, st), "bvh readback");
        ck(cudaStreamSynchronize(st), "bvh build");
        if (rc != DOF_OK) goto done;
        if (hbuf[6] == 1) { rc = dof_set_error(DOF_ERR_INVALID_ARG, "dof_scene_upload: vertex index out of range"); goto done; }
        if (hbuf[6]) { rc = dof_set_error(DOF_ERR_DEVICE_CHECK, "dof_scene_upload: BVH hierarchy check failed (%d)", hbuf[6]); goto done; }
        s->depth = n >= 2 ? (uint32_t)hbuf[7] : 1;
        if (s->depth > 64) { rc = dof_set_error(DOF_ERR_DEVICE_CHECK, "BVH depth %u exceeds the traversal stack", s->depth); goto done; }
        // scene bounds from the triangle boxes (root box)
        if (n >= 2) {
            float4 lo, hi;
            ck(cudaMemcpy(&lo, blo, sizeof(float4), cudaMemcpyDeviceToHost), "bounds");
            ck(cudaMemcpy(&hi, bhi, sizeof(float4), cudaMemcpyDeviceToHost), "bounds");
            s->lo[0] = lo.x; s->lo[1] = lo.y; s->lo[2] = lo.z;
            s->hi[0] = hi.x; s->hi[1] = hi.y; s->hi[2] = hi.z;
        }
    }
done:
    cudaFree(cen); cudaFree(ibuf); cudaFree(keys); cudaFree(vals); cudaFree(keys2); cudaFree(vals2);
    cudaFree(child); cudaFree(pnode); cudaFree(pleaf); cudaFree(arr); cudaFree(blo); cudaFree(bhi); cudaFree(tmp);
    return rc;
}

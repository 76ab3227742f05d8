// Internal declarations of libdof (GB300 / sm_103a): device-side parameter blocks,
// small FP32 helpers shared by the kernels, and the host objects behind the C ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <atomic>
#include <mutex>
#include <string>

#include "../../include/dof.h"

// ---------------------------------------------------------------------------
// device parameter blocks (passed by value to kernels)
// ---------------------------------------------------------------------------

struct DevCam {
    float3 O, R, U, F;          // current pose
    float3 pO, pR, pU, pF;      // previous pose
    float invF;                 // 1 / focal length in full-resolution pixels
    float Fpx;                  // focal length in full-resolution pixels
    float cocK;                 // c(z) = cocK * (z - d) / z  (signed diameter, fpx)
    float d;                    // focus distance
    float lens_r;               // aperture radius a / 2
    float halfW, halfH;         // W / 2, H / 2
    int W, H, W2, H2;
    uint32_t frame;
    int moved;                  // the pose changed (jitter aside)
    float jx, jy, pjx, pjy;     // sampling jitter of this and of the previous frame (full-res px)
    int exact;                  // pose and jitter unchanged: reprojection is the identity
};

struct DevParams {
    float s, var_w_mask, m;
    int spp, ray_mode;
    float inv_depth_range, alpha, alpha_motion, var_w_recon, b_max, h_edge;
    float lod_scale, lod_max, rmax_hpx, zof_ramp, inv_cover_ramp, bright_lum, inv_bright_ramp;
    float mask_near_hpx, z_far;
    uint32_t albedo_seed;
    unsigned long long seed, session;
    float3 light;               // normalised light travel direction
    float k_a, k_d, emit;
    float3 sky;
    int tiles_w, tiles_h, dil_k;
    int f16;                    // colour image buffers stored as FP16
    float taa_alpha;            // final TAA blend (0 = off)
    int blades;                 // aperture: 0 circle, 3..8 regular n-gon
    int ring;                   // row of the 81-tap table: 0 circle, blades - 2 for an n-gon
    float inv_area, inv_sqrt_area;  // sampleAlpha: 1 / A and 1 / sqrt(A), A = the aperture's area at radius 1
};

// ---------------------------------------------------------------------------
// scene (device-built LBVH)
// ---------------------------------------------------------------------------

// BVH node: boxes of both children and their references.  A reference r >= 0 is an
// internal node, r < 0 the leaf holding sorted triangle ~r.
struct __align__(16) BvhNode {
    float4 a;   // child0 lo.xyz, child0 hi.x
    float4 b;   // child0 hi.yz, child1 lo.xy
    float4 c;   // child1 lo.z, child1 hi.xyz
    int4 r;     // child0 ref, child1 ref, unused, unused
};

// 4-wide node: the boxes of up to four children (structure of arrays) and their
// references (>= 0 node, < 0 leaf ~k, kEmptyChild for an unused slot)
struct __align__(16) Bvh4Node {
    float4 lox, hix, loy, hiy, loz, hiz;
    int4 ref;
    int4 pad;
};
constexpr int kEmptyChild = (int)0x80000000;

struct SceneDev {
    const BvhNode *nodes;        // n_tris - 1 internal nodes (root = 0) when n_tris >= 2
    const float4 *tris;          // 3 float4 per sorted triangle: v0 (w = prim id bits), v1, v2 (w = material bits)
    int n_tris;                  // triangles in the tree (sorted indices 0 .. n_tris-1)
    int n_large;                 // large triangles after them, tested directly by every ray
    int root;                    // root reference (internal node, or ~0 for a one-leaf tree)
    const Bvh4Node *nodes4;      // the tree collapsed to 4-wide nodes (traversed when non-null)
    int root4;                   // its root reference
    int n_nodes4;
    int stack_need;              // traversal stack entries the traversed tree can need
};

// at most this many large triangles are kept out of the tree (see bvh.cu)
constexpr int kMaxLargeTris = 64;

// ---------------------------------------------------------------------------
// host objects
// ---------------------------------------------------------------------------

struct DofCtx {
    int device;
    std::atomic<int> refs;         // 1 for the caller's handle + 1 per live scene / history
    std::atomic<size_t> in_use;
    size_t budget;
    int sm_count;
    int bvh_builder;               // DOF_BVH_PLOC or DOF_BVH_LBVH
    int bvh_rotations;             // passes of tree rotations after the build
    int trace_blocks_per_sm, trace_refill_idle, trace_steps, ray_order_grid, trace_packets, trace_stats;
    int gather_w, gather_h, main_form;   // main filter launch shape and form
    int recon_w, recon_h;                // reconstruction launch shape
    int stack_depth;                     // requested traversal stack entries (raised to the tree's need)
    int ploc_radius;
    int bvh_width;                 // 4: traverse the collapsed 4-wide tree, 2: the binary tree
    uint32_t *d_status;            // device status word of context-level launches
    // A frame's ray path (mask .. reconstruction) runs on ray_stream (highest priority)
    // while its post-process filters run on the caller's stream; ev_fork / ev_join order
    // them around the shared inputs (tiles) and the composite.
    cudaStream_t ray_stream;
    cudaEvent_t ev_fork, ev_join;
    std::mutex launch_mu;          // one frame's enqueue at a time on ray_stream
    cudaMemPool_t pool;            // stream-ordered scratch of the rasterising G-buffer producer
};

struct DofScene {
    DofCtx *ctx;
    uint32_t n_tris, n_nodes, depth;
    uint32_t n_tree, n_large;      // triangles in the tree / tested directly
    int root;
    size_t tris_bytes, nodes_bytes;  // allocation sizes (for the context's budget)
    Bvh4Node *nodes4;
    size_t nodes4_bytes;
    int root4, n_nodes4, depth4;
    BvhNode *nodes;
    float4 *tris;
    int32_t *prim_k;               // triangle id -> sorted index (n_tris)
    size_t bytes;
    float lo[3], hi[3];
};

struct DofHistory {
    DofCtx *ctx;
    uint32_t W, H, W2, H2, N, TW, TH, max_rays, flags;
    size_t bytes;
    uint64_t frames;
    int valid;                     // a previous frame exists
    int cur;                       // which history buffer holds the latest frame
    // per-frame work buffers
    float4 *pp_in, *pre, *main_, *pp_med, *n_h;
    float *z_h, *xn, *xf;
    float2 *tiles, *tiles_dil;
    int32_t *nrays;
    uint32_t *queue;               // masked pixel indices
    uint32_t *first_ray;           // per pixel: slot of its first ray (its rays own n slots)
    uint32_t *ray_pix;             // tracer work order: q << 6 | sample, grouped by lens cell
                                   // (N * max_rays; q < 2^26 by the 16384 size limit)
    int2 *hits;                    // per ray: (sorted triangle index or -1, t bits)
    float4 *ray_a;                 // per ray as the tracer made it: (origin, dir.x) ...
    float2 *ray_b;                 // ... and (dir.y, dir.z); the shader reads them back
    uint32_t *counters;            // [0] queue length, [1] rays, [2] work cursor, [3] device status,
                                   // [4..5] node visits (u64), [6..7] triangle tests (u64)
    int32_t *ray_prim;
    float4 *rt;                    // 4 planes of N
    float4 *crt, *rt_med, *recon;
    float *ct, *var;
    float4 *mip[4];                // per level, 32 bytes per texel: (rgb, h) * valid and
                                   // (c_t, 1) * valid, laid out by st_mip
    int mip_w[4], mip_h[4];
    // final TAA (DOF_HIST_TAA): composited image of the frame, resolved images (ping-pong)
    float4 *comp, *taa[2];
    int taa_cur, taa_valid;
    // persistent state (ping-pong)
    float4 *hist[2];               // 3 planes of N each
    float *var_blur[2];
    uint32_t host_counters[4];
    // per-kernel timing ring (DOF_HIST_TIMING)
    cudaEvent_t *ev;               // kTimingSlots x (DOF_K_COUNT + 1)
    int ev_slot, ev_used;
    // frames from and to host memory (dof_frame_host): two device slots (G-buffer in,
    // image out) used in turn, a copy stream per direction, and per slot the events
    // "inputs copied", "frame done with the slot", "image copied out"
    float4 *hio_color[2], *hio_normal[2], *hio_out[2];
    float *hio_depth[2];
    cudaEvent_t hio_in[2], hio_used[2], hio_done[2];
    cudaStream_t hio_h2d, hio_d2h;
    int hio_ready, hio_normals;
    uint64_t hio_frames;
};

constexpr int kTimingSlots = 64;
// traversal stack entries; the LBVH over 63-bit keys with index tie-breaks is at most
// 63 + 32 levels deep, and uploads whose tree is deeper than this are rejected
constexpr int kTraversalStack = 96;

// record the event that closes kernel `k` of the current frame (no-op without timing)
inline void tmark(DofHistory *h, int k, cudaStream_t st) {
    if (h && h->ev && h->ev_used < kTimingSlots) cudaEventRecord(h->ev[h->ev_slot * (DOF_K_COUNT + 1) + k + 1], st);
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

int dof_set_error(int code, const char *fmt, ...);
int dof_cuda_check(cudaError_t e, const char *what);
int dof_alloc(DofCtx *ctx, size_t bytes, void **ptr, size_t *acc);
void ctx_retain(DofCtx *ctx);
void ctx_release(DofCtx *ctx);   // frees the context with its last reference
void dof_free(DofCtx *ctx, void *ptr, size_t bytes);

// launch wrappers (one per kernel group, defined in the .cu files)
int launch_bvh_build(DofScene *s, const float *d_xyz, uint32_t n_verts, const uint32_t *d_idx,
                     const uint32_t *d_mat, int builder, int ploc_radius, int rotations, cudaStream_t st);
void launch_primary(const DevCam &cam, const DevParams &p, SceneDev sc, float4 *color, float *depth,
                    float4 *normal, int32_t *prim, uint32_t *status, cudaStream_t st);
// host-side tally of this library's kernel launches (dof_launch_count); each launch
// wrapper adds the launches it enqueued
void count_launches(long long n);

// rasterising G-buffer producer (raster.cu)
void launch_prim_index(const float4 *tris, int n, int32_t *prim_k, cudaStream_t st);
size_t raster_scratch_bytes(int W, int H, int n_tot);
// stable sort of (keys, vals) by the keys' low `bits` bits (a multiple of 16), result in
// (keys, vals); (keys2, vals2) and scratch (sort_pairs_scratch_ints(n) ints) are scratch
size_t sort_pairs_scratch_ints(int n);
void sort_pairs_by_low_bits(unsigned long long *keys, uint32_t *vals, unsigned long long *keys2, uint32_t *vals2,
                            int n, int bits, int *scratch, cudaStream_t st);
cudaError_t launch_raster(const DevCam &cam, const DevParams &p, const SceneDev &sc, const int32_t *prim_k,
                          void *scratch, int sm_count, float4 *color, float *depth, float4 *normal, int32_t *prim,
                          cudaStream_t st);
// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

#ifdef __CUDACC__
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize(float3 v) { return rsqrtf(dot(v, v)) * v; }
__device__ __forceinline__ float sat(float x) { return fminf(fmaxf(x, 0.f), 1.f); }
__device__ __forceinline__ float lerpf(float a, float b, float t) { return a + t * (b - a); }
__device__ __forceinline__ float lum709(float r, float g, float b) { return 0.2126f * r + 0.7152f * g + 0.0722f * b; }

// colour image buffers: float4, or 4 x FP16 (8 bytes) when `h` (FP32 arithmetic either way)
// hint: bring the line holding p into L1 (holds no register; p must be a valid address)
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

__device__ __forceinline__ float4 ld_img(const float4 *base, size_t i, bool h) {
    if (h) {
        uint2 u = __ldg(reinterpret_cast<const uint2 *>(base) + i);
        __half2 a = *reinterpret_cast<__half2 *>(&u.x), b = *reinterpret_cast<__half2 *>(&u.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    return __ldg(base + i);
}
// the value st_img stores (FP16 storage rounds each channel to half)
__device__ __forceinline__ float4 round_img(float4 v, bool h) {
    if (!h) return v;
    float2 a = __half22float2(__floats2half2_rn(v.x, v.y)), b = __half22float2(__floats2half2_rn(v.z, v.w));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_img(float4 *base, size_t i, float4 v, bool h) {
    if (h) {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&a);
        u.y = *reinterpret_cast<uint32_t *>(&b);
        reinterpret_cast<uint2 *>(base)[i] = u;
    } else {
        base[i] = v;
    }
}

// One texel i of a level of the reconstruction's pyramid (n texels, 32 bytes each from a
// 256-byte aligned base): the colour a = (rgb, h) * valid and b = (c_t, 1) * valid.
// FP32 storage keeps two planes, a at base[i] and b at float2 index i after the n
// colours.  FP16 storage keeps one 16-byte record per texel, a as half4 then b, so a tap
// reads a texel with one load.  (A 32-byte FP32 record read by one 256-bit load made
// the reconstruction slower: a quarter of every record was padding through L1.)
__device__ __forceinline__ void st_mip(float4 *base, size_t n, size_t i, float4 a, float2 b, bool h) {
    if (h) {
        __half2 x = __floats2half2_rn(a.x, a.y), y = __floats2half2_rn(a.z, a.w);
        base[i] = make_float4(__uint_as_float(*reinterpret_cast<uint32_t *>(&x)),
                              __uint_as_float(*reinterpret_cast<uint32_t *>(&y)), b.x, b.y);
    } else {
        base[i] = a;
        reinterpret_cast<float2 *>(base + n)[i] = b;
    }
}

__device__ __forceinline__ float4 f4add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 f4scale(float s, float4 a) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }
__device__ __forceinline__ float4 f4fma(float s, float4 a, float4 acc) {
    return make_float4(fmaf(s, a.x, acc.x), fmaf(s, a.y, acc.y), fmaf(s, a.z, acc.z), fmaf(s, a.w, acc.w));
}

// signed CoC diameter (full-resolution px) of depth z
__device__ __forceinline__ float coc_of(const DevCam &c, float z) { return c.cocK * (z - c.d) / z; }

// direction through sensor point (x, y) (full-resolution px) and the lens centre
// direction through the sensor point (x, y) + jitter and the lens centre
__device__ __forceinline__ float3 pixel_dir(const DevCam &c, float x, float y) {
    float sx = (x + c.jx - c.halfW) * c.invF, sy = (y + c.jy - c.halfH) * c.invF;
    return normalize(make_float3(c.F.x + sx * c.R.x - sy * c.U.x, c.F.y + sx * c.R.y - sy * c.U.y,
                                 c.F.z + sx * c.R.z - sy * c.U.z));
}
#endif

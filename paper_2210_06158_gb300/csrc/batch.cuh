// Batched launches of libdof: every pass of a frame runs as ONE launch over the
// frames of all sessions of a batch.  A session descriptor holds the session's
// camera, parameters, scene and buffers; the launch argument (a __grid_constant__
// kernel parameter, no copy to device memory) holds up to kMaxBatch descriptors and,
// per launch shape, the prefix of the sessions' block counts, so a block finds its
// session by binary search and its position in that session's grid.
#pragma once

#include "dof_internal.cuh"

enum LaunchShape {
    SH_HPX = 0,     // 32x8 half-resolution pixels per block
    SH_FPX,         // 32x8 full-resolution pixels per block
    SH_SHADE,       // 128 queue entries per block
    SH_GATHER,      // the main filter's 81-tap gather: gather_w x gather_h hpx
    SH_RECON,       // the reconstruction's 81-tap gather: recon_w x recon_h hpx
    SH_COUNT
};

constexpr int kMaxBatch = DOF_MAX_BATCH;

struct SessDesc {
    DevCam cam;
    DevParams p;
    SceneDev sc;
    int gx[SH_COUNT];              // blocks per row of each shape
    int N, max_rays, valid, record_rays;
    // frame inputs and output (caller-owned)
    const float4 *color;
    const float *depth;
    const float4 *normal;
    int gf16;                      // colour and normal planes in half4 (DOF_FMT_F16)
    float4 *out;
    float4 *comp_out;              // composite target: out, or the history's image for the TAA
    const float4 *taa_in;          // previous resolved image (TAA)
    float4 *taa_out;
    int taa, taa_valid;
    // work buffers of the session (history-owned)
    float4 *pp_in, *pre, *main_, *pp_med, *n_h, *zn, *crt, *rt_med, *recon, *rt;
    float *z_h, *xn, *xf, *ct, *var;
    float2 *tiles, *tiles_dil;
    int32_t *nrays, *ray_prim;
    uint32_t *queue, *first_ray, *ray_pix, *counters;
    int2 *hits;
    float4 *ray_a;
    float2 *ray_b;
    float4 *mip[4];
    int mip_w[4], mip_h[4], mip_L;
    // history ping-pong
    const float4 *hist_in;
    float4 *hist_out;
    const float *var_in;           // blurred variance of the previous frame
    float *var_out;
};

struct BatchArgs {
    int ns;
    int refill_idle, steps_per_round;   // tracer scheduling
    int lens_grid;                 // tracer work order: lens-cell grid of the mask kernel (1 = pixel order)
    int packets;                   // 1: the binary tree traversed by warp packets (k_trace_packets)
    int stats;                     // 1: the packet tracer counts node visits and triangle tests
    int stack_depth;               // requested traversal stack entries (the launch takes an instance >= the need)
    int gather_w, gather_h;        // block of the main filter (SH_GATHER), <= 512 threads
    int recon_w, recon_h;          // block of the reconstruction (SH_RECON), <= 512 threads
    int main_form;                 // main filter: 0 halo tile up to 64 KB, 1 through L1, 2 halo tile up
                                   // to the SM's opt-in shared memory, 3 columns of four pixels
    int start[SH_COUNT][kMaxBatch + 1];
    uint32_t *cursor;              // device word: ray cursor of the persistent tracer
    SessDesc s[kMaxBatch];
};

// The image storage of a launch's sessions: 0 every session FP32, 1 every session FP16,
// 2 mixed (kernels specialised on it take each session's own from its parameters).
inline int image_storage_mode(const BatchArgs &A) {
    int n16 = 0;
    for (int i = 0; i < A.ns; i++) n16 += A.s[i].p.f16 != 0;
    return n16 == 0 ? 0 : (n16 == A.ns ? 1 : 2);
}
// whether any session of the launch takes the final TAA pass
inline bool any_taa(const BatchArgs &A) {
    for (int i = 0; i < A.ns; i++)
        if (A.s[i].taa) return true;
    return false;
}

#ifdef __CUDACC__
// session of a flat block index for `shape`; *local = the block's index in that session
__device__ __forceinline__ int find_session(const BatchArgs &A, int shape, int block, int &local) {
    int lo = 0, hi = A.ns;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (A.start[shape][mid] <= block) lo = mid;
        else hi = mid;
    }
    local = block - A.start[shape][lo];
    return lo;
}

// 2D position of the calling thread for a 2D shape with blocks of blockDim
__device__ __forceinline__ const SessDesc &block_session(const BatchArgs &A, int shape, int &i, int &j) {
    int lb;
    int s = find_session(A, shape, blockIdx.x, lb);
    const SessDesc &S = A.s[s];
    int gx = S.gx[shape];
    i = (lb % gx) * blockDim.x + threadIdx.x;
    j = (lb / gx) * blockDim.y + threadIdx.y;
    return S;
}
#endif

#ifdef __CUDACC__
// A2, tile dilation, for the four 8x8 tiles of a 32x8-pixel block (block origin bx, by in
// half-resolution pixels): warp w < 4 takes tile (bx / 8 + w, by / 8) and the max of
// (near radius, |rho|) over its (2K+1)^2 neighbourhood of raw tiles, lanes striding the
// neighbourhood and a shuffle reduction across the warp.  Result in out[w] (shared
// memory; the caller synchronises before reading it).  Tiles past the image's tile grid
// are left untouched.
__device__ __forceinline__ void dilate_block_tiles(const SessDesc &S, int bx, int by, float2 *out) {
    const DevParams &p = S.p;
    const unsigned lane = threadIdx.x & 31u, w = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int tx = bx / 8 + (int)w, ty = by / 8;
    if (w >= 4 || tx >= p.tiles_w || ty >= p.tiles_h) return;
    const int K = p.dil_k, side = 2 * K + 1;
    float nm = 0.f, am = 0.f;
    for (int e = (int)lane; e < side * side; e += 32) {
        const int y = ty - K + e / side, x = tx - K + e % side;
        if (x >= 0 && y >= 0 && x < p.tiles_w && y < p.tiles_h) {
            const float2 v = __ldg(&S.tiles[y * p.tiles_w + x]);
            nm = fmaxf(nm, v.x);
            am = fmaxf(am, v.y);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nm = fmaxf(nm, __shfl_xor_sync(0xffffffffu, nm, o));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
    }
    if (lane == 0) out[w] = make_float2(nm, am);
}
#endif

// device: the batch descriptor, passed by value (a __grid_constant__ kernel parameter)
// or, for captured graphs, as a pointer to device memory that a copy refreshes per step
#ifdef __CUDACC__
__device__ __forceinline__ const BatchArgs &batch_args(const BatchArgs &a) { return a; }
__device__ __forceinline__ const BatchArgs &batch_args(const BatchArgs *a) { return *a; }
#endif

// host: launch wrappers per kernel group (post.cu, trace.cu, temporal.cu, recon.cu); `A`
// gives the launch shapes, `as` is what the kernels receive (A itself, or a device
// pointer to a copy of it)
template <class AS> void launch_tiles_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *timing);  // A1
template <class AS> void launch_pp_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *timing);     // A3 - A5
int main_filter_tile_bytes(const BatchArgs &A);   // the main filter's launch form (post.cu)
template <class AS>
void launch_mask_b(const BatchArgs &A, const AS &as, bool any_adaptive, cudaStream_t st, DofHistory *timing);
template <class AS> void launch_trace_b(const BatchArgs &A, const AS &as, int blocks, cudaStream_t st, DofHistory *timing);
void preload_trace_kernels();
void preload_post_kernels();
void preload_recon_kernels();
template <class AS> void launch_temporal_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *timing);
template <class AS> void launch_recon_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *timing);  // A10, A11
template <class AS> void launch_composite_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *timing);  // A12

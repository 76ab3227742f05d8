/*
 * dof.h -- C ABI of libdof, the GB300 (sm_103a) implementation of the per-frame
 * hybrid depth-of-field pass of Tan, Chua, Biette and Bhojan, "A Hybrid System for
 * Real-Time Rendering of Depth of Field Effect in Games" (arXiv 2210.06158).
 *
 * One frame (Section 3, Fig. 1): thin-lens circle of confusion from the G-buffer
 * depth, half-resolution gather bokeh (prefilter, 81-tap main filter, median), a ray
 * mask of the blurred-foreground region, thin-lens rays for the masked pixels through
 * a device-built BVH, temporal accumulation with reprojection, median and spatial
 * reconstruction of the ray-traced layer, and the CoC-driven composite.
 *
 * Conventions
 *  - Image pointers are DEVICE pointers owned by the caller (dof_frame_host: HOST
 *    pointers), row-major and densely packed (row pitch = width * element size; no
 *    other pitch is supported).
 *  - Scene geometry passed to dof_scene_upload is in HOST memory and is copied.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Calls enqueue work on it and return without synchronising, except where stated.
 *  - Errors found on the host are returned synchronously as a negative DOF_ERR_*
 *    code, with a message from dof_last_error() (thread-local).  Errors raised on the
 *    device (bounded waits that ran out, failed internal checks) are recorded in a
 *    device status word and reported by the next call on the same context, or by
 *    dof_frame_stats().
 *  - Lengths are in metres, image coordinates in pixels with (0,0) the top-left
 *    pixel's corner; depth is the distance along the camera's forward axis.
 */
#ifndef DOF_H
#define DOF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------------ */
#define DOF_OK                 0
#define DOF_ERR_INVALID_ARG   -1   /* null pointer, odd or zero size, d <= f, N <= 0, ... */
#define DOF_ERR_OOM           -2   /* device allocation failed */
#define DOF_ERR_BUDGET        -3   /* allocation would exceed the context's memory budget */
#define DOF_ERR_CUDA          -4   /* a CUDA runtime call failed (see dof_last_error) */
#define DOF_ERR_TIMEOUT       -5   /* a bounded device wait ran out */
#define DOF_ERR_DEVICE_CHECK  -6   /* an internal device-side check failed */
#define DOF_ERR_MISMATCH      -7   /* history bound to another size / scene */

/* ---- image formats ----------------------------------------------------------- */
#define DOF_FMT_F32 0              /* colour/normal float4 (rgb/xyz + unused), depth float */
#define DOF_FMT_F16 1              /* colour/normal half4 (8 bytes per pixel), depth float */

/* ---- parameters -------------------------------------------------------------- */

/* Thin-lens camera (Section 3.3 below Eq. 6: focal length f, aperture a = f/N, focus
 * distance d, sensor width w_s) and the pose of this and of the previous frame.  The
 * pose is an orthonormal basis: `fwd` the optical axis, `right`/`up` the image x / -y
 * axes.  The focal length in pixels is F = W v / w_s with v = f d / (d - f).
 * jitter: the frame's sub-pixel camera jitter against aliasing (Section 3.1.2), in
 * full-resolution pixels, |.| <= 1: every pixel samples the sensor at its position plus
 * the jitter (G-buffer producer and thin-lens rays alike), and reprojection into the
 * previous frame subtracts prev_jitter.  Zero: no jitter. */
typedef struct {
    float f_m, f_number, focus_m, sensor_w_m;
    float pos[3], right[3], up[3], fwd[3];
    float prev_pos[3], prev_right[3], prev_up[3], prev_fwd[3];
    uint32_t frame_index;          /* Philox counter word (lens samples differ per frame) */
    float jitter[2];               /* this frame's sampling offset (x, y), full-res px */
    float prev_jitter[2];          /* the previous frame's */
} DofCamera;

/* Method constants.  Defaults (dof_params_default) are the paper's values where it
 * gives one: s = 0.8 (Section 4.2, Eq. 2), 1e5 (Eq. 4), alpha = 0.95 (Section 3.2.3),
 * 2000 and 0.9 (Eq. 5), 0.3 (Eq. 7), 0.05 and 3 (Eq. 8), 10 cm (Section 4.2). */
typedef struct {
    float s;                /* Eq. 2 scale */
    float var_w_mask;       /* Eq. 4 variance weight */
    uint32_t m;             /* Eq. 4 ray budget per pixel (adaptive mode), <= DOF_MAX_RAYS */
    uint32_t spp;           /* rays per masked pixel (fixed mode), 1..DOF_MAX_RAYS */
    uint32_t ray_mode;      /* 0 fixed spp, 1 adaptive (Eq. 4) */
    float depth_range_m;    /* main-filter depth range */
    float alpha;            /* EMA blend factor */
    float alpha_motion;     /* EMA blend factor while the camera moves */
    float var_w_recon;      /* Eq. 5 weight */
    float b_max;            /* Eq. 5 clamp */
    float h_edge;           /* Eq. 7 smoothstep edge */
    float lod_scale;        /* Eq. 8 slope */
    float lod_max;          /* Eq. 8 clamp (<= 3) */
    float max_coc_px;       /* CoC radius clamp in full-resolution px (>= 1, <= 256) */
    float zof_ramp_px;      /* width of the continuous zone-of-focus test (Eq. 6) */
    float cover_ramp_px;    /* width of the continuous coverage test D (Eq. 1) */
    float bright_lum;       /* luminance above which a sample counts as bright bokeh */
    float bright_ramp;      /* ... ramp width */
    float mask_near_hpx;    /* ray mask threshold on the dilated near CoC radius (hpx) */
    float z_far_m;          /* depth that stands for "no geometry" (sky) */
    uint32_t tile;          /* max-CoC tile size in half-resolution px: must be 8 */
    uint32_t albedo_seed;   /* hash seed of the per-triangle albedo */
    uint64_t seed;          /* Philox key word 0 */
    uint64_t session;       /* Philox key word 1 */
    float light_dir[3];     /* direction the light travels */
    float k_a, k_d;         /* ambient and Lambert coefficients */
    float sky[3];           /* radiance of rays that hit nothing */
    float emit;             /* radiance scale of material 1 (emitters) */
    uint32_t image_storage; /* DOF_STORAGE_F32, or DOF_STORAGE_F16: colour image buffers of the
                               pass in FP16 (arithmetic stays FP32; depth, CoC and history FP32) */
    float taa_alpha;        /* final TAA (Section 3.4) blend of the current frame, 0 < a <= 1;
                               0 = no TAA (the history needs DOF_HIST_TAA otherwise) */
    uint32_t aperture_blades; /* aperture shape (Section 1.1: bokeh takes the shape of an n-blade
                               diaphragm; Section 2.2: the kernel's shape can be changed to
                               produce it): 0 = circle; 3..8 = regular n-gon inscribed in the
                               circle, a vertex along the camera's right axis.  The thin-lens
                               samples are uniform over it, the 81-tap kernels of the main filter
                               and the reconstruction lie on it, sampleAlpha divides by its area.
                               Other values: DOF_ERR_INVALID_ARG. */
} DofParams;

#define DOF_STORAGE_F32 0
#define DOF_STORAGE_F16 1

#define DOF_MAX_RAYS 64

typedef struct {
    const float *color;     /* W*H float4: sharp all-in-focus colour (rgb, unused) */
    const float *depth;     /* W*H float: depth along the optical axis, +inf = sky */
    const float *normal;    /* W*H float4: surface normal (xyz, unused); read in adaptive mode */
    uint32_t width, height; /* full resolution, both even and >= 2 */
    uint32_t fmt;           /* DOF_FMT_F32 or DOF_FMT_F16; rows tightly packed */
} DofGBuffer;

typedef struct DofCtx DofCtx;
typedef struct DofScene DofScene;
typedef struct DofHistory DofHistory;

typedef struct {
    uint32_t n_tris, n_nodes, depth, stack_limit;
    uint64_t device_bytes;
    float bounds_lo[3], bounds_hi[3];   /* bounds of the triangles in the tree */
    uint32_t n_large;                   /* large triangles kept out of the tree */
    uint32_t n_nodes4;                  /* nodes of the 4-wide tree (0 when the tree is one leaf) */
    uint32_t depth4;                    /* levels of the 4-wide tree */
    uint32_t pad;
} DofSceneInfo;

typedef struct {
    uint64_t frames;           /* frames run on this history */
    uint32_t masked_pixels;    /* last frame: half-resolution pixels with rays */
    uint32_t rays;             /* last frame: rays traced */
    int32_t device_status;     /* DOF_OK or the first device-side error */
    uint32_t pad;
    uint64_t node_visits;      /* last frame: BVH nodes visited by the thin-lens rays (0 with
                                  warp packets and DOF_OPT_TRACE_STATS = 0) */
    uint64_t tri_tests;        /* last frame: ray/triangle tests of the thin-lens rays (idem) */
} DofFrameStats;

/* ---- context ----------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  mem_budget_bytes (0 = unlimited) caps
 * the device memory that scenes and histories of this context may hold; an upload or
 * history that would exceed it fails with DOF_ERR_BUDGET.  Owns nothing of the
 * caller's. */
int dof_ctx_create(int device, size_t mem_budget_bytes, DofCtx **out);
void dof_ctx_destroy(DofCtx *ctx);
/* bytes currently held by the context's scenes and histories */
size_t dof_ctx_bytes_in_use(const DofCtx *ctx);

/* Context options (dof_ctx_set_option). */
#define DOF_OPT_BVH_BUILDER 1
#define DOF_BVH_PLOC 0   /* default: PLOC clustering over the Morton order (higher tree quality) */
#define DOF_BVH_LBVH 1   /* Karras 2012 radix tree (faster build) */
/* launch shape and scheduling of the persistent ray tracer (results do not depend on them) */
#define DOF_OPT_TRACE_BLOCKS_PER_SM 2   /* 128-thread blocks per SM, 1..32 (default 8) */
#define DOF_OPT_TRACE_REFILL_IDLE   3   /* refill a warp when this many lanes are idle, 1..32 (default 16) */
#define DOF_OPT_TRACE_STEPS         4   /* traversal steps between refill checks, 1..256 (default 64) */
#define DOF_OPT_PLOC_RADIUS         5   /* PLOC nearest-neighbour search radius, 1..256 (default 48) */
#define DOF_OPT_BVH_WIDTH           6   /* tree the rays traverse: 4 (default) = the binary tree collapsed
                                         * to 4-wide nodes, 2 = the binary tree; same hits either way */
#define DOF_OPT_RAY_ORDER_GRID      7   /* order in which the tracer takes a block's rays: grouped by the
                                         * cell of their lens point on a g x g grid over the aperture,
                                         * g = 1..16 (default 4), cells in Morton order; 1 = pixel by
                                         * pixel.  Same hits either way */
/* block of the main filter's 81-tap gather in half-resolution pixels: value = width |
 * height << 16, width >= 8, width * height a multiple of 32 in 64..512 (default 32 x 8) */
#define DOF_OPT_GATHER_BLOCK        8
/* the main filter's reads: 0 (default) = the block's halo tile staged in shared memory when
 * it fits in 64 KB, else through L1; 1 = always through L1; 2 = the halo tile whenever it
 * fits in the SM's opt-in shared memory; 3 = through L1, each thread taking a column of four
 * pixels of one 8 x 8 tile (they share the tile's radius, so their taps share texel rows).
 * Same results either way */
#define DOF_OPT_MAIN_FILTER_FORM    9
/* block of the reconstruction's 81-tap gather, encoded as DOF_OPT_GATHER_BLOCK (default 32 x 8) */
#define DOF_OPT_RECON_BLOCK         10
/* entries of the tracer's per-ray traversal stack, 1..96 (default 96); the launch takes the
 * smallest compiled capacity (32, 64, 96) that holds both this and what the batch's trees
 * can need, so a small value never overflows.  Same hits either way */
#define DOF_OPT_TRACE_STACK         11
/* how the binary tree is traversed: 0 (default) = one ray per lane, persistent threads with
 * dynamic fetch; 1 = the 32 rays of a warp as one packet (one node sequence per warp, each lane
 * testing with its own ray and best hit); packets always traverse the binary tree, whatever
 * DOF_OPT_BVH_WIDTH says.  Same hits either way */
#define DOF_OPT_TRACE_PACKETS       12
/* passes of tree rotations after the BVH build of scenes uploaded afterwards, 0..16
 * (default 0): each swaps, bottom-up, a child with a grandchild where that shrinks the
 * child's box.  Same hits either way */
#define DOF_OPT_BVH_ROTATIONS       13
/* whether the warp-packet tracer counts node visits and triangle tests for
 * DofFrameStats: 1 (default) counts, 0 leaves both at 0 for its frames (2% of the
 * tracer's time at 4K).  Same hits either way */
#define DOF_OPT_TRACE_STATS         14
int dof_ctx_set_option(DofCtx *ctx, int option, int64_t value);

/* Fill `p` with the defaults above (1 spp fixed mode, 16 px radius clamp). */
void dof_params_default(DofParams *p);

/* Thread-local message of the last error on this thread ("" if none). */
const char *dof_last_error(void);

/* ---- scene (Section 4.2: the acceleration structure) ------------------------- */

/* Upload a triangle scene and build its BVH on the device from 63-bit Morton codes of
 * the triangle centroids: PLOC agglomerative clustering (Meister and Bittner 2018)
 * by default, or the LBVH radix tree of Karras 2012 (DOF_OPT_BVH_BUILDER); two child
 * boxes per node.  The binary tree is then collapsed top-down into nodes of four child
 * boxes (the largest-area child is opened until four remain).  Up to 64
 * "large" triangles (box extent above 1/16 of the scene's centroid extent, e.g. a
 * ground plane) are kept out of the tree and tested directly by every ray.
 *   xyz      host, n_verts * 3 floats
 *   tri_idx  host, n_tris * 3 vertex indices (< n_verts, checked)
 *   tri_mat  host, n_tris material ids (0 diffuse with hash albedo, 1 emitter), or NULL
 * The finished binary tree is checked before the call returns: every child reference
 * in range, and every node but the root, and every leaf, referenced exactly once.  A
 * tree that fails returns DOF_ERR_DEVICE_CHECK; the warp-packet traversal relies on the
 * check instead of a per-step guard.
 * The call copies the data, builds on `stream` and synchronises that stream before
 * returning (the scene is then immutable and usable from any stream).  The library
 * owns the returned scene; release it with dof_scene_destroy. */
int dof_scene_upload(DofCtx *ctx, const float *xyz, uint32_t n_verts, const uint32_t *tri_idx,
                     const uint32_t *tri_mat, uint32_t n_tris, void *stream, DofScene **out);
void dof_scene_destroy(DofScene *scene);
int dof_scene_info(const DofScene *scene, DofSceneInfo *info);

/* ---- G-buffer producer (input harness, Section 3 deferred shading) ----------- */

/* Pinhole primary visibility of `scene` through the camera's lens centre at each
 * full-resolution pixel centre: colour (float4, shaded as the rays of dof_frame,
 * sky on a miss), depth (float, +inf on a miss), normal (float4, face normal turned
 * towards the camera, 0 on a miss), prim (int32 triangle id, -1 on a miss; may be
 * NULL).  All outputs are caller-owned device buffers of width*height elements. */
int dof_gbuffer(DofCtx *ctx, const DofScene *scene, const DofCamera *cam, const DofParams *p,
                uint32_t width, uint32_t height, float *color, float *depth, float *normal,
                int32_t *prim, void *stream);

/* Same outputs as dof_gbuffer, bit for bit, produced object-order: every triangle is
 * set up once (the three planes through the lens centre and its edges bound the pixel
 * centres that can see it), the pixels of that conservative region run the same
 * watertight ray/triangle test, and the closest hit per pixel is kept by a 64-bit
 * atomic minimum of (distance bits, triangle id), then shaded.  Scratch (8 bytes per
 * pixel plus 68 bytes per triangle) comes from a stream-ordered pool that the context
 * keeps until it is destroyed; the call does not synchronise `stream`. */
int dof_gbuffer_raster(DofCtx *ctx, const DofScene *scene, const DofCamera *cam, const DofParams *p,
                       uint32_t width, uint32_t height, float *color, float *depth, float *normal,
                       int32_t *prim, void *stream);

/* ---- per-session history (Section 3.2.3) ------------------------------------- */

#define DOF_HIST_RECORD_RAYS 1u   /* also keep each ray's hit triangle id (tests) */
#define DOF_HIST_TIMING      2u   /* record a CUDA event after every kernel of a frame */
#define DOF_HIST_TAA         4u   /* keep the final TAA's image history (3 x 16 B per pixel) */

/* Session state for width x height frames: accumulated ray-traced layer (FP32),
 * blurred variance, and the per-frame work buffers of the pass.  max_rays (1..64)
 * bounds spp / m of the frames run on it.  Owned by the library. */
int dof_history_create(DofCtx *ctx, uint32_t width, uint32_t height, uint32_t max_rays,
                       uint32_t flags, DofHistory **out);
void dof_history_destroy(DofHistory *hist);
/* forget the accumulated history (the next frame restarts accumulation) */
int dof_history_reset(DofHistory *hist);

/* Checkpoint / resume of a session (the paper has none; the FP32 history is the whole
 * state a frame carries to the next, and the lens samples are counter-based, so a
 * session resumed from a checkpoint continues bit-identically).
 * export: with host_buf NULL, *bytes receives the size needed; otherwise *bytes must
 *   be at least that size, the history is copied into caller-owned host memory after
 *   synchronising `stream`, and *bytes is set to the size written.
 * import: the buffer must come from an export of a history of the same width, height
 *   and max_rays (DOF_ERR_MISMATCH otherwise); synchronises `stream`. */
int dof_history_export(DofHistory *hist, void *host_buf, size_t *bytes, void *stream);
int dof_history_import(DofHistory *hist, const void *host_buf, size_t bytes, void *stream);

/* ---- one frame ----------------------------------------------------------------- */

/* Run the hybrid depth-of-field pass for one frame on `stream`:
 *   gbuf   the frame's G-buffer (device, caller-owned, read only)
 *   cam    camera of this frame and pose of the previous one (host struct)
 *   p      method parameters (host struct)
 *   hist   the session's history: read and updated in place (the pass is
 *          stream-ordered; frames of one history must not overlap)
 *   out    device, width*height float4: composited image (rgb, 1)
 * Host-side validation errors return before anything is enqueued. */
int dof_frame(DofCtx *ctx, const DofScene *scene, const DofGBuffer *gbuf, const DofCamera *cam,
              const DofParams *p, DofHistory *hist, float *out, void *stream);

/* One frame from and to host memory.  color (W*H float4), depth (W*H float) and, in
 * the adaptive ray mode, normal (W*H float4; else may be NULL) are host buffers in the
 * layout of DofGBuffer; out (W*H float4) receives the composited image, as dof_frame
 * writes it; W, H are the history's.  The history keeps two device slots used in
 * turn and one copy stream per direction: the inputs are copied in once the frame two
 * calls back is done with the slot, the pass runs on `stream` after its inputs, and
 * the image is copied out once the pass is done, so the copies of one frame overlap
 * the passes of its neighbours.  The call returns once all of it is enqueued (with
 * pageable host memory the driver may copy synchronously; pinned memory overlaps).
 * The caller keeps the inputs unchanged and leaves `out` unread until the frame's
 * copy-out has completed: dof_frame_host_join(hist, s) makes stream `s` wait for the
 * copy-outs enqueued so far.  The slots (52 B per pixel) are allocated on first use. */
int dof_frame_host(DofCtx *ctx, const DofScene *scene, const float *color, const float *depth,
                   const float *normal, const DofCamera *cam, const DofParams *p, DofHistory *hist,
                   float *out, void *stream);
int dof_frame_host_join(DofHistory *hist, void *stream);

/* One session's frame of a batch. */
typedef struct {
    const DofScene *scene;
    const DofGBuffer *gbuf;
    const DofCamera *cam;
    const DofParams *params;
    DofHistory *hist;
    float *out;
} DofFrameReq;

#define DOF_MAX_BATCH 32

/* Frames of up to DOF_MAX_BATCH sessions (different sizes, scenes and parameters
 * allowed; each history at most once) in one launch per pass on `stream`: every
 * kernel covers the blocks of all the sessions, and the thin-lens rays of all the
 * sessions share one persistent tracer launch.  Each result is the one dof_frame
 * gives for that session alone (bit-identical).  Validation as dof_frame; nothing is
 * enqueued if any request is invalid.  Traversal counters of the batch are reported
 * by dof_frame_stats of the first request's history. */
int dof_batch_frame(DofCtx *ctx, const DofFrameReq *reqs, uint32_t n, void *stream);

/* ---- captured steps (CUDA graphs; no counterpart in the paper) --------------------
 * A step of dof_batch_frame over a fixed set of sessions, captured once as a CUDA graph
 * and replayed per frame: one graph launch instead of the step's ~20 kernel launches.
 * The kernels of the graph read the batch descriptor from device memory, which a copy
 * node refreshes from a pinned staging buffer at the start of every replay, so cameras,
 * parameters, G-buffer and output pointers may change between launches.
 *   dof_graph_create: validates `reqs` as dof_batch_frame and captures (nothing runs,
 *     the histories do not advance).  The graph keeps the histories and their order,
 *     the launch shapes (sizes, ray modes, spp / m, tree kinds, the main filter's
 *     shared-memory tile, which follows max_coc_px) and the context's tracer options of
 *     that moment.
 *   dof_graph_launch: one step, results identical to dof_batch_frame on the same
 *     requests.  DOF_ERR_MISMATCH if the requests need other launch shapes or other
 *     histories than the capture.  Launches of one graph on different streams are
 *     ordered by the library (one graph runs one step at a time).
 *   dof_graph_destroy: waits for the graph's last launch and frees it. */
typedef struct DofGraph DofGraph;
int dof_graph_create(DofCtx *ctx, const DofFrameReq *reqs, uint32_t n, DofGraph **out);
int dof_graph_launch(DofGraph *g, const DofFrameReq *reqs, uint32_t n, void *stream);
void dof_graph_destroy(DofGraph *g);

/* Kernel launches this library has enqueued in this process so far (frame passes, the
 * G-buffer producers and the allocation-free tile map; a replayed graph counts the
 * kernels it holds; scene builds are not counted).  Host-side tally, no synchronisation. */
unsigned long long dof_launch_count(void);

/* Synchronise `stream` and report the last frame's counters and the device status. */
int dof_frame_stats(DofHistory *hist, void *stream, DofFrameStats *out);

/* Timing slots of one frame, in launch order (DOF_HIST_TIMING brackets each with events).
 * DILATE, VAR_BLUR and MIPS are fused into PREFILTER / MASK, MEDIAN_RT and MEDIAN_RT
 * respectively: their slots bracket no kernel and count 0.  TRACE times whichever tracer
 * runs (one ray per lane, or warp packets with DOF_OPT_TRACE_PACKETS). */
enum {
    DOF_K_DOWNSCALE = 0, DOF_K_DILATE, DOF_K_PREFILTER, DOF_K_MAIN, DOF_K_MEDIAN_PP, DOF_K_EDGES,
    DOF_K_MASK, DOF_K_TRACE, DOF_K_SHADE, DOF_K_ACCUM, DOF_K_VAR_BLUR, DOF_K_MEDIAN_RT, DOF_K_MIPS,
    DOF_K_RECON, DOF_K_COMPOSITE, DOF_K_TAA, DOF_K_COUNT
};
/* For a history created with DOF_HIST_TIMING: synchronise `stream`, add the device
 * time (ms) each kernel took, summed over the frames recorded since the previous call
 * (at most 64), to ms[0..DOF_K_COUNT-1] after zeroing it, and return that frame
 * count in *frames.  Kernels not launched in a frame (e.g. EDGES in fixed mode)
 * count 0. */
int dof_kernel_times(DofHistory *hist, void *stream, float *ms, uint32_t *frames);

/* ---- inspection (tests, tools) ------------------------------------------------- */

/* Intermediate buffers of the last frame, for parity tests.  Element layouts (N = W/2 *
 * H/2 half-resolution pixels, row-major; TW x TH = ceil(W/2/8) x ceil(H/2/8) tiles):
 *   PP_IN  float4 N  (rgb, rho)         Z_H     float N
 *   TILES  float2 TW*TH (near, |rho|)   TILES_DIL float2 TW*TH
 *   PRE    float4 N  (rgb, rho)         MAIN    float4 N (rgb, bright)
 *   PP_MED float4 N                      XN, XF  float N (adaptive mode only)
 *   NRAYS  int32 N                        RAY_PRIM int32 N*max_rays (DOF_HIST_RECORD_RAYS)
 *   RT     float4 4N: planes (An, h), (Af, n), (Bn, Bf, Fw, 0), (Pfar, 0)
 *   CRT    float4 N (rgb, h)             CT, VAR, VAR_BLUR float N
 *   RT_MED float4 N                       RECON   float4 N (rgb, h)
 *   HIST   float4 3N: planes (An, h), (Af, g), (Bn, Bf, mu1, var) -- luminance mean and variance
 * With DOF_STORAGE_F16 the colour buffers MAIN, PP_MED, CRT, RT_MED and RECON hold N half4
 * in their first 8N bytes, and PRE holds per pixel a 16-byte record: (r, g) and (b, 0) as
 * half2, then rho and the depth as floats.
 * *dev_ptr is owned by the history and valid until the next call that uses it. */
enum {
    DOF_BUF_PP_IN = 0, DOF_BUF_Z_H, DOF_BUF_TILES, DOF_BUF_TILES_DIL, DOF_BUF_PRE,
    DOF_BUF_MAIN, DOF_BUF_PP_MED, DOF_BUF_XN, DOF_BUF_XF, DOF_BUF_NRAYS, DOF_BUF_RAY_PRIM,
    DOF_BUF_RT, DOF_BUF_CRT, DOF_BUF_CT, DOF_BUF_VAR, DOF_BUF_VAR_BLUR, DOF_BUF_RT_MED,
    DOF_BUF_RECON, DOF_BUF_HIST, DOF_BUF_COMPOSITE, DOF_BUF_COUNT
};
int dof_debug_buffer(DofHistory *hist, int which, void **dev_ptr, size_t *bytes);
/* Synchronous copy of intermediate buffer `which` into caller-owned host memory of
 * `bytes` bytes (must equal the buffer's size); waits for all work on the device. */
int dof_debug_read(DofHistory *hist, int which, void *host_dst, size_t bytes);

/* ---- allocation-free tile map ------------------------------------------------ */

/* No counterpart in the paper: a convenience for hosts that cannot allocate device
 * memory when they need the tile map -- e.g. an engine whose allocator reserved all
 * device memory up front, or a frame loop where cudaMalloc/cudaFree would implicitly
 * synchronise the device.  Computes the same dilated tile map as dof_frame's tile
 * stage (DOF_BUF_TILES_DIL: per 8x8 half-resolution tile the max near CoC radius and
 * max |rho|, dilated over the tile neighbourhood) from a full-resolution depth map,
 * and allocates nothing: its one intermediate (the undilated tiles) lives in a
 * built-in device array of DOF_NOALLOC_MAX_TILES tiles (512 KB, held by every GPU
 * that loads the library until the process exits).
 *   depth      device, width*height floats (8-byte aligned), read only
 *   tiles_dil  device, ceil(width/16)*ceil(height/16) float2 (8-byte aligned), written
 *   cam, p     only the lens (f, N, focus, sensor width), tile, max_coc_px and z_far_m
 *              are used
 * Sizes whose tile count exceeds DOF_NOALLOC_MAX_TILES, sizes above 16384 and lens
 * values that are not finite return DOF_ERR_INVALID_ARG.
 * Every call looks up the array's address in the current device's context with
 * cudaGetSymbolAddress (nothing is cached, so the call stays valid after a device
 * reset or from another context); the first call in a context also loads the
 * library's device code there, so make that first call before any stream capture.
 * Every call shares
 * the array and it keeps the previous call's contents (each call overwrites what it
 * reads); calls that overlap on the GPU race on it and must be serialised by the
 * caller.  Enqueued on `stream`; returns without synchronising. */
#define DOF_NOALLOC_MAX_TILES 65536
int dof_coc_tiles_noalloc(const float *depth, uint32_t width, uint32_t height, const DofCamera *cam,
                          const DofParams *p, float *tiles_dil, void *stream);

#ifdef __cplusplus
}
#endif
#endif

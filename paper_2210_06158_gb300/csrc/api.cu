// C ABI of libdof (include/dof.h): contexts, scenes, histories, and the per-frame
// orchestration of the pass on one CUDA stream.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include "batch.cuh"

int post_init_tables();
int recon_init_tables();

// ---------------------------------------------------------------------------
// errors and allocation
// ---------------------------------------------------------------------------

static thread_local char g_err[512] = "";

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches += n; }
extern "C" unsigned long long dof_launch_count(void) { return (unsigned long long)g_launches.load(); }

int dof_set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int dof_cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return DOF_OK;
    cudaGetLastError();
    int code = e == cudaErrorMemoryAllocation ? DOF_ERR_OOM : DOF_ERR_CUDA;
    return dof_set_error(code, "%s: %s", what, cudaGetErrorString(e));
}

int dof_alloc(DofCtx *ctx, size_t bytes, void **ptr, size_t *acc) {
    *ptr = nullptr;
    if (bytes == 0) return DOF_OK;
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return dof_set_error(DOF_ERR_BUDGET, "allocation of %zu bytes exceeds the budget (%zu of %zu in use)", bytes,
                             (size_t)ctx->in_use, ctx->budget);
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return dof_cuda_check(e, "cudaMalloc");
    }
    ctx->in_use += bytes;
    if (acc) *acc += bytes;
    return DOF_OK;
}

void dof_free(DofCtx *ctx, void *ptr, size_t bytes) {
    if (!ptr) return;
    cudaFree(ptr);
    ctx->in_use -= bytes;
}

namespace {

// makes `dev` current for the duration of an API call and restores the caller's device;
// also drops a stale error that another library left on this thread, so that the
// call reports only its own errors
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetLastError();
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) {
            cudaError_t e = cudaSetDevice(dev);
            if (e != cudaSuccess) {
                if (getenv("DOF_DEBUG")) fprintf(stderr, "libdof: cudaSetDevice(%d) failed: %s\n", dev, cudaGetErrorString(e));
                cudaGetLastError();
            }
        }
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite3(const float *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

int make_cam(const DofCamera *c, uint32_t W, uint32_t H, DevCam &o) {
    if (!(c->f_m > 0.f) || !(c->f_number > 0.f) || !(c->sensor_w_m > 0.f) || !(c->focus_m > c->f_m) ||
        !isfinite(c->f_m) || !isfinite(c->focus_m) || !isfinite(c->sensor_w_m))
        return dof_set_error(DOF_ERR_INVALID_ARG, "camera: need f > 0, N > 0, w_s > 0 and focus > f");
    const float *vs[8] = {c->pos, c->right, c->up, c->fwd, c->prev_pos, c->prev_right, c->prev_up, c->prev_fwd};
    for (auto v : vs)
        if (!finite3(v)) return dof_set_error(DOF_ERR_INVALID_ARG, "camera: pose is not finite");
    double f = c->f_m, N = c->f_number, d = c->focus_m, ws = c->sensor_w_m;
    double a = f / N, v = f * d / (d - f), F = (double)W * v / ws;
    auto f3 = [](const float *x) { return make_float3(x[0], x[1], x[2]); };
    o.O = f3(c->pos); o.R = f3(c->right); o.U = f3(c->up); o.F = f3(c->fwd);
    o.pO = f3(c->prev_pos); o.pR = f3(c->prev_right); o.pU = f3(c->prev_up); o.pF = f3(c->prev_fwd);
    o.Fpx = (float)F;
    o.invF = (float)(1.0 / F);
    o.cocK = (float)(a * f * (double)W / (ws * (d - f)));
    o.d = c->focus_m;
    o.lens_r = (float)(0.5 * a);
    o.halfW = 0.5f * (float)W;
    o.halfH = 0.5f * (float)H;
    o.W = (int)W; o.H = (int)H; o.W2 = (int)W / 2; o.H2 = (int)H / 2;
    o.frame = c->frame_index;
    o.moved = memcmp(c->pos, c->prev_pos, 12) || memcmp(c->right, c->prev_right, 12) ||
              memcmp(c->up, c->prev_up, 12) || memcmp(c->fwd, c->prev_fwd, 12);
    for (int k = 0; k < 2; k++)
        if (!(fabsf(c->jitter[k]) <= 1.f) || !(fabsf(c->prev_jitter[k]) <= 1.f))
            return dof_set_error(DOF_ERR_INVALID_ARG, "camera: jitter outside [-1, 1] px");
    o.jx = c->jitter[0]; o.jy = c->jitter[1];
    o.pjx = c->prev_jitter[0]; o.pjy = c->prev_jitter[1];
    o.exact = !o.moved && memcmp(c->jitter, c->prev_jitter, 8) == 0;
    return DOF_OK;
}

int make_params(const DofParams *p, uint32_t W, uint32_t H, uint32_t max_rays, DevParams &o) {
    if (p->tile != 8) return dof_set_error(DOF_ERR_INVALID_ARG, "params: tile must be 8");
    if (p->ray_mode > 1) return dof_set_error(DOF_ERR_INVALID_ARG, "params: ray_mode must be 0 or 1");
    if (p->ray_mode == 0 && (p->spp < 1 || p->spp > max_rays))
        return dof_set_error(DOF_ERR_INVALID_ARG, "params: spp %u outside 1..%u", p->spp, max_rays);
    if (p->ray_mode == 1 && (p->m < 1 || p->m > max_rays))
        return dof_set_error(DOF_ERR_INVALID_ARG, "params: m %u outside 1..%u", p->m, max_rays);
    if (!(p->max_coc_px >= 1.f && p->max_coc_px <= 256.f))
        return dof_set_error(DOF_ERR_INVALID_ARG, "params: max_coc_px must be in [1, 256]");
    if (!(p->lod_max >= 0.f && p->lod_max <= 3.f))
        return dof_set_error(DOF_ERR_INVALID_ARG, "params: lod_max must be in [0, 3]");
    if (!(p->depth_range_m > 0.f) || !(p->cover_ramp_px > 0.f) || !(p->zof_ramp_px > 0.f) ||
        !(p->bright_ramp > 0.f) || !(p->h_edge > 0.f) || !(p->z_far_m > 0.f))
        return dof_set_error(DOF_ERR_INVALID_ARG, "params: ranges and ramps must be positive");
    double l = sqrt((double)p->light_dir[0] * p->light_dir[0] + (double)p->light_dir[1] * p->light_dir[1] +
                    (double)p->light_dir[2] * p->light_dir[2]);
    if (!(l > 0.0)) return dof_set_error(DOF_ERR_INVALID_ARG, "params: light_dir is zero");
    o.s = p->s; o.var_w_mask = p->var_w_mask; o.m = (float)p->m;
    o.spp = (int)p->spp; o.ray_mode = (int)p->ray_mode;
    o.inv_depth_range = (float)(1.0 / p->depth_range_m);
    o.alpha = p->alpha; o.alpha_motion = p->alpha_motion;
    o.var_w_recon = p->var_w_recon; o.b_max = p->b_max; o.h_edge = p->h_edge;
    o.lod_scale = p->lod_scale; o.lod_max = p->lod_max;
    o.rmax_hpx = 0.5f * p->max_coc_px;
    o.zof_ramp = p->zof_ramp_px;
    o.inv_cover_ramp = (float)(1.0 / p->cover_ramp_px);
    o.bright_lum = p->bright_lum;
    o.inv_bright_ramp = (float)(1.0 / p->bright_ramp);
    o.mask_near_hpx = p->mask_near_hpx;
    o.z_far = p->z_far_m;
    o.albedo_seed = p->albedo_seed;
    o.seed = p->seed; o.session = p->session;
    o.light = make_float3((float)(p->light_dir[0] / l), (float)(p->light_dir[1] / l), (float)(p->light_dir[2] / l));
    o.k_a = p->k_a; o.k_d = p->k_d; o.emit = p->emit;
    o.sky = make_float3(p->sky[0], p->sky[1], p->sky[2]);
    uint32_t W2 = W / 2, H2 = H / 2;
    if (p->image_storage > 1) return dof_set_error(DOF_ERR_INVALID_ARG, "params: image_storage must be 0 or 1");
    o.f16 = p->image_storage == DOF_STORAGE_F16;
    if (!(p->taa_alpha >= 0.f && p->taa_alpha <= 1.f))
        return dof_set_error(DOF_ERR_INVALID_ARG, "params: taa_alpha must be in [0, 1]");
    o.taa_alpha = p->taa_alpha;
    if (p->aperture_blades != 0 && (p->aperture_blades < 3 || p->aperture_blades > 8))
        return dof_set_error(DOF_ERR_INVALID_ARG, "params: aperture_blades must be 0 or 3..8");
    o.blades = (int)p->aperture_blades;
    o.ring = o.blades ? o.blades - 2 : 0;
    {
        const double kPi = 3.14159265358979323846;
        const double A = o.blades ? 0.5 * o.blades * sin(2.0 * kPi / o.blades) : kPi;
        o.inv_area = (float)(1.0 / A);
        o.inv_sqrt_area = (float)(1.0 / sqrt(A));
    }
    o.tiles_w = (int)((W2 + 7) / 8);
    o.tiles_h = (int)((H2 + 7) / 8);
    o.dil_k = (int)ceil(0.5 * (double)p->max_coc_px / 8.0);
    return DOF_OK;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

extern "C" const char *dof_last_error(void) { return g_err; }

extern "C" void dof_params_default(DofParams *p) {
    memset(p, 0, sizeof(*p));
    p->s = 0.8f; p->var_w_mask = 1e5f; p->m = 10; p->spp = 1; p->ray_mode = 0;
    p->depth_range_m = 0.10f; p->alpha = 0.95f; p->alpha_motion = 0.8f;
    p->var_w_recon = 2000.f; p->b_max = 0.9f; p->h_edge = 0.3f;
    p->lod_scale = 0.05f; p->lod_max = 3.f; p->max_coc_px = 16.f;
    p->zof_ramp_px = 0.25f; p->cover_ramp_px = 1.f; p->bright_lum = 4.f; p->bright_ramp = 1.f;
    p->mask_near_hpx = 0.5f; p->z_far_m = 1e5f; p->tile = 8; p->albedo_seed = 1;
    p->seed = 1; p->session = 0;
    p->light_dir[0] = 0.3f; p->light_dir[1] = -1.f; p->light_dir[2] = 0.5f;
    p->k_a = 0.1f; p->k_d = 1.f;
    p->sky[0] = 0.5f; p->sky[1] = 0.6f; p->sky[2] = 0.8f;
    p->emit = 8.f;
}

extern "C" int dof_ctx_create(int device, size_t mem_budget_bytes, DofCtx **out) {
    if (!out) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_ctx_create: out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return dof_cuda_check(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_ctx_create: no device %d", device);
    DeviceGuard g(device);
    DofCtx *c = new DofCtx();
    c->device = device;
    c->budget = mem_budget_bytes;
    c->in_use = 0;
    c->refs = 1;
    c->bvh_builder = DOF_BVH_PLOC;
    c->trace_blocks_per_sm = 8;
    c->trace_refill_idle = 16;
    c->trace_steps = 64;
    c->ray_order_grid = 4;
    c->trace_packets = 0;
    c->trace_stats = 1;
    c->stack_depth = kTraversalStack;
    c->gather_w = 32;
    c->gather_h = 8;
    c->recon_w = 32;
    c->recon_h = 8;
    c->main_form = 0;
    c->ploc_radius = 48;
    c->bvh_width = 4;
    c->bvh_rotations = 0;
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    preload_trace_kernels();
    preload_post_kernels();
    preload_recon_kernels();
    if (cudaMalloc(&c->d_status, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return dof_set_error(DOF_ERR_OOM, "dof_ctx_create: status word");
    }
    int prio_least = 0, prio_greatest = 0;
    cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (cudaStreamCreateWithPriority(&c->ray_stream, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->ray_stream) cudaStreamDestroy(c->ray_stream);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        cudaFree(c->d_status);
        delete c;
        return dof_set_error(DOF_ERR_CUDA, "dof_ctx_create: stream or events");
    }
    {
        // scratch of dof_gbuffer_raster: kept in the pool between calls
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        } else {
            cudaGetLastError();
            c->pool = nullptr;
        }
    }
    if (post_init_tables() != 0 || recon_init_tables() != 0) {
        cudaFree(c->d_status);
        delete c;
        return dof_set_error(DOF_ERR_CUDA, "dof_ctx_create: uploading filter tables failed");
    }
    *out = c;
    return DOF_OK;
}

extern "C" int dof_ctx_set_option(DofCtx *ctx, int option, int64_t value) {
    if (!ctx) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_ctx_set_option: null context");
    switch (option) {
        case DOF_OPT_BVH_BUILDER:
            if (value != DOF_BVH_PLOC && value != DOF_BVH_LBVH)
                return dof_set_error(DOF_ERR_INVALID_ARG, "dof_ctx_set_option: unknown BVH builder %lld", (long long)value);
            ctx->bvh_builder = (int)value;
            return DOF_OK;
        case DOF_OPT_TRACE_BLOCKS_PER_SM:
            if (value < 1 || value > 32) return dof_set_error(DOF_ERR_INVALID_ARG, "trace blocks per SM must be 1..32");
            ctx->trace_blocks_per_sm = (int)value;
            return DOF_OK;
        case DOF_OPT_TRACE_REFILL_IDLE:
            if (value < 1 || value > 32) return dof_set_error(DOF_ERR_INVALID_ARG, "refill threshold must be 1..32");
            ctx->trace_refill_idle = (int)value;
            return DOF_OK;
        case DOF_OPT_PLOC_RADIUS:
            if (value < 1 || value > 256) return dof_set_error(DOF_ERR_INVALID_ARG, "PLOC radius must be 1..256");
            ctx->ploc_radius = (int)value;
            return DOF_OK;
        case DOF_OPT_BVH_WIDTH:
            if (value != 2 && value != 4) return dof_set_error(DOF_ERR_INVALID_ARG, "BVH width must be 2 or 4");
            ctx->bvh_width = (int)value;
            return DOF_OK;
        case DOF_OPT_TRACE_STEPS:
            if (value < 1 || value > 256) return dof_set_error(DOF_ERR_INVALID_ARG, "steps per round must be 1..256");
            ctx->trace_steps = (int)value;
            return DOF_OK;
        case DOF_OPT_RAY_ORDER_GRID:
            if (value < 1 || value > 16) return dof_set_error(DOF_ERR_INVALID_ARG, "ray order grid must be 1..16");
            ctx->ray_order_grid = (int)value;
            return DOF_OK;
        case DOF_OPT_TRACE_PACKETS:
            if (value != 0 && value != 1) return dof_set_error(DOF_ERR_INVALID_ARG, "trace packets must be 0 or 1");
            ctx->trace_packets = (int)value;
            return DOF_OK;
        case DOF_OPT_TRACE_STATS:
            if (value != 0 && value != 1) return dof_set_error(DOF_ERR_INVALID_ARG, "trace stats must be 0 or 1");
            ctx->trace_stats = (int)value;
            return DOF_OK;
        case DOF_OPT_BVH_ROTATIONS:
            if (value < 0 || value > 16) return dof_set_error(DOF_ERR_INVALID_ARG, "BVH rotation passes must be 0..16");
            ctx->bvh_rotations = (int)value;
            return DOF_OK;
        case DOF_OPT_GATHER_BLOCK:
        case DOF_OPT_RECON_BLOCK: {
            const long long w = value & 0xFFFF, h = (value >> 16) & 0xFFFF;
            if (value < 0 || (value >> 32) || w < 8 || h < 1 || (w * h) % 32 || w * h < 64 || w * h > 512)
                return dof_set_error(DOF_ERR_INVALID_ARG, "gather block: width >= 8, whole warps, 64..512 threads");
            if (option == DOF_OPT_GATHER_BLOCK) {
                ctx->gather_w = (int)w;
                ctx->gather_h = (int)h;
            } else {
                ctx->recon_w = (int)w;
                ctx->recon_h = (int)h;
            }
            return DOF_OK;
        }
        case DOF_OPT_TRACE_STACK:
            if (value < 1 || value > kTraversalStack)
                return dof_set_error(DOF_ERR_INVALID_ARG, "trace stack depth must be 1..%d", kTraversalStack);
            ctx->stack_depth = (int)value;
            return DOF_OK;
        case DOF_OPT_MAIN_FILTER_FORM:
            if (value < 0 || value > 3) return dof_set_error(DOF_ERR_INVALID_ARG, "main filter form must be 0..3");
            ctx->main_form = (int)value;
            return DOF_OK;
        default:
            return dof_set_error(DOF_ERR_INVALID_ARG, "dof_ctx_set_option: unknown option %d", option);
    }
}

void ctx_retain(DofCtx *ctx) { ctx->refs++; }

void ctx_release(DofCtx *ctx) {
    if (--ctx->refs == 0) {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->ray_stream);
        cudaStreamDestroy(ctx->ray_stream);
        cudaEventDestroy(ctx->ev_fork);
        cudaEventDestroy(ctx->ev_join);
        if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
        cudaFree(ctx->d_status);
        delete ctx;
    }
}

// The context lives on until its last scene and history are destroyed, so handles may
// be released in any order.
extern "C" void dof_ctx_destroy(DofCtx *ctx) {
    if (ctx) ctx_release(ctx);
}

extern "C" size_t dof_ctx_bytes_in_use(const DofCtx *ctx) { return ctx ? (size_t)ctx->in_use : 0; }

// ---------------------------------------------------------------------------
// scene
// ---------------------------------------------------------------------------

extern "C" int dof_scene_upload(DofCtx *ctx, const float *xyz, uint32_t n_verts, const uint32_t *tri_idx,
                                const uint32_t *tri_mat, uint32_t n_tris, void *stream, DofScene **out) {
    if (!ctx || !out || (n_tris && (!xyz || !tri_idx || !n_verts)))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_scene_upload: null argument");
    if (n_tris > (1u << 30)) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_scene_upload: too many triangles");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    DofScene *s = new DofScene();
    memset(s, 0, sizeof(*s));
    s->ctx = ctx;
    s->n_tris = n_tris;
    s->n_nodes = n_tris >= 2 ? n_tris - 1 : 0;
    int rc = DOF_OK;
    float *d_xyz = nullptr;
    uint32_t *d_idx = nullptr, *d_mat = nullptr;
    if (n_tris == 0) { s->depth = 0; s->root = ~0; ctx_retain(ctx); *out = s; return DOF_OK; }
    s->tris_bytes = sizeof(float4) * 3 * (size_t)n_tris;
    s->nodes_bytes = sizeof(BvhNode) * (size_t)s->n_nodes;
    rc = dof_alloc(ctx, s->tris_bytes, (void **)&s->tris, &s->bytes);
    if (rc == DOF_OK) rc = dof_alloc(ctx, 4 * (size_t)n_tris, (void **)&s->prim_k, &s->bytes);
    if (rc == DOF_OK && s->n_nodes) rc = dof_alloc(ctx, s->nodes_bytes, (void **)&s->nodes, &s->bytes);
    if (rc == DOF_OK) rc = dof_cuda_check(cudaMalloc(&d_xyz, sizeof(float) * 3 * (size_t)n_verts), "scene vertices");
    if (rc == DOF_OK) rc = dof_cuda_check(cudaMalloc(&d_idx, sizeof(uint32_t) * 3 * (size_t)n_tris), "scene indices");
    if (rc == DOF_OK && tri_mat) rc = dof_cuda_check(cudaMalloc(&d_mat, sizeof(uint32_t) * (size_t)n_tris), "scene materials");
    if (rc == DOF_OK) rc = dof_cuda_check(cudaMemcpyAsync(d_xyz, xyz, sizeof(float) * 3 * (size_t)n_verts, cudaMemcpyHostToDevice, st), "upload");
    if (rc == DOF_OK) rc = dof_cuda_check(cudaMemcpyAsync(d_idx, tri_idx, sizeof(uint32_t) * 3 * (size_t)n_tris, cudaMemcpyHostToDevice, st), "upload");
    if (rc == DOF_OK && tri_mat) rc = dof_cuda_check(cudaMemcpyAsync(d_mat, tri_mat, sizeof(uint32_t) * (size_t)n_tris, cudaMemcpyHostToDevice, st), "upload");
    if (rc == DOF_OK) rc = launch_bvh_build(s, d_xyz, n_verts, d_idx, d_mat, ctx->bvh_builder, ctx->ploc_radius, ctx->bvh_rotations, st);
    if (rc == DOF_OK) {
        launch_prim_index(s->tris, (int)n_tris, s->prim_k, st);
        rc = dof_cuda_check(cudaStreamSynchronize(st), "scene triangle index");
    }
    cudaFree(d_xyz); cudaFree(d_idx); cudaFree(d_mat);
    if (rc != DOF_OK) {
        dof_free(ctx, s->tris, s->tris_bytes);
        dof_free(ctx, s->prim_k, 4 * (size_t)n_tris);
        dof_free(ctx, s->nodes, s->nodes_bytes);
        dof_free(ctx, s->nodes4, s->nodes4_bytes);
        delete s;
        return rc;
    }
    ctx_retain(ctx);
    *out = s;
    return DOF_OK;
}

extern "C" void dof_scene_destroy(DofScene *s) {
    if (!s) return;
    DofCtx *ctx = s->ctx;
    {
        DeviceGuard g(ctx->device);
        dof_free(ctx, s->tris, s->tris_bytes);
        dof_free(ctx, s->prim_k, 4 * (size_t)s->n_tris);
        dof_free(ctx, s->nodes, s->nodes_bytes);
        dof_free(ctx, s->nodes4, s->nodes4_bytes);
    }
    delete s;
    ctx_release(ctx);
}

extern "C" int dof_scene_info(const DofScene *s, DofSceneInfo *info) {
    if (!s || !info) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_scene_info: null argument");
    info->n_tris = s->n_tris;
    info->n_nodes = s->n_nodes;
    info->n_large = s->n_large;
    info->n_nodes4 = (uint32_t)s->n_nodes4;
    info->depth4 = (uint32_t)s->depth4;
    info->depth = s->depth;
    info->stack_limit = kTraversalStack;
    info->device_bytes = s->bytes;
    for (int k = 0; k < 3; k++) { info->bounds_lo[k] = s->lo[k]; info->bounds_hi[k] = s->hi[k]; }
    return DOF_OK;
}

static SceneDev scene_dev(const DofScene *s) {
    SceneDev d;
    d.nodes = s->nodes;
    d.tris = s->tris;
    d.n_tris = (int)s->n_tree;
    d.n_large = (int)s->n_large;
    d.root = s->root;
    // the 4-wide tree, when its traversal stack bound (3 per level) fits; warp packets
    // traverse the binary tree
    bool wide = s->nodes4 && s->ctx->bvh_width == 4 && !s->ctx->trace_packets && 3 * s->depth4 + 3 <= kTraversalStack;
    d.nodes4 = wide ? s->nodes4 : nullptr;
    d.root4 = s->root4;
    d.n_nodes4 = s->n_nodes4;
    // a binary node pushes at most one child per level, a 4-wide node three
    d.stack_need = wide ? 3 * s->depth4 + 3 : (int)s->depth;
    return d;
}

// ---------------------------------------------------------------------------
// G-buffer producer
// ---------------------------------------------------------------------------

extern "C" int dof_gbuffer(DofCtx *ctx, const DofScene *scene, const DofCamera *cam, const DofParams *p,
                           uint32_t width, uint32_t height, float *color, float *depth, float *normal, int32_t *prim,
                           void *stream) {
    if (!ctx || !scene || !cam || !p || !color || !depth || !normal)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_gbuffer: null argument");
    if (width < 2 || height < 2 || (width & 1) || (height & 1))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_gbuffer: size must be even and >= 2");
    if (!aligned(color, 16) || !aligned(normal, 16) || !aligned(depth, 8))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_gbuffer: misaligned output");
    DeviceGuard g(ctx->device);
    DevCam dc;
    DevParams dp;
    int rc = make_cam(cam, width, height, dc);
    if (rc) return rc;
    rc = make_params(p, width, height, DOF_MAX_RAYS, dp);
    if (rc) return rc;
    cudaGetLastError();   // drop a stale error of an earlier call of another library on this thread
    launch_primary(dc, dp, scene_dev(scene), reinterpret_cast<float4 *>(color), depth,
                   reinterpret_cast<float4 *>(normal), prim, ctx->d_status, (cudaStream_t)stream);
    return dof_cuda_check(cudaGetLastError(), "dof_gbuffer launch");
}

extern "C" int dof_gbuffer_raster(DofCtx *ctx, const DofScene *scene, const DofCamera *cam, const DofParams *p,
                                  uint32_t width, uint32_t height, float *color, float *depth, float *normal,
                                  int32_t *prim, void *stream) {
    if (!ctx || !scene || !cam || !p || !color || !depth || !normal)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_gbuffer_raster: null argument");
    if (width < 2 || height < 2 || (width & 1) || (height & 1))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_gbuffer_raster: size must be even and >= 2");
    if (!aligned(color, 16) || !aligned(normal, 16) || !aligned(depth, 8))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_gbuffer_raster: misaligned output");
    if (!ctx->pool) return dof_set_error(DOF_ERR_CUDA, "dof_gbuffer_raster: no memory pool on this device");
    DeviceGuard g(ctx->device);
    DevCam dc;
    DevParams dp;
    int rc = make_cam(cam, width, height, dc);
    if (rc) return rc;
    rc = make_params(p, width, height, DOF_MAX_RAYS, dp);
    if (rc) return rc;
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    const SceneDev sd = scene_dev(scene);
    const size_t bytes = raster_scratch_bytes((int)width, (int)height, (int)scene->n_tris);
    void *scratch = nullptr;
    rc = dof_cuda_check(cudaMallocFromPoolAsync(&scratch, bytes, ctx->pool, st), "dof_gbuffer_raster scratch");
    if (rc) return rc;
    cudaError_t e = launch_raster(dc, dp, sd, scene->prim_k, scratch, ctx->sm_count, reinterpret_cast<float4 *>(color),
                                  depth, reinterpret_cast<float4 *>(normal), prim, st);
    cudaError_t f = cudaFreeAsync(scratch, st);
    rc = dof_cuda_check(e, "dof_gbuffer_raster launch");
    if (rc) return rc;
    return dof_cuda_check(f, "dof_gbuffer_raster scratch release");
}

// ---------------------------------------------------------------------------
// history
// ---------------------------------------------------------------------------

static void history_free(DofHistory *h) {
    DofCtx *c = h->ctx;
    size_t N = h->N, T = (size_t)h->TW * h->TH;
    dof_free(c, h->pp_in, 16 * N); dof_free(c, h->pre, 16 * N); dof_free(c, h->main_, 16 * N);
    dof_free(c, h->pp_med, 16 * N); dof_free(c, h->n_h, 16 * N);
    dof_free(c, h->z_h, 4 * N); dof_free(c, h->xn, 4 * N); dof_free(c, h->xf, 4 * N);
    dof_free(c, h->tiles, 8 * T); dof_free(c, h->tiles_dil, 8 * T);
    dof_free(c, h->nrays, 4 * N); dof_free(c, h->queue, 4 * N); dof_free(c, h->counters, 32);
    dof_free(c, h->first_ray, 4 * N); dof_free(c, h->ray_pix, 4 * N * h->max_rays);
    dof_free(c, h->hits, 8 * N * h->max_rays);
    dof_free(c, h->ray_a, 16 * N * h->max_rays); dof_free(c, h->ray_b, 8 * N * h->max_rays);
    dof_free(c, h->ray_prim, 4 * N * h->max_rays);
    dof_free(c, h->rt, 64 * N); dof_free(c, h->crt, 16 * N); dof_free(c, h->rt_med, 16 * N);
    dof_free(c, h->recon, 16 * N); dof_free(c, h->ct, 4 * N); dof_free(c, h->var, 4 * N);
    for (int l = 0; l < 4; l++) {
        size_t n = (size_t)h->mip_w[l] * h->mip_h[l];
        dof_free(c, h->mip[l], 32 * n);
    }
    for (int k = 0; k < 2; k++) {
        dof_free(c, h->hist[k], 48 * N);
        dof_free(c, h->var_blur[k], 4 * N);
    }
    size_t P = (size_t)h->W * h->H;
    dof_free(c, h->comp, 16 * P);
    dof_free(c, h->taa[0], 16 * P);
    dof_free(c, h->taa[1], 16 * P);
    if (h->ev) {
        for (int k = 0; k < kTimingSlots * (DOF_K_COUNT + 1); k++)
            if (h->ev[k]) cudaEventDestroy(h->ev[k]);
        delete[] h->ev;
        h->ev = nullptr;
    }
    if (h->hio_h2d) cudaStreamSynchronize(h->hio_h2d);
    if (h->hio_d2h) cudaStreamSynchronize(h->hio_d2h);
    for (int k = 0; k < 2; k++) {
        dof_free(c, h->hio_color[k], 16 * P);
        dof_free(c, h->hio_depth[k], 4 * P);
        dof_free(c, h->hio_normal[k], 16 * P);
        dof_free(c, h->hio_out[k], 16 * P);
        if (h->hio_in[k]) cudaEventDestroy(h->hio_in[k]);
        if (h->hio_used[k]) cudaEventDestroy(h->hio_used[k]);
        if (h->hio_done[k]) cudaEventDestroy(h->hio_done[k]);
    }
    if (h->hio_h2d) cudaStreamDestroy(h->hio_h2d);
    if (h->hio_d2h) cudaStreamDestroy(h->hio_d2h);
}

extern "C" int dof_history_create(DofCtx *ctx, uint32_t width, uint32_t height, uint32_t max_rays, uint32_t flags,
                                  DofHistory **out) {
    if (!ctx || !out) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_create: null argument");
    *out = nullptr;
    if (width < 2 || height < 2 || (width & 1) || (height & 1) || width > 16384 || height > 16384)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_create: size must be even, 2..16384");
    if (max_rays < 1 || max_rays > DOF_MAX_RAYS)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_create: max_rays must be 1..%d", DOF_MAX_RAYS);
    DeviceGuard g(ctx->device);
    DofHistory *h = new DofHistory();
    memset(h, 0, sizeof(*h));
    h->ctx = ctx;
    h->W = width; h->H = height; h->W2 = width / 2; h->H2 = height / 2;
    h->N = h->W2 * h->H2;
    h->TW = (h->W2 + 7) / 8; h->TH = (h->H2 + 7) / 8;
    h->max_rays = max_rays;
    h->flags = flags;
    size_t N = h->N, T = (size_t)h->TW * h->TH;
    h->mip_w[0] = (int)h->W2; h->mip_h[0] = (int)h->H2;
    for (int l = 1; l < 4; l++) { h->mip_w[l] = (h->mip_w[l - 1] + 1) / 2; h->mip_h[l] = (h->mip_h[l - 1] + 1) / 2; }
    int rc = DOF_OK;
    auto A = [&](void **p, size_t b) { if (rc == DOF_OK) rc = dof_alloc(ctx, b, p, &h->bytes); };
    A((void **)&h->pp_in, 16 * N); A((void **)&h->pre, 16 * N); A((void **)&h->main_, 16 * N);
    A((void **)&h->pp_med, 16 * N); A((void **)&h->n_h, 16 * N);
    A((void **)&h->z_h, 4 * N); A((void **)&h->xn, 4 * N); A((void **)&h->xf, 4 * N);
    A((void **)&h->tiles, 8 * T); A((void **)&h->tiles_dil, 8 * T);
    A((void **)&h->nrays, 4 * N); A((void **)&h->queue, 4 * N); A((void **)&h->counters, 32);
    A((void **)&h->first_ray, 4 * N); A((void **)&h->ray_pix, 4 * N * max_rays);
    A((void **)&h->hits, 8 * N * max_rays);
    A((void **)&h->ray_a, 16 * N * max_rays); A((void **)&h->ray_b, 8 * N * max_rays);
    if (flags & DOF_HIST_RECORD_RAYS) A((void **)&h->ray_prim, 4 * N * max_rays);
    A((void **)&h->rt, 64 * N); A((void **)&h->crt, 16 * N); A((void **)&h->rt_med, 16 * N);
    A((void **)&h->recon, 16 * N); A((void **)&h->ct, 4 * N); A((void **)&h->var, 4 * N);
    for (int l = 0; l < 4; l++) {
        size_t n = (size_t)h->mip_w[l] * h->mip_h[l];
        A((void **)&h->mip[l], 32 * n);
    }
    for (int k = 0; k < 2; k++) {
        A((void **)&h->hist[k], 48 * N);
        A((void **)&h->var_blur[k], 4 * N);
    }
    if (flags & DOF_HIST_TAA) {
        size_t P = (size_t)h->W * h->H;
        A((void **)&h->comp, 16 * P);
        A((void **)&h->taa[0], 16 * P);
        A((void **)&h->taa[1], 16 * P);
    }
    if (rc == DOF_OK) {
        // history starts empty; the remaining buffers are defined before use each frame
        for (int k = 0; k < 2 && rc == DOF_OK; k++) {
            rc = dof_cuda_check(cudaMemset(h->hist[k], 0, 48 * N), "history clear");
            if (rc == DOF_OK) rc = dof_cuda_check(cudaMemset(h->var_blur[k], 0, 4 * N), "history clear");
        }
        if (rc == DOF_OK) rc = dof_cuda_check(cudaMemset(h->xf, 0, 4 * N), "history clear");
        if (rc == DOF_OK) rc = dof_cuda_check(cudaMemset(h->counters, 0, 32), "history clear");
        if (rc == DOF_OK && h->ray_prim) rc = dof_cuda_check(cudaMemset(h->ray_prim, 0xFF, 4 * N * max_rays), "clear");
    }
    if (rc == DOF_OK && (flags & DOF_HIST_TIMING)) {
        int n = kTimingSlots * (DOF_K_COUNT + 1);
        h->ev = new cudaEvent_t[n]();
        for (int k = 0; k < n && rc == DOF_OK; k++) rc = dof_cuda_check(cudaEventCreate(&h->ev[k]), "timing events");
    }
    if (rc != DOF_OK) {
        history_free(h);
        delete h;
        return rc;
    }
    ctx_retain(ctx);
    *out = h;
    return DOF_OK;
}

extern "C" void dof_history_destroy(DofHistory *h) {
    if (!h) return;
    DofCtx *ctx = h->ctx;
    {
        DeviceGuard g(ctx->device);
        history_free(h);
    }
    delete h;
    ctx_release(ctx);
}

extern "C" int dof_history_reset(DofHistory *h) {
    if (!h) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_reset: null history");
    h->valid = 0;
    h->taa_valid = 0;
    return DOF_OK;
}

// ---------------------------------------------------------------------------
// frame
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// frames: one launch per pass over the sessions of a batch
// ---------------------------------------------------------------------------

static int make_desc(DofCtx *ctx, const DofFrameReq &r, SessDesc &d) {
    const DofScene *scene = r.scene;
    const DofGBuffer *gb = r.gbuf;
    DofHistory *h = r.hist;
    if (!scene || !gb || !r.cam || !r.params || !h || !r.out)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_frame: null argument");
    if (h->ctx != ctx || scene->ctx != ctx) return dof_set_error(DOF_ERR_MISMATCH, "dof_frame: objects of another context");
    if (gb->width != h->W || gb->height != h->H)
        return dof_set_error(DOF_ERR_MISMATCH, "dof_frame: G-buffer %ux%u, history %ux%u", gb->width, gb->height, h->W, h->H);
    if (gb->fmt != DOF_FMT_F32 && gb->fmt != DOF_FMT_F16)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_frame: unsupported G-buffer format %u", gb->fmt);
    if (!gb->color || !gb->depth || (r.params->ray_mode == 1 && !gb->normal))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_frame: G-buffer plane is NULL");
    const size_t ga = gb->fmt == DOF_FMT_F16 ? 8 : 16;
    if (!aligned(gb->color, ga) || !aligned(gb->depth, 8) || (gb->normal && !aligned(gb->normal, ga)) || !aligned(r.out, 16))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_frame: misaligned buffer");
    memset(&d, 0, sizeof(d));
    int rc = make_cam(r.cam, h->W, h->H, d.cam);
    if (rc) return rc;
    rc = make_params(r.params, h->W, h->H, h->max_rays, d.p);
    if (rc) return rc;
    d.sc = scene_dev(scene);
    d.N = (int)h->N;
    d.max_rays = (int)h->max_rays;
    d.valid = h->valid;
    d.record_rays = (h->flags & DOF_HIST_RECORD_RAYS) && h->ray_prim;
    d.color = reinterpret_cast<const float4 *>(gb->color);
    d.depth = gb->depth;
    d.normal = reinterpret_cast<const float4 *>(gb->normal);
    d.gf16 = gb->fmt == DOF_FMT_F16;
    d.out = reinterpret_cast<float4 *>(r.out);
    d.pp_in = h->pp_in; d.pre = h->pre; d.main_ = h->main_; d.pp_med = h->pp_med; d.n_h = h->n_h;
    d.zn = h->crt;   // adaptive-mode scratch: crt is only written later, by the accumulation
    d.crt = h->crt; d.rt_med = h->rt_med; d.recon = h->recon; d.rt = h->rt;
    d.z_h = h->z_h; d.xn = h->xn; d.xf = h->xf; d.ct = h->ct; d.var = h->var;
    d.tiles = h->tiles; d.tiles_dil = h->tiles_dil;
    d.nrays = h->nrays; d.ray_prim = h->ray_prim;
    d.queue = h->queue; d.first_ray = h->first_ray; d.ray_pix = h->ray_pix; d.counters = h->counters;
    d.hits = h->hits; d.ray_a = h->ray_a; d.ray_b = h->ray_b;
    int L = (int)ceilf(r.params->lod_max) + 1;
    d.mip_L = L < 1 ? 1 : (L > 4 ? 4 : L);
    for (int l = 0; l < 4; l++) {
        d.mip[l] = h->mip[l]; d.mip_w[l] = h->mip_w[l]; d.mip_h[l] = h->mip_h[l];
    }
    d.hist_in = h->hist[h->cur];
    d.hist_out = h->hist[h->cur ^ 1];
    d.var_in = h->var_blur[h->cur];
    d.var_out = h->var_blur[h->cur ^ 1];
    d.comp_out = d.out;
    if (d.p.taa_alpha > 0.f) {
        if (!h->comp) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_frame: taa_alpha > 0 needs a history with DOF_HIST_TAA");
        d.taa = 1;
        d.taa_valid = h->taa_valid;
        d.comp_out = h->comp;
        d.taa_in = h->taa[h->taa_cur];
        d.taa_out = h->taa[h->taa_cur ^ 1];
    }
    return DOF_OK;
}

static void shape_grid(const BatchArgs &A, const SessDesc &d, const DofHistory *h, int shape, int &gx, int &gy) {
    switch (shape) {
        case SH_GATHER: {
            // the column-strip form of the main filter: each thread takes four rows
            const int rows = A.main_form == 3 ? 4 * A.gather_h : A.gather_h;
            gx = ((int)h->W2 + A.gather_w - 1) / A.gather_w;
            gy = ((int)h->H2 + rows - 1) / rows;
            break;
        }
        case SH_RECON: gx = ((int)h->W2 + A.recon_w - 1) / A.recon_w; gy = ((int)h->H2 + A.recon_h - 1) / A.recon_h; break;
        case SH_HPX: gx = ((int)h->W2 + 31) / 32; gy = ((int)h->H2 + 7) / 8; break;
        case SH_FPX: gx = ((int)h->W + 31) / 32; gy = ((int)h->H + 7) / 8; break;
        default: gx = ((int)h->N + 127) / 128; gy = 1; break;   // SH_SHADE
    }
}

// The batch descriptor of one step of `reqs` (validated); *adaptive: a session uses Eq. 4.
static int build_batch(DofCtx *ctx, const DofFrameReq *reqs, uint32_t n, BatchArgs &A, bool &adaptive) {
    if (n > (uint32_t)kMaxBatch) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_batch_frame: %u > %d sessions", n, kMaxBatch);
    memset(&A, 0, sizeof(A));
    A.ns = (int)n;
    A.gather_w = ctx->gather_w;
    A.gather_h = ctx->gather_h;
    A.recon_w = ctx->recon_w;
    A.recon_h = ctx->recon_h;
    A.main_form = ctx->main_form;
    adaptive = false;
    for (uint32_t s = 0; s < n; s++) {
        for (uint32_t t = 0; t < s; t++)
            if (reqs[t].hist == reqs[s].hist)
                return dof_set_error(DOF_ERR_INVALID_ARG, "dof_batch_frame: history %u appears twice", s);
        int rc = make_desc(ctx, reqs[s], A.s[s]);
        if (rc) return rc;
        adaptive |= A.s[s].p.ray_mode == 1;
        for (int sh = 0; sh < SH_COUNT; sh++) {
            int gx, gy;
            shape_grid(A, A.s[s], reqs[s].hist, sh, gx, gy);
            A.s[s].gx[sh] = gx;
            long long next = (long long)A.start[sh][s] + (long long)gx * gy;
            if (next > 0x7FFFFFFFll) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_batch_frame: batch too large");
            A.start[sh][s + 1] = (int)next;
        }
    }
    A.cursor = &reqs[0].hist->counters[2];
    A.refill_idle = ctx->trace_refill_idle;
    A.steps_per_round = ctx->trace_steps;
    A.lens_grid = ctx->ray_order_grid;
    A.packets = ctx->trace_packets;
    A.stats = ctx->trace_stats;
    A.stack_depth = ctx->stack_depth;
    return DOF_OK;
}

// Every launch of one step.  `A` gives the launch shapes; the kernels receive `as`.
template <class AS>
static void enqueue_step(DofCtx *ctx, const BatchArgs &A, const AS &as, bool adaptive, cudaStream_t st, DofHistory *tm) {
    const int trace_blocks = ctx->sm_count * ctx->trace_blocks_per_sm;
    launch_tiles_b(A, as, st, tm);
    if (tm) {
        // per-kernel timing: every kernel in sequence on the caller's stream
        launch_pp_b(A, as, st, tm);
        launch_mask_b(A, as, adaptive, st, tm);
        launch_trace_b(A, as, trace_blocks, st, tm);
        launch_temporal_b(A, as, st, tm);
        launch_recon_b(A, as, st, tm);
        launch_composite_b(A, as, st, tm);
    } else {
        // the ray path (A6 - A11) on the high-priority stream, the post-process filters
        // (A3 - A5, which only the composite reads) beside it on the caller's stream: the
        // filters fill the SMs that the tracer's tail leaves idle
        std::lock_guard<std::mutex> lock(ctx->launch_mu);
        cudaStream_t rs = ctx->ray_stream;
        cudaEventRecord(ctx->ev_fork, st);
        cudaStreamWaitEvent(rs, ctx->ev_fork, 0);
        launch_mask_b(A, as, adaptive, rs, nullptr);
        launch_trace_b(A, as, trace_blocks, rs, nullptr);
        launch_temporal_b(A, as, rs, nullptr);
        launch_recon_b(A, as, rs, nullptr);
        cudaEventRecord(ctx->ev_join, rs);
        launch_pp_b(A, as, st, nullptr);
        cudaStreamWaitEvent(st, ctx->ev_join, 0);
        launch_composite_b(A, as, st, nullptr);
    }
}

// host side of a step that was enqueued: the histories' ping-pong advances
static void finish_step(const DofFrameReq *reqs, uint32_t n) {
    for (uint32_t s = 0; s < n; s++) {
        DofHistory *h = reqs[s].hist;
        h->cur ^= 1;
        h->valid = 1;
        h->frames++;
        if (reqs[s].params->taa_alpha > 0.f) {
            h->taa_cur ^= 1;
            h->taa_valid = 1;
        }
    }
}

static int run_frames(DofCtx *ctx, const DofFrameReq *reqs, uint32_t n, cudaStream_t st) {
    if (n == 0) return DOF_OK;
    static thread_local BatchArgs A;   // ~22 KB: kept off the stack
    bool adaptive = false;
    int rc = build_batch(ctx, reqs, n, A, adaptive);
    if (rc) return rc;
    DofHistory *tm = reqs[0].hist;
    cudaGetLastError();   // drop a stale error of an earlier call of another library on this thread
    if (tm->ev && tm->ev_used < kTimingSlots) {
        // the frame's start; every kernel slot is marked in launch order after it (a kernel
        // that is not launched this frame is marked right after its predecessor)
        cudaEventRecord(tm->ev[tm->ev_slot * (DOF_K_COUNT + 1)], st);
    } else {
        tm = nullptr;
    }
    enqueue_step(ctx, A, A, adaptive, st, tm);
    rc = dof_cuda_check(cudaGetLastError(), "dof_frame launch");
    if (rc) return rc;
    finish_step(reqs, n);
    if (tm) {
        tm->ev_slot = (tm->ev_slot + 1) % kTimingSlots;
        tm->ev_used++;
    }
    return DOF_OK;
}

// ---------------------------------------------------------------------------
// captured steps (CUDA graphs)
// ---------------------------------------------------------------------------

struct DofGraph {
    DofCtx *ctx;
    uint32_t n;
    DofHistory *hist[kMaxBatch];
    int start[SH_COUNT][kMaxBatch + 1];
    bool adaptive, wide;
    int trace_blocks, refill_idle, steps_per_round, lens_grid, stack_depth, packets, stats;
    int gather_w, gather_h, main_form, recon_w, recon_h;
    int main_tile;                // the main filter's shared-memory bytes (0: through L1)
    int store_mode;               // image_storage_mode of the captured step
    bool taa;                     // the captured step has the final TAA pass
    long long kernels;            // kernel launches in one replay
    BatchArgs *d_args;            // read by the captured kernels
    BatchArgs *h_stage;           // pinned source of the captured copy
    cudaEvent_t staged;           // recorded after the copy: the staging buffer may be rewritten
    cudaEvent_t done;             // end of the last launch (orders launches on different streams)
    cudaStream_t last;
    bool launched;
    cudaGraphExec_t exec;
};

static bool all_wide(const BatchArgs &A) {
    bool w = A.ns > 0;
    for (int i = 0; i < A.ns; i++) w = w && A.s[i].sc.nodes4 != nullptr;
    return w;
}

static void graph_free(DofGraph *g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->staged) cudaEventDestroy(g->staged);
    if (g->done) cudaEventDestroy(g->done);
    if (g->h_stage) cudaFreeHost(g->h_stage);
    if (g->d_args) cudaFree(g->d_args);
}

extern "C" int dof_graph_create(DofCtx *ctx, const DofFrameReq *reqs, uint32_t n, DofGraph **out) {
    if (!ctx || !reqs || !out || n == 0) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_graph_create: null argument");
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    static thread_local BatchArgs A;
    bool adaptive = false;
    int rc = build_batch(ctx, reqs, n, A, adaptive);
    if (rc) return rc;
    DofGraph *g = new DofGraph();
    memset(g, 0, sizeof(*g));
    g->ctx = ctx;
    g->n = n;
    for (uint32_t s = 0; s < n; s++) g->hist[s] = reqs[s].hist;
    memcpy(g->start, A.start, sizeof(A.start));
    g->adaptive = adaptive;
    g->wide = all_wide(A);
    g->trace_blocks = ctx->sm_count * ctx->trace_blocks_per_sm;
    g->main_tile = main_filter_tile_bytes(A);
    g->store_mode = image_storage_mode(A);
    g->taa = any_taa(A);
    g->refill_idle = A.refill_idle;
    g->steps_per_round = A.steps_per_round;
    g->lens_grid = A.lens_grid;
    g->packets = A.packets;
    g->stats = A.stats;
    g->stack_depth = A.stack_depth;
    g->gather_w = A.gather_w;
    g->gather_h = A.gather_h;
    g->main_form = A.main_form;
    g->recon_w = A.recon_w;
    g->recon_h = A.recon_h;
    cudaGetLastError();
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    auto ck = [&](cudaError_t e, const char *w) { if (rc == DOF_OK && e != cudaSuccess) rc = dof_cuda_check(e, w); };
    ck(cudaMalloc(&g->d_args, sizeof(BatchArgs)), "dof_graph_create: device arguments");
    ck(cudaHostAlloc(&g->h_stage, sizeof(BatchArgs), cudaHostAllocDefault), "dof_graph_create: staging");
    ck(cudaEventCreateWithFlags(&g->staged, cudaEventDisableTiming), "dof_graph_create: event");
    ck(cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming), "dof_graph_create: event");
    ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "dof_graph_create: stream");
    if (rc == DOF_OK) {
        const BatchArgs *dp = g->d_args;
        ck(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "dof_graph_create: begin capture");
        if (rc == DOF_OK) {
            cudaMemcpyAsync(g->d_args, g->h_stage, sizeof(BatchArgs), cudaMemcpyHostToDevice, cs);
            cudaEventRecordWithFlags(g->staged, cs, cudaEventRecordExternal);
            // captured kernels run at each replay, not now: they are counted per launch
            const long long before = g_launches.load();
            enqueue_step(ctx, A, dp, adaptive, cs, nullptr);
            g->kernels = g_launches.load() - before;
            g_launches -= g->kernels;
            cudaError_t e = cudaStreamEndCapture(cs, &graph);
            ck(e, "dof_graph_create: capture");
        }
    }
    if (rc == DOF_OK) ck(cudaGraphInstantiate(&g->exec, graph, 0), "dof_graph_create: instantiate");
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    if (rc != DOF_OK) {
        graph_free(g);
        delete g;
        return rc;
    }
    ctx_retain(ctx);
    *out = g;
    return DOF_OK;
}

extern "C" int dof_graph_launch(DofGraph *g, const DofFrameReq *reqs, uint32_t n, void *stream) {
    if (!g || !reqs) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_graph_launch: null argument");
    if (n != g->n) return dof_set_error(DOF_ERR_MISMATCH, "dof_graph_launch: %u sessions, captured %u", n, g->n);
    for (uint32_t s = 0; s < n; s++)
        if (reqs[s].hist != g->hist[s])
            return dof_set_error(DOF_ERR_MISMATCH, "dof_graph_launch: session %u is not the captured history", s);
    DofCtx *ctx = g->ctx;
    DeviceGuard dg(ctx->device);
    static thread_local BatchArgs A;
    bool adaptive = false;
    int rc = build_batch(ctx, reqs, n, A, adaptive);
    if (rc) return rc;
    if (memcmp(A.start, g->start, sizeof(A.start)) != 0 || adaptive != g->adaptive || all_wide(A) != g->wide ||
        ctx->sm_count * ctx->trace_blocks_per_sm != g->trace_blocks || main_filter_tile_bytes(A) != g->main_tile ||
        A.gather_w != g->gather_w || A.gather_h != g->gather_h || A.main_form != g->main_form ||
        A.recon_w != g->recon_w || A.recon_h != g->recon_h || A.packets != g->packets || A.stats != g->stats ||
        image_storage_mode(A) != g->store_mode || any_taa(A) != g->taa)
        return dof_set_error(DOF_ERR_MISMATCH, "dof_graph_launch: launch shapes differ from the captured step");
    // the kernels' scheduling knobs come from the staged copy; keep the captured ones
    A.refill_idle = g->refill_idle;
    A.steps_per_round = g->steps_per_round;
    A.lens_grid = g->lens_grid;
    A.stack_depth = g->stack_depth;
    cudaStream_t st = (cudaStream_t)stream;
    cudaGetLastError();
    // the previous launch's copy has consumed the staging buffer
    rc = dof_cuda_check(cudaEventSynchronize(g->staged), "dof_graph_launch: staging");
    if (rc) return rc;
    memcpy(g->h_stage, &A, sizeof(BatchArgs));
    if (g->launched && st != g->last) cudaStreamWaitEvent(st, g->done, 0);
    rc = dof_cuda_check(cudaGraphLaunch(g->exec, st), "dof_graph_launch");
    if (rc) return rc;
    count_launches(g->kernels);
    cudaEventRecord(g->done, st);
    g->last = st;
    g->launched = true;
    finish_step(reqs, n);
    return DOF_OK;
}

extern "C" void dof_graph_destroy(DofGraph *g) {
    if (!g) return;
    DofCtx *ctx = g->ctx;
    {
        DeviceGuard dg(ctx->device);
        if (g->launched) cudaEventSynchronize(g->done);
        graph_free(g);
    }
    delete g;
    ctx_release(ctx);
}

extern "C" int dof_frame(DofCtx *ctx, const DofScene *scene, const DofGBuffer *gb, const DofCamera *cam,
                         const DofParams *p, DofHistory *h, float *out, void *stream) {
    if (!ctx || !scene || !gb || !cam || !p || !h || !out)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_frame: null argument");
    DofFrameReq r{scene, gb, cam, p, h, out};
    DeviceGuard g(ctx->device);
    return run_frames(ctx, &r, 1, (cudaStream_t)stream);
}

// the slots of dof_frame_host, made on first use (the normal planes when first needed)
static int host_io_init(DofHistory *h, bool normals) {
    DofCtx *c = h->ctx;
    const size_t P = (size_t)h->W * h->H;
    int rc = DOF_OK;
    if (!h->hio_ready) {
        for (int k = 0; k < 2 && rc == DOF_OK; k++) {
            rc = dof_alloc(c, 16 * P, (void **)&h->hio_color[k], &h->bytes);
            if (rc == DOF_OK) rc = dof_alloc(c, 4 * P, (void **)&h->hio_depth[k], &h->bytes);
            if (rc == DOF_OK) rc = dof_alloc(c, 16 * P, (void **)&h->hio_out[k], &h->bytes);
            if (rc == DOF_OK &&
                (cudaEventCreateWithFlags(&h->hio_in[k], cudaEventDisableTiming) != cudaSuccess ||
                 cudaEventCreateWithFlags(&h->hio_used[k], cudaEventDisableTiming) != cudaSuccess ||
                 cudaEventCreateWithFlags(&h->hio_done[k], cudaEventDisableTiming) != cudaSuccess))
                rc = dof_set_error(DOF_ERR_CUDA, "dof_frame_host: events");
        }
        if (rc == DOF_OK && (cudaStreamCreateWithFlags(&h->hio_h2d, cudaStreamNonBlocking) != cudaSuccess ||
                             cudaStreamCreateWithFlags(&h->hio_d2h, cudaStreamNonBlocking) != cudaSuccess))
            rc = dof_set_error(DOF_ERR_CUDA, "dof_frame_host: copy streams");
        if (rc != DOF_OK) {
            cudaGetLastError();
            return rc;      // what was made is released with the history
        }
        h->hio_ready = 1;
    }
    if (normals && !h->hio_normals) {
        for (int k = 0; k < 2 && rc == DOF_OK; k++)
            rc = dof_alloc(c, 16 * P, (void **)&h->hio_normal[k], &h->bytes);
        if (rc != DOF_OK) return rc;
        h->hio_normals = 1;
    }
    return DOF_OK;
}

extern "C" int dof_frame_host(DofCtx *ctx, const DofScene *scene, const float *color, const float *depth,
                              const float *normal, const DofCamera *cam, const DofParams *p, DofHistory *h,
                              float *out, void *stream) {
    if (!ctx || !scene || !color || !depth || !cam || !p || !h || !out)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_frame_host: null argument");
    if (h->ctx != ctx) return dof_set_error(DOF_ERR_MISMATCH, "dof_frame_host: history of another context");
    DeviceGuard g(ctx->device);
    int rc = host_io_init(h, normal != nullptr);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int k = (int)(h->hio_frames & 1);
    const size_t P = (size_t)h->W * h->H;
    DofGBuffer gb{};
    gb.color = reinterpret_cast<const float *>(h->hio_color[k]);
    gb.depth = h->hio_depth[k];
    gb.normal = normal ? reinterpret_cast<const float *>(h->hio_normal[k]) : nullptr;
    gb.width = h->W;
    gb.height = h->H;
    gb.fmt = DOF_FMT_F32;
    cudaGetLastError();
    // inputs: once the frame two calls back is done with this slot
    cudaError_t e = cudaStreamWaitEvent(h->hio_h2d, h->hio_used[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hio_color[k], color, 16 * P, cudaMemcpyHostToDevice, h->hio_h2d);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->hio_depth[k], depth, 4 * P, cudaMemcpyHostToDevice, h->hio_h2d);
    if (e == cudaSuccess && normal)
        e = cudaMemcpyAsync(h->hio_normal[k], normal, 16 * P, cudaMemcpyHostToDevice, h->hio_h2d);
    if (e == cudaSuccess) e = cudaEventRecord(h->hio_in[k], h->hio_h2d);
    // the frame: after its inputs, and once the image of two calls back has been copied out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->hio_in[k], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->hio_done[k], 0);
    rc = dof_cuda_check(e, "dof_frame_host input copy");
    if (rc) return rc;
    DofFrameReq r{scene, &gb, cam, p, h, reinterpret_cast<float *>(h->hio_out[k])};
    rc = run_frames(ctx, &r, 1, st);
    if (rc) return rc;
    // the image: copied out once the frame is done
    e = cudaEventRecord(h->hio_used[k], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->hio_d2h, h->hio_used[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->hio_out[k], 16 * P, cudaMemcpyDeviceToHost, h->hio_d2h);
    if (e == cudaSuccess) e = cudaEventRecord(h->hio_done[k], h->hio_d2h);
    rc = dof_cuda_check(e, "dof_frame_host output copy");
    if (rc) return rc;
    h->hio_frames++;
    return DOF_OK;
}

extern "C" int dof_frame_host_join(DofHistory *h, void *stream) {
    if (!h) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_frame_host_join: null history");
    if (!h->hio_ready) return DOF_OK;
    DeviceGuard g(h->ctx->device);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaStreamWaitEvent((cudaStream_t)stream, h->hio_done[k], 0);
    return dof_cuda_check(e, "dof_frame_host_join");
}

extern "C" int dof_batch_frame(DofCtx *ctx, const DofFrameReq *reqs, uint32_t n, void *stream) {
    if (!ctx || (n && !reqs)) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_batch_frame: null argument");
    DeviceGuard g(ctx->device);
    return run_frames(ctx, reqs, n, (cudaStream_t)stream);
}

extern "C" int dof_kernel_times(DofHistory *h, void *stream, float *ms, uint32_t *frames) {
    if (!h || !ms || !frames) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_kernel_times: null argument");
    if (!h->ev) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_kernel_times: history has no DOF_HIST_TIMING");
    DeviceGuard g(h->ctx->device);
    int rc = dof_cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "dof_kernel_times sync");
    if (rc) return rc;
    for (int k = 0; k < DOF_K_COUNT; k++) ms[k] = 0.f;
    int first = (h->ev_slot - h->ev_used + kTimingSlots) % kTimingSlots;
    for (int f = 0; f < h->ev_used; f++) {
        int s = (first + f) % kTimingSlots;
        for (int k = 0; k < DOF_K_COUNT; k++) {
            float t = 0.f;
            rc = dof_cuda_check(cudaEventElapsedTime(&t, h->ev[s * (DOF_K_COUNT + 1) + k],
                                                     h->ev[s * (DOF_K_COUNT + 1) + k + 1]), "cudaEventElapsedTime");
            if (rc) return rc;
            ms[k] += t;
        }
    }
    *frames = (uint32_t)h->ev_used;
    h->ev_used = 0;
    return DOF_OK;
}

extern "C" int dof_frame_stats(DofHistory *h, void *stream, DofFrameStats *out) {
    if (!h || !out) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_frame_stats: null argument");
    DeviceGuard g(h->ctx->device);
    uint32_t c[8];
    int rc = dof_cuda_check(cudaMemcpyAsync(c, h->counters, sizeof(c), cudaMemcpyDeviceToHost, (cudaStream_t)stream),
                            "dof_frame_stats");
    if (rc == DOF_OK) rc = dof_cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "dof_frame_stats sync");
    if (rc) return rc;
    out->frames = h->frames;
    out->masked_pixels = c[0];
    out->rays = c[1];
    out->device_status = c[3] ? DOF_ERR_DEVICE_CHECK : DOF_OK;
    out->pad = 0;
    out->node_visits = (uint64_t)c[4] | ((uint64_t)c[5] << 32);
    out->tri_tests = (uint64_t)c[6] | ((uint64_t)c[7] << 32);
    return DOF_OK;
}

extern "C" int dof_debug_buffer(DofHistory *h, int which, void **ptr, size_t *bytes) {
    if (!h || !ptr || !bytes) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_debug_buffer: null argument");
    size_t N = h->N, T = (size_t)h->TW * h->TH;
    int last = h->cur;   // after a frame, `cur` holds the newest history
    switch (which) {
        case DOF_BUF_PP_IN: *ptr = h->pp_in; *bytes = 16 * N; break;
        case DOF_BUF_Z_H: *ptr = h->z_h; *bytes = 4 * N; break;
        case DOF_BUF_TILES: *ptr = h->tiles; *bytes = 8 * T; break;
        case DOF_BUF_TILES_DIL: *ptr = h->tiles_dil; *bytes = 8 * T; break;
        case DOF_BUF_PRE: *ptr = h->pre; *bytes = 16 * N; break;
        case DOF_BUF_MAIN: *ptr = h->main_; *bytes = 16 * N; break;
        case DOF_BUF_PP_MED: *ptr = h->pp_med; *bytes = 16 * N; break;
        case DOF_BUF_XN: *ptr = h->xn; *bytes = 4 * N; break;
        case DOF_BUF_XF: *ptr = h->xf; *bytes = 4 * N; break;
        case DOF_BUF_NRAYS: *ptr = h->nrays; *bytes = 4 * N; break;
        case DOF_BUF_RAY_PRIM: *ptr = h->ray_prim; *bytes = h->ray_prim ? 4 * N * h->max_rays : 0; break;
        case DOF_BUF_RT: *ptr = h->rt; *bytes = 64 * N; break;
        case DOF_BUF_CRT: *ptr = h->crt; *bytes = 16 * N; break;
        case DOF_BUF_CT: *ptr = h->ct; *bytes = 4 * N; break;
        case DOF_BUF_VAR: *ptr = h->var; *bytes = 4 * N; break;
        case DOF_BUF_VAR_BLUR: *ptr = h->var_blur[last]; *bytes = 4 * N; break;
        case DOF_BUF_RT_MED: *ptr = h->rt_med; *bytes = 16 * N; break;
        case DOF_BUF_RECON: *ptr = h->recon; *bytes = 16 * N; break;
        case DOF_BUF_HIST: *ptr = h->hist[last]; *bytes = 48 * N; break;
        case DOF_BUF_COMPOSITE: *ptr = h->comp; *bytes = h->comp ? 16 * (size_t)h->W * h->H : 0; break;
        default: return dof_set_error(DOF_ERR_INVALID_ARG, "dof_debug_buffer: unknown buffer %d", which);
    }
    return DOF_OK;
}

extern "C" int dof_debug_read(DofHistory *h, int which, void *dst, size_t bytes) {
    void *src = nullptr;
    size_t n = 0;
    int rc = dof_debug_buffer(h, which, &src, &n);
    if (rc) return rc;
    if (!dst && bytes) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_debug_read: null destination");
    if (bytes != n) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_debug_read: %zu bytes requested, buffer has %zu", bytes, n);
    if (!n) return DOF_OK;
    DeviceGuard g(h->ctx->device);
    rc = dof_cuda_check(cudaDeviceSynchronize(), "dof_debug_read sync");
    if (rc) return rc;
    return dof_cuda_check(cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost), "dof_debug_read");
}

// ---------------------------------------------------------------------------
// checkpoint
// ---------------------------------------------------------------------------

namespace {
struct HistHeader {
    uint32_t magic, version, width, height, max_rays, valid;
    uint64_t frames, n;
};
constexpr uint32_t kHistMagic = 0x48464F44u;   // "DOFH"
}

extern "C" int dof_history_export(DofHistory *h, void *buf, size_t *bytes, void *stream) {
    if (!h || !bytes) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_export: null argument");
    size_t N = h->N, need = sizeof(HistHeader) + 48 * N + 4 * N;
    if (!buf) { *bytes = need; return DOF_OK; }
    if (*bytes < need) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_export: buffer of %zu bytes, need %zu", *bytes, need);
    DeviceGuard g(h->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = dof_cuda_check(cudaStreamSynchronize(st), "dof_history_export sync");
    if (rc) return rc;
    HistHeader hd{kHistMagic, 1u, h->W, h->H, h->max_rays, (uint32_t)h->valid, h->frames, N};
    char *p = static_cast<char *>(buf);
    memcpy(p, &hd, sizeof(hd));
    rc = dof_cuda_check(cudaMemcpy(p + sizeof(hd), h->hist[h->cur], 48 * N, cudaMemcpyDeviceToHost), "export history");
    if (rc == DOF_OK)
        rc = dof_cuda_check(cudaMemcpy(p + sizeof(hd) + 48 * N, h->var_blur[h->cur], 4 * N, cudaMemcpyDeviceToHost),
                            "export variance");
    if (rc == DOF_OK) *bytes = need;
    return rc;
}

extern "C" int dof_history_import(DofHistory *h, const void *buf, size_t bytes, void *stream) {
    if (!h || !buf) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_import: null argument");
    size_t N = h->N, need = sizeof(HistHeader) + 48 * N + 4 * N;
    HistHeader hd;
    if (bytes < sizeof(hd)) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_import: truncated buffer");
    memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kHistMagic || hd.version != 1u)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_import: not a history checkpoint");
    if (hd.width != h->W || hd.height != h->H || hd.max_rays != h->max_rays || hd.n != N)
        return dof_set_error(DOF_ERR_MISMATCH, "dof_history_import: checkpoint of %ux%u (max_rays %u), history %ux%u (%u)",
                             hd.width, hd.height, hd.max_rays, h->W, h->H, h->max_rays);
    if (bytes < need) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_history_import: truncated buffer");
    DeviceGuard g(h->ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = dof_cuda_check(cudaStreamSynchronize(st), "dof_history_import sync");
    if (rc) return rc;
    const char *p = static_cast<const char *>(buf);
    rc = dof_cuda_check(cudaMemcpy(h->hist[h->cur], p + sizeof(hd), 48 * N, cudaMemcpyHostToDevice), "import history");
    if (rc == DOF_OK)
        rc = dof_cuda_check(cudaMemcpy(h->var_blur[h->cur], p + sizeof(hd) + 48 * N, 4 * N, cudaMemcpyHostToDevice),
                            "import variance");
    if (rc == DOF_OK) {
        h->valid = (int)hd.valid;
        h->taa_valid = 0;   // the TAA image history is not part of a checkpoint
        h->frames = hd.frames;
    }
    return rc;
}

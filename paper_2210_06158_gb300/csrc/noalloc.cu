// Allocation-free variant of the tile stage of the post-process (tile max-CoC and
// its neighbourhood dilation), for callers that must not allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc at the point where they want the
// tile map: an engine whose allocator has reserved all device memory up front and
// hands out nothing during a frame, or a frame loop in which cudaMalloc/cudaFree
// would implicitly synchronise the device and stall the frame.  This entry point
// keeps its only intermediate -- the per-tile maxima before dilation -- in a
// file-scope __device__ array instead of a buffer it would have to allocate.
//
// The array holds at most kMaxTiles tiles (512 KB).  Every GPU on which the library
// is loaded holds that array for the life of the process.  All calls share it and it
// keeps whatever the previous call left there; each call overwrites every tile it
// reads before reading it, so nothing has to start at zero.  Calls whose work
// overlaps on the GPU (different streams, or different host threads without
// ordering) race on the array and must be serialised by the caller.
#include <math.h>
#include <string.h>

#include "dof_internal.cuh"

namespace {

constexpr int kMaxTiles = DOF_NOALLOC_MAX_TILES;

// the scratch array: raw (undilated) tile maxima (near radius, |rho|)
__device__ __align__(256) float2 g_tile_scratch[kMaxTiles];

struct TileArgs {
    float cocK, d, rmax, z_far;
    int W, H, W2, H2, TW, TH, K;
};

// Tile max of one 8x8 block of half-resolution pixels from the full-resolution depth:
// depth of a half-resolution pixel = the nearest of its 2x2 block (clamped to z_far),
// rho = clamp(c(z)/4, +-rmax), c(z) = cocK (z - d) / z.
__global__ void __launch_bounds__(64) k_tiles_scratch(TileArgs a, const float *__restrict__ depth, float2 *raw) {
    int i = blockIdx.x * 8 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    float nm = 0.f, am = 0.f;
    if (i < a.W2 && j < a.H2) {
        size_t f0 = (size_t)(2 * j) * a.W + 2 * i, f1 = f0 + a.W;
        float2 d01 = __ldg(reinterpret_cast<const float2 *>(&depth[f0]));
        float2 d23 = __ldg(reinterpret_cast<const float2 *>(&depth[f1]));
        float z = fminf(fminf(fminf(d01.x, a.z_far), fminf(d01.y, a.z_far)),
                        fminf(fminf(d23.x, a.z_far), fminf(d23.y, a.z_far)));
        float rho = fminf(fmaxf(0.25f * (a.cocK * (z - a.d) / z), -a.rmax), a.rmax);
        nm = fmaxf(0.f, -rho);
        am = fabsf(rho);
    }
    for (int o = 16; o > 0; o >>= 1) {
        nm = fmaxf(nm, __shfl_xor_sync(0xffffffffu, nm, o));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
    }
    __shared__ float2 red[2];
    int t = threadIdx.y * 8 + threadIdx.x;
    if ((t & 31) == 0) red[t >> 5] = make_float2(nm, am);
    __syncthreads();
    if (t == 0) raw[blockIdx.y * a.TW + blockIdx.x] = make_float2(fmaxf(red[0].x, red[1].x), fmaxf(red[0].y, red[1].y));
}

// neighbourhood max over (2K+1)^2 tiles, from the scratch array into the caller's map
__global__ void k_dilate_scratch(TileArgs a, const float2 *raw, float2 *dil) {
    int tx = blockIdx.x * blockDim.x + threadIdx.x, ty = blockIdx.y * blockDim.y + threadIdx.y;
    if (tx >= a.TW || ty >= a.TH) return;
    float nm = 0.f, am = 0.f;
    for (int y = max(ty - a.K, 0); y <= min(ty + a.K, a.TH - 1); y++)
        for (int x = max(tx - a.K, 0); x <= min(tx + a.K, a.TW - 1); x++) {
            float2 v = raw[y * a.TW + x];
            nm = fmaxf(nm, v.x);
            am = fmaxf(am, v.y);
        }
    dil[ty * a.TW + tx] = make_float2(nm, am);
}

// Device address of g_tile_scratch in the current device's context.  It is looked up
// on every call, not cached: after cudaDeviceReset, or from another context on the same
// device, the library's device code is loaded afresh and the array moves, so an address
// kept from an earlier call could point at memory that is no longer this array.  The
// lookup enqueues no work; the first one in a context loads the library's device code
// there.
int scratch_for_current_device(float2 **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_tile_scratch);
    if (e != cudaSuccess || !p) return dof_cuda_check(e, "dof_coc_tiles_noalloc: cudaGetSymbolAddress");
    *out = static_cast<float2 *>(p);
    return DOF_OK;
}

}  // namespace

extern "C" int dof_coc_tiles_noalloc(const float *depth, uint32_t width, uint32_t height, const DofCamera *cam,
                                     const DofParams *p, float *tiles_dil, void *stream) {
    if (!depth || !cam || !p || !tiles_dil)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_coc_tiles_noalloc: null argument");
    if (width < 2 || height < 2 || (width & 1) || (height & 1) || width > 16384 || height > 16384)
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_coc_tiles_noalloc: size must be even, 2..16384");
    if (((uintptr_t)depth % 8) || ((uintptr_t)tiles_dil % 8))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_coc_tiles_noalloc: depth and tiles must be 8-byte aligned");
    if (p->tile != 8) return dof_set_error(DOF_ERR_INVALID_ARG, "dof_coc_tiles_noalloc: tile must be 8");
    if (!(p->max_coc_px >= 1.f && p->max_coc_px <= 256.f))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_coc_tiles_noalloc: max_coc_px must be in [1, 256]");
    if (!(p->z_far_m > 0.f) || !isfinite(p->z_far_m))
        return dof_set_error(DOF_ERR_INVALID_ARG, "dof_coc_tiles_noalloc: z_far must be finite and > 0");
    if (!(cam->f_m > 0.f) || !(cam->f_number > 0.f) || !(cam->sensor_w_m > 0.f) || !(cam->focus_m > cam->f_m) ||
        !isfinite(cam->f_m) || !isfinite(cam->f_number) || !isfinite(cam->focus_m) || !isfinite(cam->sensor_w_m))
        return dof_set_error(DOF_ERR_INVALID_ARG,
                             "dof_coc_tiles_noalloc: need finite f > 0, N > 0, w_s > 0 and focus > f");
    TileArgs a;
    a.W = (int)width; a.H = (int)height; a.W2 = a.W / 2; a.H2 = a.H / 2;
    a.TW = (a.W2 + 7) / 8; a.TH = (a.H2 + 7) / 8;
    if ((long long)a.TW * a.TH > kMaxTiles)
        return dof_set_error(DOF_ERR_INVALID_ARG,
                             "dof_coc_tiles_noalloc: %ux%u needs %d tiles, more than the %d of the built-in scratch",
                             width, height, a.TW * a.TH, kMaxTiles);
    double f = cam->f_m, N = cam->f_number, d = cam->focus_m, ws = cam->sensor_w_m;
    a.cocK = (float)((f / N) * f * (double)width / (ws * (d - f)));
    a.d = cam->focus_m;
    a.rmax = 0.5f * p->max_coc_px;
    a.z_far = p->z_far_m;
    a.K = (int)ceil(0.5 * (double)p->max_coc_px / 8.0);
    float2 *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    k_tiles_scratch<<<dim3(a.TW, a.TH), dim3(8, 8), 0, st>>>(a, depth, scratch);
    k_dilate_scratch<<<dim3((a.TW + 15) / 16, (a.TH + 15) / 16), dim3(16, 16), 0, st>>>(
        a, scratch, reinterpret_cast<float2 *>(tiles_dil));
    count_launches(2);
    return dof_cuda_check(cudaGetLastError(), "dof_coc_tiles_noalloc launch");
}

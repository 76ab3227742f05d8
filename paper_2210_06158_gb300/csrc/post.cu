// Post-process stage of libdof (Section 3.1): CoC + 2x2 downscale + tile max,
// tile dilation, 9-tap bilateral prefilter, 81-tap main gather filter (Eq. 1), and the
// 3x3 median postfilter (a 19-exchange min/max network, Section 3.1.3).
#include "batch.cuh"
#include "filters.cuh"

namespace {

// A1: one thread per half-resolution pixel, blocks of 32x8 pixels = four 8x8 max-CoC
// tiles.  Colour = mean of the 2x2 full-resolution block, depth = the nearest of the
// four (clamped to z_far), CoC radius rho = clamp(c(z)/4) and normal of that sample;
// tile max of near and |rho| (lanes of a tile row by shuffles, rows through shared
// memory).
template <class AS>
__global__ void __launch_bounds__(256) k_downscale_tiles(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_HPX, i, j);
    const DevCam &cam = S.cam;
    const DevParams &p = S.p;
    const float4 *__restrict__ color = S.color;
    const float *__restrict__ depth = S.depth;
    const float4 *__restrict__ normal = S.normal;
    // the first block of each session zeroes the session's per-frame counters (queue
    // length, rays, work cursor, traversal counts; not the sticky status word): nothing of
    // this frame reads them before the ray path, which starts after this kernel
    if (i == (int)threadIdx.x && j == (int)threadIdx.y && threadIdx.x == 0 && threadIdx.y == 0) {
        uint32_t *c = S.counters;
        c[0] = c[1] = c[2] = 0u;
        c[4] = c[5] = c[6] = c[7] = 0u;
    }
    float nm = 0.f, am = 0.f;
    if (i < cam.W2 && j < cam.H2) {
        size_t f0 = (size_t)(2 * j) * cam.W + 2 * i, f1 = f0 + cam.W;
        const bool gh = S.gf16;
        float4 c0 = ld_img(color, f0, gh), c1 = ld_img(color, f0 + 1, gh), c2 = ld_img(color, f1, gh),
               c3 = ld_img(color, f1 + 1, gh);
        float2 d01 = __ldg(reinterpret_cast<const float2 *>(&depth[f0]));
        float2 d23 = __ldg(reinterpret_cast<const float2 *>(&depth[f1]));
        float z[4] = {fminf(d01.x, p.z_far), fminf(d01.y, p.z_far), fminf(d23.x, p.z_far), fminf(d23.y, p.z_far)};
        int k = 0;
#pragma unroll
        for (int m = 1; m < 4; m++)
            if (z[m] < z[k]) k = m;
        float zm = z[k];
        float rho = fminf(fmaxf(0.25f * coc_of(cam, zm), -p.rmax_hpx), p.rmax_hpx);
        size_t q = (size_t)j * cam.W2 + i;
        S.pp_in[q] = make_float4(0.25f * (c0.x + c1.x + c2.x + c3.x), 0.25f * (c0.y + c1.y + c2.y + c3.y),
                               0.25f * (c0.z + c1.z + c2.z + c3.z), rho);
        S.z_h[q] = zm;
        if (p.ray_mode == 1) {
            size_t fk = (k < 2 ? f0 : f1) + (k & 1);
            S.n_h[q] = ld_img(normal, fk, gh);
        }
        nm = fmaxf(0.f, -rho);
        am = fabsf(rho);
    }
    // max over the 8 lanes of each tile in this row
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        nm = fmaxf(nm, __shfl_xor_sync(0xffffffffu, nm, o));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
    }
    __shared__ float2 red[8][4];
    const int lane = threadIdx.x, row = threadIdx.y;
    if ((lane & 7) == 0) red[row][lane >> 3] = make_float2(nm, am);
    __syncthreads();
    if (row == 0 && lane < 4) {
        float2 m = red[0][lane];
#pragma unroll
        for (int r = 1; r < 8; r++) m = make_float2(fmaxf(m.x, red[r][lane].x), fmaxf(m.y, red[r][lane].y));
        const int tx = (i - lane) / 8 + lane, ty = j / 8;
        if (tx < p.tiles_w && ty < p.tiles_h) S.tiles[ty * p.tiles_w + tx] = m;
    }
}

// A2 + A3: the dilated max-CoC of the block's four tiles (written out for the main
// filter), then the 9-tap bilateral prefilter, radius max(R/8, sqrt(2)/2), taps at
// angles k pi/4
template <class AS>
__global__ void __launch_bounds__(256) k_prefilter(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_HPX, i, j);
    const DevParams &p = S.p;
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const float4 *__restrict__ pp_in = S.pp_in;
    float4 *pre = S.pre;
    __shared__ float2 dil_s[4];
    const int bx = i - (int)threadIdx.x, by = j - (int)threadIdx.y;
    dilate_block_tiles(S, bx, by, dil_s);
    __syncthreads();
    if (threadIdx.y == 0 && threadIdx.x < 4) {
        const int tx = bx / 8 + (int)threadIdx.x, ty = by / 8;
        if (tx < p.tiles_w && ty < p.tiles_h) S.tiles_dil[ty * p.tiles_w + tx] = dil_s[threadIdx.x];
    }
    if (i >= W2 || j >= H2) return;
    size_t q = (size_t)j * W2 + i;
    float R = dil_s[threadIdx.x >> 3].y;
    float rp = fmaxf(R * 0.125f, 0.70710678118654752f);
    float4 c0 = __ldg(&pp_in[q]);
    float inv = 1.f / fmaxf(1.f, fabsf(c0.w));
    float ax = c0.x, ay = c0.y, az = c0.z, ws = 1.f;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        float2 u = c_pre8[k];
        float4 s = bilinear4(pp_in, W2, H2, i + rp * u.x, j + rp * u.y);
        float w = sat(1.f - fabsf(s.w - c0.w) * inv);
        ax += w * s.x; ay += w * s.y; az += w * s.z; ws += w;
    }
    float r = 1.f / ws;
    const float4 v = make_float4(ax * r, ay * r, az * r, c0.w);
    pre[q] = p.f16 ? pre_record(v, __ldg(&S.z_h[q])) : v;
}

// A4: 81-tap main filter (Eq. 1).  Rings k = 1..4 of 8k taps at radius kR/4 of the
// dilated max CoC R; foreground/background weights with the coverage ramp D and
// sampleAlpha; normalised weighted sum plus the share of bright samples.  Blocks whose
// whole footprint (+-rmax + 1) lies inside the image take taps without index clamping.
// Accumulators of one pixel of the main filter.
struct MainAcc {
    float ax, ay, az, bright, wsum;
};

// One tap of the main filter: its bilinear sample s (rgb, signed CoC) and depth zi at
// distance dist from the pixel (depth z0, |CoC| r0).  Every form of the filter adds its
// taps through this one function.  Each rounding is written out (explicit FMAs, or
// products and sums that the compiler may not contract), as are the tap positions and
// depth sums in the callers, so that all forms give the same bits whatever the
// surrounding code lets the compiler fuse.
__device__ __forceinline__ void main_tap_add(const DevParams &p, float dist, float z0, float r0, float4 s, float zi,
                                             MainAcc &m) {
    const float ri = fabsf(s.w);
    const float wf = sat(__fmul_rn(__fsub_rn(z0, zi), p.inv_depth_range));
    const float rr = fmaxf(ri, p.inv_sqrt_area);
    const float a = __fdividef(p.inv_area, __fmul_rn(rr, rr));
    const float Df = sat(fmaf(__fsub_rn(ri, dist), p.inv_cover_ramp, 0.5f));
    const float Db = sat(fmaf(__fsub_rn(fminf(ri, r0), dist), p.inv_cover_ramp, 0.5f));
    const float W = __fmul_rn(fmaf(wf, Df, __fmul_rn(__fsub_rn(1.f, wf), Db)), a);
    const float lum = fmaf(0.0722f, s.z, fmaf(0.7152f, s.y, __fmul_rn(0.2126f, s.x)));
    m.ax = fmaf(W, s.x, m.ax);
    m.ay = fmaf(W, s.y, m.ay);
    m.az = fmaf(W, s.z, m.az);
    m.bright = fmaf(W, sat(__fmul_rn(__fsub_rn(lum, p.bright_lum), p.inv_bright_ramp)), m.bright);
    m.wsum = __fadd_rn(m.wsum, W);
}

template <bool CLAMP, bool H>
__device__ __forceinline__ void main_taps(int i, int j, int W2, int H2, const DevParams &p, const float4 *__restrict__ pre,
                                          const float *__restrict__ z_h, float R, float z0, float r0, MainAcc &m) {
    const int ring = p.ring;
#pragma unroll 3
    for (int t = 0; t < 81; t++) {
        const float3 u = c_rings[ring][t];
        const float dist = __fmul_rn(u.z, R);
        const float x = fmaf(dist, u.x, (float)i), y = fmaf(dist, u.y, (float)j);
        float4 s;
        float zi;
        if (CLAMP) bilinear4z<H>(pre, z_h, W2, H2, x, y, s, zi);
        else bilinear4z_interior<H>(pre, z_h, W2, x, y, s, zi);
        main_tap_add(p, dist, z0, r0, s, zi, m);
    }
}

// the pixel's own depth and |CoC| from the prefilter's output (ld_pre)
__device__ __forceinline__ void pre_centre(const float4 *__restrict__ pre, const float *__restrict__ z_h, size_t q,
                                           bool f16, float &z0, float &r0) {
    const float4 t = __ldg(&pre[q]);
    z0 = f16 ? t.w : __ldg(&z_h[q]);
    r0 = fabsf(f16 ? t.z : t.w);
}

// kStore: the launch's image storage (image_storage_mode) in all three forms
template <class AS, int kStore>
__global__ void __launch_bounds__(512) k_main_filter(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_GATHER, i, j);
    const DevParams &p = S.p;
    const bool f16 = kStore == 2 ? p.f16 != 0 : kStore == 1;
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const float4 *__restrict__ pre = S.pre;
    const float *__restrict__ z_h = S.z_h;
    const float2 *__restrict__ dil = S.tiles_dil;
    float4 *out = S.main_;
    const int reach = (int)ceilf(p.rmax_hpx) + 2;
    const int bx = i - (int)threadIdx.x, by = j - (int)threadIdx.y;
    const bool interior = bx - reach >= 0 && by - reach >= 0 && bx + (int)blockDim.x + reach < W2 &&
                          by + (int)blockDim.y + reach < H2;
    if (i >= W2 || j >= H2) return;
    size_t q = (size_t)j * W2 + i;
    float R = __ldg(&dil[(j >> 3) * p.tiles_w + (i >> 3)]).y;
    float z0, r0;
    pre_centre(pre, z_h, q, f16, z0, r0);
    MainAcc m{0.f, 0.f, 0.f, 0.f, 0.f};
    if (f16) {
        if (interior) main_taps<false, true>(i, j, W2, H2, p, pre, z_h, R, z0, r0, m);
        else main_taps<true, true>(i, j, W2, H2, p, pre, z_h, R, z0, r0, m);
    } else {
        if (interior) main_taps<false, false>(i, j, W2, H2, p, pre, z_h, R, z0, r0, m);
        else main_taps<true, false>(i, j, W2, H2, p, pre, z_h, R, z0, r0, m);
    }
    float r = 1.f / m.wsum;
    st_img(out, q, make_float4(m.ax * r, m.ay * r, m.az * r, m.bright * r), f16);
}

// A4 by columns of four pixels: R is the dilated maximum of the pixel's 8 x 8 tile, so
// the four pixels (i, 4jt .. 4jt + 3) of one tile column take every tap at the same x
// (same x weights) and, as long as floor(y + r) = floor(y) + r, at consecutive texel
// rows.  The thread then reads the five rows y0 .. y0 + 4 once (two texels each) instead
// of four rows pairs, and finishes pixel r when row r + 1 arrives; otherwise (the rare
// tap whose rows are not consecutive in FP32) each pixel reads its own two rows.  Every
// pixel sums its texels in the same order and with the same weights as the other forms.
template <bool CLAMP, bool H>
__device__ __forceinline__ void main_strip_taps(int i, int jb, int W2, int H2, const DevParams &p,
                                                const float4 *__restrict__ pre, const float *__restrict__ z_h, float R,
                                                const float *z0, const float *r0, MainAcc *m) {
    const int ring = p.ring;
#pragma unroll 1
    for (int t = 0; t < 81; t++) {
        const float3 u = c_rings[ring][t];
        const float dist = __fmul_rn(u.z, R);
        const float x = fmaf(dist, u.x, (float)i);
        const float xf = floorf(x), fx = x - xf;
        const int x0 = (int)xf;
        float fy[4];
        int y0[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const float y = fmaf(dist, u.y, (float)(jb + r));
            const float yf = floorf(y);
            fy[r] = y - yf;
            y0[r] = (int)yf;
        }
        if (y0[1] == y0[0] + 1 && y0[2] == y0[0] + 2 && y0[3] == y0[0] + 3) {
            const int xa = CLAMP ? min(max(x0, 0), W2 - 1) : x0, xb = CLAMP ? min(max(x0 + 1, 0), W2 - 1) : x0 + 1;
            auto row = [&](int k, float4 &a, float4 &b, float &za, float &zb) {
                const int y = CLAMP ? min(max(y0[0] + k, 0), H2 - 1) : y0[0] + k;
                const size_t q = (size_t)y * W2;
                ld_pre<H>(pre, z_h, q + xa, a, za);
                ld_pre<H>(pre, z_h, q + xb, b, zb);
            };
            float4 a0, b0;
            float za0, zb0;
            row(0, a0, b0, za0, zb0);
#pragma unroll
            for (int r = 0; r < 4; r++) {
                float4 a1, b1;
                float za1, zb1;
                row(r + 1, a1, b1, za1, zb1);
                const float w00 = __fmul_rn(1.f - fx, 1.f - fy[r]), w10 = __fmul_rn(fx, 1.f - fy[r]);
                const float w01 = __fmul_rn(1.f - fx, fy[r]), w11 = __fmul_rn(fx, fy[r]);
                const float4 s = f4fma(w11, b1, f4fma(w01, a1, f4fma(w10, b0, f4scale(w00, a0))));
                const float zi = fmaf(w11, zb1, fmaf(w01, za1, fmaf(w10, zb0, __fmul_rn(w00, za0))));
                main_tap_add(p, dist, z0[r], r0[r], s, zi, m[r]);
                a0 = a1; b0 = b1; za0 = za1; zb0 = zb1;
            }
        } else {
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const float y = fmaf(dist, u.y, (float)(jb + r));
                float4 s;
                float zi;
                if (CLAMP) bilinear4z<H>(pre, z_h, W2, H2, x, y, s, zi);
                else bilinear4z_interior<H>(pre, z_h, W2, x, y, s, zi);
                main_tap_add(p, dist, z0[r], r0[r], s, zi, m[r]);
            }
        }
    }
}

template <class AS, int kStore>
__global__ void __launch_bounds__(512) k_main_filter_strip(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, jt;
    const SessDesc &S = block_session(A, SH_GATHER, i, jt);
    const DevParams &p = S.p;
    const bool f16 = kStore == 2 ? p.f16 != 0 : kStore == 1;
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const float4 *__restrict__ pre = S.pre;
    const float *__restrict__ z_h = S.z_h;
    const float2 *__restrict__ dil = S.tiles_dil;
    float4 *out = S.main_;
    const int reach = (int)ceilf(p.rmax_hpx) + 2;
    const int jb = 4 * jt;
    const int bx = i - (int)threadIdx.x, by = 4 * (jt - (int)threadIdx.y);
    const bool interior = bx - reach >= 0 && by - reach >= 0 && bx + (int)blockDim.x + reach < W2 &&
                          by + 4 * (int)blockDim.y + reach < H2;
    if (i >= W2 || jb >= H2) return;
    const float R = __ldg(&dil[(jb >> 3) * p.tiles_w + (i >> 3)]).y;
    float z0[4], r0[4];
    MainAcc m[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const size_t q = (size_t)min(jb + r, H2 - 1) * W2 + i;
        pre_centre(pre, z_h, q, f16, z0[r], r0[r]);
        m[r] = MainAcc{0.f, 0.f, 0.f, 0.f, 0.f};
    }
    if (f16) {
        if (interior) main_strip_taps<false, true>(i, jb, W2, H2, p, pre, z_h, R, z0, r0, m);
        else main_strip_taps<true, true>(i, jb, W2, H2, p, pre, z_h, R, z0, r0, m);
    } else {
        if (interior) main_strip_taps<false, false>(i, jb, W2, H2, p, pre, z_h, R, z0, r0, m);
        else main_strip_taps<true, false>(i, jb, W2, H2, p, pre, z_h, R, z0, r0, m);
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        if (jb + r >= H2) break;
        const float rw = 1.f / m[r].wsum;
        st_img(out, (size_t)(jb + r) * W2 + i, make_float4(m[r].ax * rw, m[r].ay * rw, m[r].az * rw, m[r].bright * rw),
               f16);
    }
}

// A4 with the block's neighbourhood staged in shared memory: the block's pixels (the
// gather block, SH_GATHER) plus a halo of h = ceil(rmax) + 2 on every side, of the
// prefiltered colour and of z, loaded once with indices clamped to the image.  Every tap
// then reads the tile, which holds exactly the clamped values the other form reads
// through L1, in the same order, so the two forms give the same bits.
constexpr int kMainTileAutoBytes = 64 * 1024;

__host__ __device__ inline int main_tile_halo(float rmax_hpx) { return (int)ceilf(rmax_hpx) + 2; }
// the staged tile: (rgb, rho) and z per texel, or with FP16 storage the 16-byte records
__host__ __device__ inline int main_tile_bytes(float rmax_hpx, int bw, int bh, bool f16) {
    const int h = main_tile_halo(rmax_hpx);
    return (bw + 2 * h) * (bh + 2 * h) * (int)(f16 ? sizeof(float4) : sizeof(float4) + sizeof(float));
}

// the 81 taps of pixel (i, j) from the staged tile (origin (ox, oy), width tw)
template <bool H>
__device__ __forceinline__ void main_tile_taps(const float4 *sm_pre, const float *sm_z, int tw, int ox, int oy, int i,
                                               int j, const DevParams &p, float R, float z0, float r0, MainAcc &m) {
    const int ring = p.ring;
#pragma unroll 3
    for (int t = 0; t < 81; t++) {
        const float3 u = c_rings[ring][t];
        const float dist = __fmul_rn(u.z, R);
        const float x = fmaf(dist, u.x, (float)i), y = fmaf(dist, u.y, (float)j);
        const float xf = floorf(x), yf = floorf(y);
        const float fx = x - xf, fy = y - yf;
        const int b = ((int)yf - oy) * tw + ((int)xf - ox);
        const float w00 = __fmul_rn(1.f - fx, 1.f - fy), w10 = __fmul_rn(fx, 1.f - fy);
        const float w01 = __fmul_rn(1.f - fx, fy), w11 = __fmul_rn(fx, fy);
        float4 c00, c10, c01, c11;
        float z00, z10, z01, z11;
        if (H) {
            pre_unpack(sm_pre[b], c00, z00);
            pre_unpack(sm_pre[b + 1], c10, z10);
            pre_unpack(sm_pre[b + tw], c01, z01);
            pre_unpack(sm_pre[b + tw + 1], c11, z11);
        } else {
            c00 = sm_pre[b]; c10 = sm_pre[b + 1]; c01 = sm_pre[b + tw]; c11 = sm_pre[b + tw + 1];
            z00 = sm_z[b]; z10 = sm_z[b + 1]; z01 = sm_z[b + tw]; z11 = sm_z[b + tw + 1];
        }
        const float4 s = f4fma(w11, c11, f4fma(w01, c01, f4fma(w10, c10, f4scale(w00, c00))));
        const float zi = fmaf(w11, z11, fmaf(w01, z01, fmaf(w10, z10, __fmul_rn(w00, z00))));
        main_tap_add(p, dist, z0, r0, s, zi, m);
    }
}

template <class AS, int kStore>
__global__ void __launch_bounds__(512) k_main_filter_tiled(const __grid_constant__ AS as_) {
    extern __shared__ float4 sm_pre[];
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_GATHER, i, j);
    const DevParams &p = S.p;
    const bool f16 = kStore == 2 ? p.f16 != 0 : kStore == 1;
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const float4 *__restrict__ pre = S.pre;
    const float *__restrict__ z_h = S.z_h;
    const float2 *__restrict__ dil = S.tiles_dil;
    float4 *out = S.main_;
    const int h = main_tile_halo(p.rmax_hpx);
    const int bw = (int)blockDim.x, bh = (int)blockDim.y;
    const int tw = bw + 2 * h, th = bh + 2 * h;
    float *sm_z = reinterpret_cast<float *>(sm_pre + tw * th);     // FP32 storage only
    const int ox = i - (int)threadIdx.x - h, oy = j - (int)threadIdx.y - h;
    for (int e = (int)(threadIdx.y * blockDim.x + threadIdx.x); e < tw * th; e += bw * bh) {
        const int ty = e / tw, tx = e - ty * tw;
        const int x = min(max(ox + tx, 0), W2 - 1), y = min(max(oy + ty, 0), H2 - 1);
        const size_t g = (size_t)y * W2 + x;
        sm_pre[e] = __ldg(&pre[g]);
        if (!f16) sm_z[e] = __ldg(&z_h[g]);
    }
    __syncthreads();
    if (i >= W2 || j >= H2) return;
    const size_t q = (size_t)j * W2 + i;
    const float R = __ldg(&dil[(j >> 3) * p.tiles_w + (i >> 3)]).y;
    float z0, r0;
    pre_centre(pre, z_h, q, f16, z0, r0);
    MainAcc m{0.f, 0.f, 0.f, 0.f, 0.f};
    if (f16) main_tile_taps<true>(sm_pre, sm_z, tw, ox, oy, i, j, p, R, z0, r0, m);
    else main_tile_taps<false>(sm_pre, sm_z, tw, ox, oy, i, j, p, R, z0, r0, m);
    const float r = 1.f / m.wsum;
    st_img(out, q, make_float4(m.ax * r, m.ay * r, m.az * r, m.bright * r), f16);
}

// A5: per-channel 3x3 median (clamp-to-edge).  The block's 34x10 neighbourhood is
// loaded once, coalesced, into one shared-memory plane per channel; each thread then
// selects the median of its 9 values channel by channel (an exact selection, so the
// order of the channels changes nothing).
template <class AS>
__global__ void __launch_bounds__(256) k_median_pp(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_HPX, i, j);
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const float4 *__restrict__ src = S.main_;
    float4 *dst = S.pp_med;
    const bool h = S.p.f16;
    __shared__ float t[4][10][34];
    const int bx = i - (int)threadIdx.x, by = j - (int)threadIdx.y;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    {
        float4 v[2];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int e = min(tid + 256 * r, 10 * 34 - 1);
            const int ty = e / 34, tx = e - 34 * ty;
            const int x = min(max(bx + tx - 1, 0), W2 - 1), y = min(max(by + ty - 1, 0), H2 - 1);
            v[r] = ld_img(src, (size_t)y * W2 + x, h);
        }
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int e = tid + 256 * r;
            if (e < 10 * 34) {
                const int ty = e / 34, tx = e - 34 * ty;
                t[0][ty][tx] = v[r].x; t[1][ty][tx] = v[r].y; t[2][ty][tx] = v[r].z; t[3][ty][tx] = v[r].w;
            }
        }
    }
    __syncthreads();
    if (i >= W2 || j >= H2) return;
    const int cx = (int)threadIdx.x, cy = (int)threadIdx.y;
    float m[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        float a[9];
#pragma unroll
        for (int dy = 0; dy < 3; dy++)
#pragma unroll
            for (int dx = 0; dx < 3; dx++) a[3 * dy + dx] = t[c][cy + dy][cx + dx];
        m[c] = median9s(a);
    }
    st_img(dst, (size_t)j * W2 + i, make_float4(m[0], m[1], m[2], m[3]), h);
}

}  // namespace

int post_init_tables() { return upload_filter_tables(); }

// A1 (and the per-frame counter reset).  The tile dilation (A2) runs inside the kernels
// that read it (the prefilter, which also writes it out, and the mask), so its timing
// slot brackets nothing.
template <class AS>
void launch_tiles_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *tm) {
    const int n = A.ns;
    k_downscale_tiles<AS><<<A.start[SH_HPX][n], dim3(32, 8), 0, st>>>(as);
    count_launches(1);
    tmark(tm, DOF_K_DOWNSCALE, st);
    tmark(tm, DOF_K_DILATE, st);
}

// The SM's opt-in shared memory per block (queried once).
static int smem_optin_bytes() {
    static int bytes = 0;
    if (!bytes) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0)
            bytes = v;
        else
            bytes = 48 * 1024;
        cudaGetLastError();
    }
    return bytes;
}

// Dynamic shared memory of the main filter's staged form for this batch, or 0 when the
// form through L1 runs: always for form 1, else when a session's halo tile exceeds the
// form's limit (64 KB for form 0, the SM's opt-in shared memory for form 2).
int main_filter_tile_bytes(const BatchArgs &A) {
    if (A.main_form == 1 || A.main_form == 3) return 0;
    int bytes = 0;
    for (int s = 0; s < A.ns; s++)
        bytes = max(bytes, main_tile_bytes(A.s[s].p.rmax_hpx, A.gather_w, A.gather_h, A.s[s].p.f16 != 0));
    const int limit = A.main_form == 2 ? smem_optin_bytes() : kMainTileAutoBytes;
    return bytes <= limit ? bytes : 0;
}

// The main filter's forms loaded now, on the current device (which one runs depends on
// the batch's radii, form and storage), the staged form allowed the SM's opt-in shared
// memory.
template <class AS, int kStore>
static void preload_main_filter() {
    cudaFuncAttributes a;
    cudaFuncGetAttributes(&a, k_main_filter<AS, kStore>);
    cudaFuncGetAttributes(&a, k_main_filter_strip<AS, kStore>);
    cudaFuncSetAttribute(k_main_filter_tiled<AS, kStore>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem_optin_bytes());
}
void preload_post_kernels() {
    preload_main_filter<BatchArgs, 0>();
    preload_main_filter<BatchArgs, 1>();
    preload_main_filter<BatchArgs, 2>();
    preload_main_filter<const BatchArgs *, 0>();
    preload_main_filter<const BatchArgs *, 1>();
    preload_main_filter<const BatchArgs *, 2>();
    cudaGetLastError();
}

template <class AS, int kStore>
static void launch_main_filter(const BatchArgs &A, const AS &as, int tile_bytes, cudaStream_t st) {
    const dim3 grid(A.start[SH_GATHER][A.ns]), gb(A.gather_w, A.gather_h);
    if (tile_bytes > 0) k_main_filter_tiled<AS, kStore><<<grid, gb, tile_bytes, st>>>(as);
    else if (A.main_form == 3) k_main_filter_strip<AS, kStore><<<grid, gb, 0, st>>>(as);
    else k_main_filter<AS, kStore><<<grid, gb, 0, st>>>(as);
}

template <class AS>
void launch_pp_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *tm) {
    const int n = A.ns;
    k_prefilter<AS><<<A.start[SH_HPX][n], dim3(32, 8), 0, st>>>(as);
    tmark(tm, DOF_K_PREFILTER, st);
    // the shared-memory form when every session's halo tile fits
    const int tile_bytes = main_filter_tile_bytes(A);
    switch (image_storage_mode(A)) {
    case 0: launch_main_filter<AS, 0>(A, as, tile_bytes, st); break;
    case 1: launch_main_filter<AS, 1>(A, as, tile_bytes, st); break;
    default: launch_main_filter<AS, 2>(A, as, tile_bytes, st); break;
    }
    tmark(tm, DOF_K_MAIN, st);
    k_median_pp<AS><<<A.start[SH_HPX][n], dim3(32, 8), 0, st>>>(as);
    count_launches(3);
    tmark(tm, DOF_K_MEDIAN_PP, st);
}

// the two argument forms: by value (a kernel parameter) and from device memory (graphs)
template void launch_tiles_b<BatchArgs>(const BatchArgs &, const BatchArgs &, cudaStream_t, DofHistory *);
template void launch_tiles_b<const BatchArgs *>(const BatchArgs &, const BatchArgs *const &, cudaStream_t, DofHistory *);
template void launch_pp_b<BatchArgs>(const BatchArgs &, const BatchArgs &, cudaStream_t, DofHistory *);
template void launch_pp_b<const BatchArgs *>(const BatchArgs &, const BatchArgs *const &, cudaStream_t, DofHistory *);

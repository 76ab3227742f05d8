// Gather-filter helpers of libdof shared by the post-process and reconstruction
// kernels: tap tables in constant memory, software bilinear fetches (FP32 weights;
// texture-unit filtering is not used because its weights are low-precision fixed
// point), and the median-of-9 min/max network.
#pragma once

#include <math.h>

#include "dof_internal.cuh"

// unit offsets (cos, sin) of the 8 prefilter taps (angles k pi / 4)
static __constant__ float2 c_pre8[8];
// 81-tap ring kernels: (x, y, radius fraction) -- centre, then rings k = 1..4 of 8k
// taps in the directions 2 pi m / (8k) at radius k / 4.  Row 0: the circle, (x, y) =
// (cos, sin); row n - 2 (n = 3..8): the regular n-gon of circumradius 1 with a vertex
// at angle 0, (x, y) = its boundary point in the same direction, at distance
// cos(pi / n) / cos(phi - pi / n), phi = the direction modulo 2 pi / n.  The radius
// fraction stays the tap's distance in the aperture's own norm.
constexpr int kRingRows = 7;
static __constant__ float3 c_rings[kRingRows][81];

// Fill this translation unit's copy of the tables (computed in double, rounded once).
static inline int upload_filter_tables() {
    float2 pre[8];
    for (int k = 0; k < 8; k++) pre[k] = make_float2((float)cos(k * M_PI / 4.0), (float)sin(k * M_PI / 4.0));
    static float3 ring[kRingRows][81];
    for (int row = 0; row < kRingRows; row++) {
        const int n = row ? row + 2 : 0;
        ring[row][0] = make_float3(0.f, 0.f, 0.f);
        int t = 1;
        for (int k = 1; k <= 4; k++)
            for (int m = 0; m < 8 * k; m++, t++) {
                const double th = 2.0 * M_PI * m / (8.0 * k);
                double rho = 1.0;
                if (n) {
                    const double sector = 2.0 * M_PI / n;
                    const double phi = th - sector * floor(th / sector);
                    rho = cos(M_PI / n) / cos(phi - M_PI / n);
                }
                ring[row][t] = make_float3((float)(rho * cos(th)), (float)(rho * sin(th)), (float)(k / 4.0));
            }
    }
    cudaError_t e1 = cudaMemcpyToSymbol(c_pre8, pre, sizeof(pre));
    cudaError_t e2 = cudaMemcpyToSymbol(c_rings, ring, sizeof(ring));
    return (e1 == cudaSuccess && e2 == cudaSuccess) ? 0 : -1;
}

#ifdef __CUDACC__
// bilinear fetch, clamp-to-edge, texel centres at integer coordinates
__device__ __forceinline__ float4 bilinear4(const float4 *__restrict__ img, int w, int h, float x, float y) {
    float xf = floorf(x), yf = floorf(y);
    float fx = x - xf, fy = y - yf;
    int x0 = (int)xf, y0 = (int)yf;
    int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
    int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
    float4 a = __ldg(&img[(size_t)ya * w + xa]), b = __ldg(&img[(size_t)ya * w + xb]);
    float4 c = __ldg(&img[(size_t)yb * w + xa]), d = __ldg(&img[(size_t)yb * w + xb]);
    float w00 = (1.f - fx) * (1.f - fy), w10 = fx * (1.f - fy), w01 = (1.f - fx) * fy, w11 = fx * fy;
    return f4fma(w11, d, f4fma(w01, c, f4fma(w10, b, f4scale(w00, a))));
}

// The prefilter's output texel (rgb, rho) and the depth z as the main filter reads them.
// FP32 storage: (rgb, rho) in pre, z in z_h.  FP16 storage: one 16-byte record per
// texel in pre, (r, g) and (b, 0) as half2, then rho and z as floats, so that a tap
// reads a texel with one load (rho and z keep FP32: the filter's weights compare them).
__device__ __forceinline__ float4 pre_record(float4 c, float z) {
    __half2 rg = __floats2half2_rn(c.x, c.y), b0 = __floats2half2_rn(c.z, 0.f);
    return make_float4(__uint_as_float(*reinterpret_cast<uint32_t *>(&rg)),
                       __uint_as_float(*reinterpret_cast<uint32_t *>(&b0)), c.w, z);
}
__device__ __forceinline__ void pre_unpack(float4 t, float4 &c, float &z) {
    uint32_t ux = __float_as_uint(t.x), uy = __float_as_uint(t.y);
    const float2 rg = __half22float2(*reinterpret_cast<__half2 *>(&ux));
    const float2 b0 = __half22float2(*reinterpret_cast<__half2 *>(&uy));
    c = make_float4(rg.x, rg.y, b0.x, t.z);
    z = t.w;
}
template <bool H>
__device__ __forceinline__ void ld_pre(const float4 *__restrict__ pre, const float *__restrict__ z_h, size_t i,
                                       float4 &c, float &z) {
    if (H) {
        pre_unpack(__ldg(pre + i), c, z);
    } else {
        c = __ldg(pre + i);
        z = __ldg(z_h + i);
    }
}

// Bilinear fetch of (rgb, rho) and z from the prefilter's output (ld_pre), clamp to edge.
template <bool H>
__device__ __forceinline__ void bilinear4z(const float4 *__restrict__ img, const float *__restrict__ z, int w, int h,
                                           float x, float y, float4 &out, float &zo) {
    float xf = floorf(x), yf = floorf(y);
    float fx = x - xf, fy = y - yf;
    int x0 = (int)xf, y0 = (int)yf;
    int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
    int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
    size_t qa = (size_t)ya * w, qb = (size_t)yb * w;
    float w00 = __fmul_rn(1.f - fx, 1.f - fy), w10 = __fmul_rn(fx, 1.f - fy), w01 = __fmul_rn(1.f - fx, fy),
          w11 = __fmul_rn(fx, fy);
    float4 c00, c10, c01, c11;
    float z00, z10, z01, z11;
    ld_pre<H>(img, z, qa + xa, c00, z00);
    ld_pre<H>(img, z, qa + xb, c10, z10);
    ld_pre<H>(img, z, qb + xa, c01, z01);
    ld_pre<H>(img, z, qb + xb, c11, z11);
    out = f4fma(w11, c11, f4fma(w01, c01, f4fma(w10, c10, f4scale(w00, c00))));
    zo = fmaf(w11, z11, fmaf(w01, z01, fmaf(w10, z10, __fmul_rn(w00, z00))));
}

// Bilinear fetch of (rgb, rho) and z without clamping: the caller guarantees that
// floor(x), floor(y) and their +1 neighbours lie inside the image.
template <bool H>
__device__ __forceinline__ void bilinear4z_interior(const float4 *__restrict__ img, const float *__restrict__ z, int w,
                                                    float x, float y, float4 &out, float &zo) {
    float xf = floorf(x), yf = floorf(y);
    float fx = x - xf, fy = y - yf;
    const size_t q = (size_t)(__float2int_rz(yf) * w + __float2int_rz(xf));
    float w00 = __fmul_rn(1.f - fx, 1.f - fy), w10 = __fmul_rn(fx, 1.f - fy), w01 = __fmul_rn(1.f - fx, fy),
          w11 = __fmul_rn(fx, fy);
    float4 c00, c10, c01, c11;
    float z00, z10, z01, z11;
    ld_pre<H>(img, z, q, c00, z00);
    ld_pre<H>(img, z, q + 1, c10, z10);
    ld_pre<H>(img, z, q + w, c01, z01);
    ld_pre<H>(img, z, q + w + 1, c11, z11);
    out = f4fma(w11, c11, f4fma(w01, c01, f4fma(w10, c10, f4scale(w00, c00))));
    zo = fmaf(w11, z11, fmaf(w01, z01, fmaf(w10, z10, __fmul_rn(w00, z00))));
}

__device__ __forceinline__ void cx4(float4 &a, float4 &b) {
    float4 lo = make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), fminf(a.w, b.w));
    float4 hi = make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
    a = lo;
    b = hi;
}

__device__ __forceinline__ void cx1(float &a, float &b) {
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}

// median of 9 scalars by the same 19-exchange network as median9
__device__ __forceinline__ float median9s(float *p) {
    cx1(p[1], p[2]); cx1(p[4], p[5]); cx1(p[7], p[8]);
    cx1(p[0], p[1]); cx1(p[3], p[4]); cx1(p[6], p[7]);
    cx1(p[1], p[2]); cx1(p[4], p[5]); cx1(p[7], p[8]);
    cx1(p[0], p[3]); cx1(p[5], p[8]); cx1(p[4], p[7]);
    cx1(p[3], p[6]); cx1(p[1], p[4]); cx1(p[2], p[5]);
    cx1(p[4], p[7]); cx1(p[4], p[2]); cx1(p[6], p[4]);
    cx1(p[4], p[2]);
    return p[4];
}

// per-channel median of 9 by the 19-exchange min/max network (Paeth; the GPU median
// of Smith 1996 cited in Section 3.1.3)
__device__ __forceinline__ float4 median9(float4 *p) {
    cx4(p[1], p[2]); cx4(p[4], p[5]); cx4(p[7], p[8]);
    cx4(p[0], p[1]); cx4(p[3], p[4]); cx4(p[6], p[7]);
    cx4(p[1], p[2]); cx4(p[4], p[5]); cx4(p[7], p[8]);
    cx4(p[0], p[3]); cx4(p[5], p[8]); cx4(p[4], p[7]);
    cx4(p[3], p[6]); cx4(p[1], p[4]); cx4(p[2], p[5]);
    cx4(p[4], p[7]); cx4(p[4], p[2]); cx4(p[6], p[4]);
    cx4(p[4], p[2]);
    return p[4];
}
#endif

// Ray geometry shared by the ray kernels (trace.cu) and the rasteriser (raster.cu): the
// ray record with its watertight-test shear, the watertight ray/triangle test, the
// closest-hit record and the shading of a hit.
#pragma once

#include "dof_internal.cuh"

#ifdef __CUDACC__
namespace {

// ---------------------------------------------------------------------------
// ray / box / triangle
// ---------------------------------------------------------------------------
struct Ray {
    float3 o, d, inv;
    float3 off0, off1;  // o * inv moved outward per axis (the fused slab test)
    int perm;           // 2 kz + (kx, ky swapped): the axis order of the watertight test
    int oct;            // direction octant: bit 0/1/2 set where inv.x/y/z < 0
    float Sx, Sy, Sz;
};

__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ Ray make_ray(float3 o, float3 d) {
    Ray r;
    r.o = o; r.d = d;
    auto safe = [](float x) { return fabsf(x) < 1e-30f ? copysignf(1e-30f, x) : x; };
    r.inv = make_float3(1.f / safe(d.x), 1.f / safe(d.y), 1.f / safe(d.z));
    // fma(lo, inv, -o inv) differs from (lo - o) inv by at most 2^-24 |o inv| from the
    // rounding of o inv (the rest is relative to t); the offsets move each slab plane
    // outward by 2^-22 |o inv|, which covers that and the rounding of the offset itself.
    // The lo plane is the near one where inv >= 0, the far one where inv < 0.
    auto out = [](float oi, float inv, float &o0, float &o1) {
        const float e = fabsf(oi) * 2.38418579e-7f;
        o0 = inv >= 0.f ? oi + e : oi - e;
        o1 = inv >= 0.f ? oi - e : oi + e;
    };
    out(o.x * r.inv.x, r.inv.x, r.off0.x, r.off1.x);
    out(o.y * r.inv.y, r.inv.y, r.off0.y, r.off1.y);
    out(o.z * r.inv.z, r.inv.z, r.off0.z, r.off1.z);
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const bool sw = comp(d, kz) < 0.f;
    if (sw) { int t = kx; kx = ky; ky = t; }
    r.perm = 2 * kz + (sw ? 1 : 0);
    r.oct = (r.inv.x < 0.f ? 1 : 0) | (r.inv.y < 0.f ? 2 : 0) | (r.inv.z < 0.f ? 4 : 0);
    float dz = comp(d, kz);
    r.Sx = comp(d, kx) / dz;
    r.Sy = comp(d, ky) / dz;
    r.Sz = 1.f / dz;
    return r;
}

template <int K> __device__ __forceinline__ float cmp3(float3 v) { return K == 0 ? v.x : (K == 1 ? v.y : v.z); }

// Watertight ray/triangle test (Woop, Benthin and Wald, JCGT 2013): shear the
// vertices into ray space, evaluate the three edge functions (without FMA
// contraction, so a shared edge evaluates to exact negatives), double precision only
// when an edge function is exactly zero.  Returns t > 0 or -1.  The axis order is a
// template argument (one instance per permutation), so no component is selected at
// run time.  t = T / det is divided out only when it is positive and not certainly
// beyond `tmax`: |T| > |det| tmax (1 + 2^-20), evaluated in FP32, implies
// T / det > tmax (1 + 2^-21), which rounds above tmax, so a skipped triangle is one
// that the caller's t <= tmax comparison would reject anyway.
template <int KZ, bool SW>
__device__ __forceinline__ float tri_hit_k(const Ray &r, float4 v0, float4 v1, float4 v2, float tmax) {
    constexpr int KX0 = KZ == 2 ? 0 : KZ + 1;
    constexpr int KY0 = KX0 == 2 ? 0 : KX0 + 1;
    constexpr int KX = SW ? KY0 : KX0, KY = SW ? KX0 : KY0;
    const float3 A = make_float3(v0.x - r.o.x, v0.y - r.o.y, v0.z - r.o.z);
    const float3 B = make_float3(v1.x - r.o.x, v1.y - r.o.y, v1.z - r.o.z);
    const float3 C = make_float3(v2.x - r.o.x, v2.y - r.o.y, v2.z - r.o.z);
    const float Akz = cmp3<KZ>(A), Bkz = cmp3<KZ>(B), Ckz = cmp3<KZ>(C);
    const float Ax = __fsub_rn(cmp3<KX>(A), __fmul_rn(r.Sx, Akz));
    const float Ay = __fsub_rn(cmp3<KY>(A), __fmul_rn(r.Sy, Akz));
    const float Bx = __fsub_rn(cmp3<KX>(B), __fmul_rn(r.Sx, Bkz));
    const float By = __fsub_rn(cmp3<KY>(B), __fmul_rn(r.Sy, Bkz));
    const float Cx = __fsub_rn(cmp3<KX>(C), __fmul_rn(r.Sx, Ckz));
    const float Cy = __fsub_rn(cmp3<KY>(C), __fmul_rn(r.Sy, Ckz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.f || V == 0.f || W == 0.f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return -1.f;
    const float det = U + V + W;
    if (det == 0.f) return -1.f;
    const float T = U * (r.Sz * Akz) + V * (r.Sz * Bkz) + W * (r.Sz * Ckz);
    if (det > 0.f ? T <= 0.f : T >= 0.f) return -1.f;           // t <= 0
    if (fabsf(T) > fabsf(det) * tmax * 1.00000095f) return -1.f;  // t > tmax
    const float t = T / det;
    return t > 0.f ? t : -1.f;
}

__device__ __forceinline__ float tri_hit(const Ray &r, float4 v0, float4 v1, float4 v2, float tmax = INFINITY) {
    // conditional branches, not a jump table (an indirect branch stalls the warp)
    const int pm = r.perm;
    if (pm >= 4) return pm == 4 ? tri_hit_k<2, false>(r, v0, v1, v2, tmax) : tri_hit_k<2, true>(r, v0, v1, v2, tmax);
    if (pm >= 2) return pm == 2 ? tri_hit_k<1, false>(r, v0, v1, v2, tmax) : tri_hit_k<1, true>(r, v0, v1, v2, tmax);
    return pm == 0 ? tri_hit_k<0, false>(r, v0, v1, v2, tmax) : tri_hit_k<0, true>(r, v0, v1, v2, tmax);
}

struct HitRec {
    float t;
    int prim;   // original triangle id, -1 = miss
    int k;      // sorted index
};

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16; h *= 0x85EBCA6Bu; h ^= h >> 13; h *= 0xC2B2AE35u; h ^= h >> 16;
    return h;
}

// colour of a hit: per-triangle hash albedo, Lambert + ambient under one directional
// light (material 1: emitter); also the face normal turned towards the ray
__device__ __forceinline__ float3 shade(const DevParams &p, const SceneDev &sc, const HitRec &h, float3 dir,
                                        float3 &n) {
    const float4 *tp = sc.tris + 3 * (size_t)h.k;
    float4 v0 = __ldg(tp), v1 = __ldg(tp + 1), v2 = __ldg(tp + 2);
    n = normalize(cross(make_float3(v1.x - v0.x, v1.y - v0.y, v1.z - v0.z),
                        make_float3(v2.x - v0.x, v2.y - v0.y, v2.z - v0.z)));
    if (dot(n, dir) > 0.f) n = -1.f * n;
    uint32_t base = fmix32(p.albedo_seed);
    float alb[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        uint32_t hh = fmix32(base ^ (uint32_t)(3 * h.prim + c));
        alb[c] = 0.1f + 0.8f * ((float)(hh >> 8) * 5.9604644775390625e-8f);
    }
    if (__float_as_int(v2.w) == 1) return make_float3(p.emit * alb[0], p.emit * alb[1], p.emit * alb[2]);
    float lam = fmaxf(0.f, -dot(n, p.light));
    float k = p.k_a + p.k_d * lam;
    return make_float3(alb[0] * k, alb[1] * k, alb[2] * k);
}

}  // namespace
#endif

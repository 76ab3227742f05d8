// Temporal accumulation and reprojection of the ray-traced layer (Section 3.2.3):
// near field reprojected with the G-buffer surface, far field from the mean far-hit
// position (3x3 neighbour fallback), an exponential moving average whose history
// weight is the covered share of the bilinear footprint, merge on the hit ratio,
// luminance moments and variance; then the 5x5 binomial blur of the variance.
#include "batch.cuh"

namespace {

// rel = the point relative to the previous lens centre; the previous frame's pixels
// sampled the sensor at their position plus its jitter
__device__ __forceinline__ bool project_prev(const DevCam &c, float3 rel, float &xh, float &yh) {
    float zc = dot(rel, c.pF);
    if (!(zc > 0.f)) return false;
    float iz = c.Fpx / zc;
    float x = c.halfW + dot(rel, c.pR) * iz - c.pjx;
    float y = c.halfH - dot(rel, c.pU) * iz - c.pjy;
    xh = 0.5f * x - 0.5f;
    yh = 0.5f * y - 0.5f;
    return fabsf(xh) < 1e7f && fabsf(yh) < 1e7f;
}

struct NearH {
    float4 a;          // sum w (An, h)
    float bn, m1;      // sum w Bn, sum w mu1
    float wv[4], x[4]; // per tap: w (0 for a dropped tap), and its (mu1, variance) for the
    float v[4];        // second variance pass; indexed by the unrolled tap, so in registers
};
struct FarH { float4 a; float bf; };            // (Af, g), Bf

// bilinear history fetch with dropped taps (outside, or without history)
template <bool NEAR>
__device__ __forceinline__ float fetch(const float4 *__restrict__ H0, const float4 *__restrict__ H1,
                                       const float4 *__restrict__ H2, int W2, int H2n, float x, float y,
                                       NearH &nh, FarH &fh) {
    float xf = floorf(x), yf = floorf(y);
    float fx = x - xf, fy = y - yf;
    int x0 = (int)xf, y0 = (int)yf;
    float wsum = 0.f;
#pragma unroll
    for (int t = 0; t < 4; t++) {
        int dx = t & 1, dy = t >> 1;
        int xi = x0 + dx, yi = y0 + dy;
        if (xi < 0 || yi < 0 || xi >= W2 || yi >= H2n) continue;
        size_t q = (size_t)yi * W2 + xi;
        // the three planes are requested together (the third one used to wait for the
        // validity test on the first two)
        const float4 h0 = __ldg(&H0[q]), h1 = __ldg(&H1[q]), h2 = __ldg(&H2[q]);
        if (!(h0.w + h1.w > 0.f)) continue;
        float w = (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy);
        if (NEAR) {
            nh.a = f4fma(w, h0, nh.a);
            nh.bn += w * h2.x;
            nh.m1 += w * h2.z;
            nh.wv[t] = w; nh.x[t] = h2.z; nh.v[t] = h2.w;
        } else {
            fh.a = f4fma(w, h1, fh.a);
            fh.bf += w * h2.y;
        }
        wsum += w;
    }
    return wsum;
}

// The luminance moments are kept as (mean, variance) rather than (mean, mean of
// squares): with weights a_k summing to one (a_k = alpha w_k for the history taps,
// 1 - alpha W for the current value), the new variance is
//     sum a_k v_k + sum a_k (x_k - mean')^2,
// which equals mean-of-squares' - mean'^2 exactly but without its cancellation (the
// ray count of Eq. 4 multiplies the variance by 1e5).
template <class AS>
__global__ void __launch_bounds__(256) k_accumulate(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_HPX, i, j);
    const DevCam &cam = S.cam;
    const DevParams &p = S.p;
    const float *__restrict__ z_h = S.z_h;
    const float4 *__restrict__ rt = S.rt;
    const int32_t *__restrict__ nrays = S.nrays;
    const float4 *__restrict__ hin = S.hist_in;
    const int has_hist = S.valid;
    float4 *hout = S.hist_out, *crt = S.crt;
    float *ct = S.ct, *var = S.var;
    const int W2 = cam.W2, H2 = cam.H2;
    if (i >= W2 || j >= H2) return;
    const size_t N = (size_t)W2 * H2, q = (size_t)j * W2 + i;
    // the pixel's own planes are requested before the branch on its ray count, so the
    // loads overlap
    const int nr = __ldg(&nrays[q]);
    const float zq = __ldg(&z_h[q]);
    float4 rA = __ldg(&rt[q]), rB = __ldg(&rt[N + q]), rC = __ldg(&rt[2 * N + q]), rD = __ldg(&rt[3 * N + q]);
    if (nr <= 0) {
        float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        hout[q] = zero; hout[N + q] = zero; hout[2 * N + q] = zero;
        st_img(crt, q, zero, p.f16);
        ct[q] = 0.f; var[q] = 0.f;
        return;
    }
    float h = rA.w, g = 1.f - h;
    float L = lum709(rA.x + rB.x, rA.y + rB.y, rA.z + rB.z);
    float3 dp = pixel_dir(cam, 2.f * i + 1.f, 2.f * j + 1.f);
    const float3 dO = cam.O - cam.pO;
    // near field: the G-buffer surface, relative to the previous lens centre
    float3 relN = dO + (zq / dot(dp, cam.F)) * dp;
    float3 Xf;
    if (rC.z > 0.f) {
        Xf = make_float3(rD.x, rD.y, rD.z);
    } else {
        float3 acc = make_float3(0.f, 0.f, 0.f);
        int cnt = 0;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int x = i + dx, y = j + dy;
                if (x < 0 || y < 0 || x >= W2 || y >= H2) continue;
                size_t qn = (size_t)y * W2 + x;
                if (__ldg(&nrays[qn]) > 0 && __ldg(&rt[2 * N + qn]).z > 0.f) {
                    float4 d = __ldg(&rt[3 * N + qn]);
                    acc = acc + make_float3(d.x, d.y, d.z);
                    cnt++;
                }
            }
        Xf = cnt ? (1.f / (float)cnt) * acc : cam.O + (zq / dot(dp, cam.F)) * dp;
    }
    NearH nh, ndummy;
    FarH fh, fdummy;
    nh.a = make_float4(0.f, 0.f, 0.f, 0.f); nh.bn = nh.m1 = 0.f;
#pragma unroll
    for (int t = 0; t < 4; t++) nh.wv[t] = nh.x[t] = nh.v[t] = 0.f;
    ndummy = nh;
    fh.a = nh.a; fh.bf = 0.f;
    fdummy = fh;
    float Wn = 0.f, Wf = 0.f, xh, yh;
    if (has_hist) {
        const float4 *H0 = hin, *H1 = hin + N, *H2p = hin + 2 * N;
        // an unchanged camera (pose and jitter) maps the G-buffer surface exactly onto its
        // own pixel
        bool okn = !cam.exact ? project_prev(cam, relN, xh, yh) : (xh = (float)i, yh = (float)j, true);
        if (okn) Wn = fetch<true>(H0, H1, H2p, W2, H2, xh, yh, nh, fdummy);
        // the far field keeps its pixel under an unchanged camera, too (the mean far
        // position would move it by a fraction of a pixel every frame)
        bool okf = !cam.exact ? project_prev(cam, Xf - cam.pO, xh, yh) : (xh = (float)i, yh = (float)j, true);
        if (okf) Wf = fetch<false>(H0, H1, H2p, W2, H2, xh, yh, ndummy, fh);
    }
    const float a = cam.moved ? p.alpha_motion : p.alpha;
    const float kn = 1.f - a * Wn, kf = 1.f - a * Wf;
    float4 An = make_float4(a * nh.a.x + kn * rA.x, a * nh.a.y + kn * rA.y, a * nh.a.z + kn * rA.z,
                            a * nh.a.w + kn * h);
    float4 Af = make_float4(a * fh.a.x + kf * rB.x, a * fh.a.y + kf * rB.y, a * fh.a.z + kf * rB.z,
                            a * fh.a.w + kf * g);
    float Bn = a * nh.bn + kn * rC.x, Bf = a * fh.bf + kf * rC.y;
    float m1 = a * nh.m1 + kn * L;
    float dl = L - m1;
    float v = kn * dl * dl;
    // the taps in order; a dropped tap (w = 0, x = v = 0) adds exactly +0
#pragma unroll
    for (int t = 0; t < 4; t++) {
        float dx = nh.x[t] - m1;
        v += a * nh.wv[t] * (nh.v[t] + dx * dx);
    }
    hout[q] = An;
    hout[N + q] = Af;
    hout[2 * N + q] = make_float4(Bn, Bf, m1, v);
    var[q] = v;
    if (!cam.moved) {
        float r = 1.f / (An.w + Af.w);
        st_img(crt, q, make_float4((An.x + Af.x) * r, (An.y + Af.y) * r, (An.z + Af.z) * r, An.w * r), p.f16);
        ct[q] = (Bn + Bf) * r;
    } else {
        float rn = An.w > 0.f ? 1.f / An.w : 0.f, rf = Af.w > 0.f ? 1.f / Af.w : 0.f;
        st_img(crt, q, make_float4(h * An.x * rn + (1.f - h) * Af.x * rf, h * An.y * rn + (1.f - h) * Af.y * rf,
                                   h * An.z * rn + (1.f - h) * Af.z * rf, h), p.f16);
        ct[q] = h * Bn * rn + (1.f - h) * Bf * rf;
    }
}

}  // namespace

template <class AS>
void launch_temporal_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *tm) {
    const int n = A.ns;
    k_accumulate<AS><<<A.start[SH_HPX][n], dim3(32, 8), 0, st>>>(as);
    count_launches(1);
    tmark(tm, DOF_K_ACCUM, st);
    // the variance blur runs fused with the RT median and mip level 0 (recon.cu)
    tmark(tm, DOF_K_VAR_BLUR, st);
}

// the two argument forms: by value (a kernel parameter) and from device memory (graphs)
template void launch_temporal_b<BatchArgs>(const BatchArgs &, const BatchArgs &, cudaStream_t, DofHistory *);
template void launch_temporal_b<const BatchArgs *>(const BatchArgs &, const BatchArgs *const &, cudaStream_t, DofHistory *);

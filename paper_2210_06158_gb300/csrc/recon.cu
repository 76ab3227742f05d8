// Reconstruction and composite of libdof: 3x3 median of the ray-traced colour over
// pixels with rays, mip pyramid of the premultiplied layer, 81-tap spatial
// reconstruction at LOD clamp(0.05 c_t, 0, 3) blended by b = clamp(2000 sigma^2, 0,
// 0.9) (Section 3.2.4, Eq. 5, Eq. 8), and the per-pixel composite of sharp,
// post-processed and ray-traced colour (Section 3.3, Eq. 6, Eq. 7).
#include "batch.cuh"
#include "filters.cuh"

namespace {

// A9 / A10 / A11, fused per half-resolution pixel: the 5x5 binomial blur of the
// luminance variance (Section 3.2.3), the lower median of the ray-traced colour over the
// valid 3x3 neighbours (invalid slots padded with -inf / +inf so the median-of-9 network
// selects index (k-1)/2 of the k valid values), and the mip pyramid of the
// reconstruction: level 0, (rgb, h) * v and (c_t, 1) * v, then levels 1-3 as 2x2 box
// averages.  The block's neighbourhoods (variance +-2, colour and ray counts +-1) are
// loaded once into shared memory with clamped indices.  A block covers 32x8 pixels of
// level 0 at a multiple of (32, 8), which holds every texel its 16x4 texels of level 1,
// 8x2 of level 2 and 4x1 of level 3 average (indices clamped to each level's size stay
// inside the block); each level is summed from the values of the level below as they are
// stored (FP16 storage rounds them), in the order (0,0), (1,0), (0,1), (1,1).
template <class AS>
__global__ void __launch_bounds__(256) k_resolve_rt(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_HPX, i, j);
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const float4 *__restrict__ crt = S.crt;
    const int32_t *__restrict__ nrays = S.nrays;
    const float *__restrict__ var = S.var;
    const bool hs = S.p.f16;
    __shared__ float t_var[12][36];
    __shared__ float4 t_crt[10][34];
    __shared__ int t_n[10][34];
    __shared__ float4 m0a[8][32];
    __shared__ float2 m0b[8][32];
    const int bx = i - (int)threadIdx.x, by = j - (int)threadIdx.y;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    // the tiles: each thread's (at most two) elements of each are requested before any is
    // stored, so the loads overlap
    {
        float v[2];
        float4 c[2];
        int nn[2];
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int e = tid + 256 * r;
            const int ev = min(e, 12 * 36 - 1), ec = min(e, 10 * 34 - 1);
            const int vy = ev / 36, vx = ev - 36 * vy;
            v[r] = __ldg(&var[(size_t)min(max(by + vy - 2, 0), H2 - 1) * W2 + min(max(bx + vx - 2, 0), W2 - 1)]);
            const int cy2 = ec / 34, cx2 = ec - 34 * cy2;
            const size_t qn = (size_t)min(max(by + cy2 - 1, 0), H2 - 1) * W2 + min(max(bx + cx2 - 1, 0), W2 - 1);
            c[r] = ld_img(crt, qn, hs);
            nn[r] = __ldg(&nrays[qn]);
        }
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const int e = tid + 256 * r;
            if (e < 12 * 36) t_var[e / 36][e % 36] = v[r];
            if (e < 10 * 34) {
                t_crt[e / 34][e % 34] = c[r];
                t_n[e / 34][e % 34] = nn[r];
            }
        }
    }
    __syncthreads();
    const int cx = (int)threadIdx.x, cy = (int)threadIdx.y;
    if (i < W2 && j < H2) {
        const size_t q = (size_t)j * W2 + i;
        // variance blur
        {
            const float b[5] = {1.f, 4.f, 6.f, 4.f, 1.f};
            float acc = 0.f;
#pragma unroll
            for (int dy = 0; dy < 5; dy++) {
                float row = 0.f;
#pragma unroll
                for (int dx = 0; dx < 5; dx++) row += b[dx] * t_var[cy + dy][cx + dx];
                acc += b[dy] * row;
            }
            S.var_out[q] = acc * (1.f / 256.f);
        }
        float4 med = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 centre = t_crt[cy + 1][cx + 1];
        const bool valid = t_n[cy + 1][cx + 1] > 0;
        if (valid) {
            float4 v[9];
            bool ok[9];
            int k = 0, n = 0;
#pragma unroll
            for (int dy = 0; dy < 3; dy++)
#pragma unroll
                for (int dx = 0; dx < 3; dx++) {
                    const int x = i + dx - 1, y = j + dy - 1;
                    const bool in = x >= 0 && y >= 0 && x < W2 && y < H2;
                    ok[n] = in && t_n[cy + dy][cx + dx] > 0;
                    v[n] = in ? t_crt[cy + dy][cx + dx] : centre;
                    k += ok[n];
                    n++;
                }
            int lows = 4 - (k - 1) / 2;   // -inf pads; the rest of the invalid slots get +inf
#pragma unroll
            for (int m = 0; m < 9; m++)
                if (!ok[m]) {
                    float pad = lows > 0 ? -INFINITY : INFINITY;
                    lows--;
                    v[m] = make_float4(pad, pad, pad, pad);
                }
            float4 m9 = median9(v);
            med = make_float4(m9.x, m9.y, m9.z, centre.w);
        }
        st_img(S.rt_med, q, med, hs);
        // mip level 0 from the median as stored (FP16 storage rounds it)
        const float vv = valid ? 1.f : 0.f;
        const float4 l0 = f4scale(vv, round_img(med, hs));
        const float2 l0b = make_float2(vv * __ldg(&S.ct[q]), vv);
        st_mip(S.mip[0], (size_t)W2 * H2, q, l0, l0b, hs);
        m0a[cy][cx] = round_img(l0, hs);
        m0b[cy][cx] = l0b;
    }
    // levels 1-3 from the block's texels of the level below (shared memory), as stored
    __shared__ float4 m1a[4][16], m2a[2][8];
    __shared__ float2 m1b[4][16], m2b[2][8];
    __syncthreads();
    const int L = S.mip_L;
    if (1 < L && tid < 64) {
        const int ux = tid & 15, uy = tid >> 4;          // level-1 texel of the block
        const int i1 = bx / 2 + ux, j1 = by / 2 + uy;
        if (i1 < S.mip_w[1] && j1 < S.mip_h[1]) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 b = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int x = min(2 * i1 + (t & 1), W2 - 1) - bx, y = min(2 * j1 + (t >> 1), H2 - 1) - by;
                a = f4add(a, m0a[y][x]);
                const float2 c = m0b[y][x];
                b.x += c.x; b.y += c.y;
            }
            const float4 v = f4scale(0.25f, a);
            const float2 u = make_float2(0.25f * b.x, 0.25f * b.y);
            const size_t o = (size_t)j1 * S.mip_w[1] + i1;
            st_mip(S.mip[1], (size_t)S.mip_w[1] * S.mip_h[1], o, v, u, hs);
            m1a[uy][ux] = round_img(v, hs);
            m1b[uy][ux] = u;
        }
    }
    __syncthreads();
    if (2 < L && tid < 16) {
        const int ux = tid & 7, uy = tid >> 3;           // level-2 texel of the block
        const int i2 = bx / 4 + ux, j2 = by / 4 + uy;
        if (i2 < S.mip_w[2] && j2 < S.mip_h[2]) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 b = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int x = min(2 * i2 + (t & 1), S.mip_w[1] - 1) - bx / 2;
                const int y = min(2 * j2 + (t >> 1), S.mip_h[1] - 1) - by / 2;
                a = f4add(a, m1a[y][x]);
                const float2 c = m1b[y][x];
                b.x += c.x; b.y += c.y;
            }
            const float4 v = f4scale(0.25f, a);
            const float2 u = make_float2(0.25f * b.x, 0.25f * b.y);
            const size_t o = (size_t)j2 * S.mip_w[2] + i2;
            st_mip(S.mip[2], (size_t)S.mip_w[2] * S.mip_h[2], o, v, u, hs);
            m2a[uy][ux] = round_img(v, hs);
            m2b[uy][ux] = u;
        }
    }
    __syncthreads();
    if (3 < L && tid < 4) {
        const int i3 = bx / 8 + tid, j3 = by / 8;        // level-3 texel of the block
        if (i3 < S.mip_w[3] && j3 < S.mip_h[3]) {
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 b = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int x = min(2 * i3 + (t & 1), S.mip_w[2] - 1) - bx / 4;
                const int y = min(2 * j3 + (t >> 1), S.mip_h[2] - 1) - by / 4;
                a = f4add(a, m2a[y][x]);
                const float2 c = m2b[y][x];
                b.x += c.x; b.y += c.y;
            }
            const size_t o = (size_t)j3 * S.mip_w[3] + i3;
            st_mip(S.mip[3], (size_t)S.mip_w[3] * S.mip_h[3], o, f4scale(0.25f, a), make_float2(0.25f * b.x, 0.25f * b.y),
                   hs);
        }
    }
}

// One level of the pyramid as a tap reads it: texel centres of level l sit at
// 2^l (x + 0.5) - 0.5 in half-resolution pixels, so a half-resolution position x maps
// to x 2^-l + (2^-l - 1) / 2 in level texels.
struct MipLevel {
    const float4 *m;     // the colour plane (FP32 storage) or the records (FP16)
    const float2 *m1;    // FP32 storage: the (c_t, 1) plane
    int w, h;
    float s, c;
};

__device__ __forceinline__ MipLevel mip_level(const SessDesc &S, int l) {
    MipLevel L;
    L.m = S.mip[l]; L.w = S.mip_w[l]; L.h = S.mip_h[l];
    L.m1 = reinterpret_cast<const float2 *>(L.m + (size_t)L.w * L.h);
    L.s = 1.f / (float)(1 << l);
    L.c = 0.5f * L.s - 0.5f;
    return L;
}

// texel i of a level as st_mip stored it
template <bool H>
__device__ __forceinline__ void ld_mip(const MipLevel &L, int i, float4 &a, float2 &b) {
    if (H) {
        const float4 t = __ldg(L.m + i);
        uint32_t ux = __float_as_uint(t.x), uy = __float_as_uint(t.y);
        const float2 fa = __half22float2(*reinterpret_cast<__half2 *>(&ux));
        const float2 fb = __half22float2(*reinterpret_cast<__half2 *>(&uy));
        a = make_float4(fa.x, fa.y, fb.x, fb.y);
        b = make_float2(t.z, t.w);
    } else {
        a = __ldg(L.m + i);
        b = __ldg(L.m1 + i);
    }
}

// Bilinear sample of one level at (x, y), scaled by the level's trilinear weight wl and
// added to (a, b): the trilinear blend of Eq. 8 is folded into the bilinear weights.
template <bool CLAMP, bool H>
__device__ __forceinline__ void bilin_acc(const MipLevel &L, float x, float y, float wl, float4 &a, float2 &b) {
    const float xl = fmaf(x, L.s, L.c), yl = fmaf(y, L.s, L.c);
    const float xf = floorf(xl), yf = floorf(yl);
    const float fx = xl - xf, fy = yl - yf;
    const int x0 = (int)xf, y0 = (int)yf;
    const float gx = 1.f - fx, gy0 = (1.f - fy) * wl, gy1 = fy * wl;
    const float w00 = gx * gy0, w10 = fx * gy0, w01 = gx * gy1, w11 = fx * gy1;
    const int w = L.w;
    int qa, qb, xa, xb;
    if (CLAMP) {
        xa = min(max(x0, 0), w - 1); xb = min(max(x0 + 1, 0), w - 1);
        const int ya = min(max(y0, 0), L.h - 1), yb = min(max(y0 + 1, 0), L.h - 1);
        qa = ya * w; qb = yb * w;
    } else {
        xa = x0; xb = x0 + 1;
        qa = y0 * w; qb = qa + w;
    }
    float4 a00, a10, a01, a11;
    float2 c00, c10, c01, c11;
    ld_mip<H>(L, qa + xa, a00, c00);
    ld_mip<H>(L, qa + xb, a10, c10);
    ld_mip<H>(L, qb + xa, a01, c01);
    ld_mip<H>(L, qb + xb, a11, c11);
    a = f4fma(w00, a00, a);
    a = f4fma(w10, a10, a);
    a = f4fma(w01, a01, a);
    a = f4fma(w11, a11, a);
    b.x = fmaf(w11, c11.x, fmaf(w01, c01.x, fmaf(w10, c10.x, fmaf(w00, c00.x, b.x))));
    b.y = fmaf(w11, c11.y, fmaf(w01, c01.y, fmaf(w10, c10.y, fmaf(w00, c00.y, b.y))));
}

template <bool CLAMP, bool H>
__device__ __forceinline__ void recon_taps(const MipLevel &L0, const MipLevel &L1, int i, int j, float R, float t,
                                           float inv_ramp, int ring, float4 &num, float &den) {
    const float fi = (float)i, fj = (float)j, t0 = 1.f - t;
#pragma unroll 3
    for (int k = 0; k < 81; k++) {
        const float3 u = c_rings[ring][k];
        // dist and the cover weight D are rounded explicitly (no contraction left to the
        // compiler), so that every instance of this kernel computes the same bits
        const float dist = __fmul_rn(u.z, R);
        const float x = fmaf(dist, u.x, fi), y = fmaf(dist, u.y, fj);
        float4 S = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 Sb = make_float2(0.f, 0.f);
        bilin_acc<CLAMP, H>(L0, x, y, t0, S, Sb);
        bilin_acc<CLAMP, H>(L1, x, y, t, S, Sb);
        const float Sc = Sb.x, Sv = Sb.y;
        const float ri = Sv > 0.f ? __fdividef(Sc, Sv) : 0.f;
        const float D = sat(__fmaf_rn(__fsub_rn(ri, dist), inv_ramp, 0.5f));
        num = f4fma(D, S, num);
        den = fmaf(D, Sv, den);
    }
}

// A11: reconstruction.  Blocks whose footprint (+-rmax + 2, at every level) lies
// inside the image take taps without index clamping.  kStore: the launch's image storage
// (image_storage_mode); the specialised instances hold the code of one storage only, and
// with it fewer registers.  72 registers hold either storage's taps without spilling
// (three 256-thread blocks per SM; a cap of 64 spilled the FP32 form's state through
// L1, the unit that bounds it, and was 1-2% slower).
template <class AS, int kStore>
__global__ void __maxnreg__(72) k_recon(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_RECON, i, j);
    const DevParams &p = S.p;
    const bool f16 = kStore == 2 ? p.f16 != 0 : kStore == 1;
    const int W2 = S.cam.W2, H2 = S.cam.H2;
    const int mL = S.mip_L;
    const float4 *__restrict__ med = S.rt_med;
    const float *__restrict__ ct = S.ct;
    const float *__restrict__ var_blur = S.var_out;
    const int32_t *__restrict__ nrays = S.nrays;
    float4 *out = S.recon;
    const int reach = (int)ceilf(p.rmax_hpx) + (2 << (mL - 1)) + 2;
    const int bx = i - (int)threadIdx.x, by = j - (int)threadIdx.y;
    const bool interior = bx - reach >= 0 && by - reach >= 0 && bx + (int)blockDim.x + reach < W2 &&
                          by + (int)blockDim.y + reach < H2;
    if (i >= W2 || j >= H2) return;
    size_t q = (size_t)j * W2 + i;
    if (__ldg(&nrays[q]) <= 0) { st_img(out, q, make_float4(0.f, 0.f, 0.f, 0.f), f16); return; }
    const float4 o = ld_img(med, q, f16);
    const float b = fminf(fmaxf(__ldg(&var_blur[q]) * p.var_w_recon, 0.f), p.b_max);
    // Eq. 5 blends by b: below 2^-24 the filtered term changes the result by less than
    // the rounding of the 81-tap sum itself, so the taps are not taken
    if (!(b >= 5.9604645e-8f)) {
        st_img(out, q, make_float4(o.x + 0.f, o.y + 0.f, o.z + 0.f, o.w + 0.f), f16);
        return;
    }
    float R = __ldg(&ct[q]);
    float lod = fminf(fmaxf(R * p.lod_scale, 0.f), p.lod_max);
    int l0 = (int)floorf(lod);
    float t = lod - (float)l0;
    if (l0 >= mL - 1) { l0 = mL - 1; t = 0.f; }
    const int l1 = min(l0 + 1, mL - 1);
    const MipLevel L0 = mip_level(S, l0), L1 = mip_level(S, l1);
    float4 num = make_float4(0.f, 0.f, 0.f, 0.f);
    float den = 0.f;
    if (f16) {
        if (interior) recon_taps<false, true>(L0, L1, i, j, R, t, p.inv_cover_ramp, p.ring, num, den);
        else recon_taps<true, true>(L0, L1, i, j, R, t, p.inv_cover_ramp, p.ring, num, den);
    } else {
        if (interior) recon_taps<false, false>(L0, L1, i, j, R, t, p.inv_cover_ramp, p.ring, num, den);
        else recon_taps<true, false>(L0, L1, i, j, R, t, p.inv_cover_ramp, p.ring, num, den);
    }
    float4 f = den > 0.f ? f4scale(1.f / den, num) : o;
    st_img(out, q, make_float4(lerpf(o.x, f.x, b), lerpf(o.y, f.y, b), lerpf(o.z, f.z, b), lerpf(o.w, f.w, b)), f16);
}

// A12: composite.  One thread per half-resolution pixel (i, j) writes its 2x2
// full-resolution pixels: their bilinear taps into the half-resolution layers (texel
// centres at 0.5 (x + 0.5) - 0.5, i.e. i -/+ 1/4) all lie in the clamped 3x3
// neighbourhood of (i, j), which is loaded once; weights 1/4 and 3/4 are exact.
template <class AS>
__global__ void __launch_bounds__(256, 4) k_composite(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int i, j;
    const SessDesc &S = block_session(A, SH_HPX, i, j);
    const DevCam &cam = S.cam;
    const DevParams &p = S.p;
    const float4 *__restrict__ color = S.color;
    const float *__restrict__ depth = S.depth;
    const float4 *__restrict__ pp_med = S.pp_med;
    const float4 *__restrict__ recon = S.recon;
    const int32_t *__restrict__ nrays = S.nrays;
    float4 *out = S.comp_out;
    const int W2 = cam.W2, H2 = cam.H2;
    if (i >= W2 || j >= H2) return;
    const bool hs = p.f16;
    // the 2x2 full-resolution inputs are prefetched into L1 first (no registers held),
    // so their misses overlap the neighbourhood's loads
#pragma unroll
    for (int b = 0; b < 2; b++) {
        const size_t f = (size_t)(2 * j + b) * cam.W + 2 * i;
        prefetch_l1(&depth[f]);
        prefetch_l1(S.gf16 ? reinterpret_cast<const void *>(reinterpret_cast<const uint2 *>(color) + f)
                           : reinterpret_cast<const void *>(color + f));
    }
    // accumulators of the 2x2 full-resolution pixels (a, b) -> index 2 b + a; the
    // neighbourhood is visited in raster order, so each pixel sums its four taps in
    // the order (x0, y0), (x0 + 1, y0), (x0, y0 + 1), (x0 + 1, y0 + 1)
    float4 pp[4], rt[4];
    float cov[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        pp[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        rt[k] = pp[k];
        cov[k] = 0.f;
    }
#pragma unroll
    for (int ny = 0; ny < 3; ny++)
#pragma unroll
        for (int nx = 0; nx < 3; nx++) {
            int x = min(max(i + nx - 1, 0), W2 - 1), y = min(max(j + ny - 1, 0), H2 - 1);
            size_t q = (size_t)y * W2 + x;
            const float4 P = ld_img(pp_med, q, hs);
            const bool V = __ldg(&nrays[q]) > 0;
            // a pixel without rays holds zeros in the reconstruction, so the load need not
            // wait for its ray count (only pixels with rays are summed below)
            const float4 R = ld_img(recon, q, hs);
#pragma unroll
            for (int b = 0; b < 2; b++)
#pragma unroll
                for (int a = 0; a < 2; a++) {
                    const int dx = nx - a, dy = ny - b;
                    if (dx < 0 || dx > 1 || dy < 0 || dy > 1) continue;
                    // fx = 3/4 for a = 0 (taps i - 1, i), 1/4 for a = 1 (taps i, i + 1)
                    const float fx = a ? 0.25f : 0.75f, fy = b ? 0.25f : 0.75f;
                    const float w = (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy);
                    const int k = 2 * b + a;
                    pp[k] = f4fma(w, P, pp[k]);
                    if (V) {
                        rt[k] = f4fma(w, R, rt[k]);
                        cov[k] += w;
                    }
                }
        }
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
        for (int a = 0; a < 2; a++) {
            const int k = 2 * b + a;
            const size_t f = (size_t)(2 * j + b) * cam.W + (2 * i + a);
            float z = fminf(__ldg(&depth[f]), p.z_far);
            float c = coc_of(cam, z);
            float ws = sat((1.41421356237309505f - fabsf(c) + 0.5f * p.zof_ramp) / p.zof_ramp);
            const float4 pk = pp[k], rk = rt[k];
            const float cv = cov[k];
            float4 s = ld_img(color, f, S.gf16);
            float bx = pk.x, by = pk.y, bz = pk.z;
            if (cv > 0.f) {
                float ic = 1.f / cv;
                float rx = rk.x * ic, ry = rk.y * ic, rz = rk.z * ic, hh = rk.w * ic;
                float tb;
                if (c < 0.f) {
                    tb = pk.w;
                } else {
                    float u = sat(hh / p.h_edge);
                    tb = u * u * (3.f - 2.f * u);
                }
                bx = lerpf(pk.x, lerpf(rx, pk.x, tb), cv);
                by = lerpf(pk.y, lerpf(ry, pk.y, tb), cv);
                bz = lerpf(pk.z, lerpf(rz, pk.z, tb), cv);
            }
            out[f] = make_float4(lerpf(bx, s.x, ws), lerpf(by, s.y, ws), lerpf(bz, s.z, ws), 1.f);
        }
}


// A13: final TAA (Section 3.4, after Karis 2014), per full-resolution pixel of the
// sessions that ask for it: the surface the pixel shows (depth along its jittered ray)
// projected into the previous frame (minus that frame's jitter) samples the previous
// resolved image bilinearly (clamp to edge, also for points outside the previous image);
// clamped per channel to the min / max of the current 3x3 neighbourhood;
// out = h + taa_alpha (cur - h).  No previous frame or a point behind the previous
// camera: out = cur.
template <class AS>
__global__ void __launch_bounds__(256) k_taa(const __grid_constant__ AS as_) {
    const BatchArgs &A = batch_args(as_);
    int x, y;
    const SessDesc &S = block_session(A, SH_FPX, x, y);
    const DevCam &cam = S.cam;
    const DevParams &p = S.p;
    const int W = cam.W, H = cam.H;
    if (!S.taa || x >= W || y >= H) return;
    const float4 *__restrict__ cur = S.comp_out;
    const size_t q = (size_t)y * W + x;
    const float4 c = __ldg(&cur[q]);
    float3 lo = make_float3(c.x, c.y, c.z), hi = lo;
#pragma unroll
    for (int dy = -1; dy <= 1; dy++)
#pragma unroll
        for (int dx = -1; dx <= 1; dx++) {
            int xx = min(max(x + dx, 0), W - 1), yy = min(max(y + dy, 0), H - 1);
            float4 n = __ldg(&cur[(size_t)yy * W + xx]);
            lo = make_float3(fminf(lo.x, n.x), fminf(lo.y, n.y), fminf(lo.z, n.z));
            hi = make_float3(fmaxf(hi.x, n.x), fmaxf(hi.y, n.y), fmaxf(hi.z, n.z));
        }
    float4 o = make_float4(c.x, c.y, c.z, 1.f);
    if (S.taa_valid) {
        float z = fminf(__ldg(&S.depth[q]), p.z_far);
        float3 dir = pixel_dir(cam, x + 0.5f, y + 0.5f);
        float3 rel = (cam.O + (z / dot(dir, cam.F)) * dir) - cam.pO;
        float zc = dot(rel, cam.pF);
        if (zc > 0.f) {
            float iz = cam.Fpx / zc;
            float u = cam.halfW + dot(rel, cam.pR) * iz - cam.pjx;
            float v = cam.halfH - dot(rel, cam.pU) * iz - cam.pjy;
            {
                float tx = u - 0.5f, ty = v - 0.5f;
                float xf = floorf(tx), yf = floorf(ty);
                float fx = tx - xf, fy = ty - yf;
                int x0 = (int)xf, y0 = (int)yf;
                float3 hsum = make_float3(0.f, 0.f, 0.f);
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    int ddx = t & 1, ddy = t >> 1;
                    int xi = min(max(x0 + ddx, 0), W - 1), yi = min(max(y0 + ddy, 0), H - 1);
                    float w = (ddx ? fx : 1.f - fx) * (ddy ? fy : 1.f - fy);
                    float4 hv = __ldg(&S.taa_in[(size_t)yi * W + xi]);
                    hsum = hsum + w * make_float3(hv.x, hv.y, hv.z);
                }
                float hx = fminf(fmaxf(hsum.x, lo.x), hi.x), hy = fminf(fmaxf(hsum.y, lo.y), hi.y);
                float hz = fminf(fmaxf(hsum.z, lo.z), hi.z);
                o = make_float4(hx + p.taa_alpha * (c.x - hx), hy + p.taa_alpha * (c.y - hy),
                                hz + p.taa_alpha * (c.z - hz), 1.f);
            }
        }
    }
    S.out[q] = o;
    S.taa_out[q] = o;
}

}  // namespace

int recon_init_tables() { return upload_filter_tables(); }

template <class AS>
void launch_recon_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *tm) {
    const int n = A.ns;
    dim3 b(32, 8);
    // the variance blur, the RT median and the whole mip pyramid in one kernel (the mip
    // timing slot brackets nothing)
    k_resolve_rt<AS><<<A.start[SH_HPX][n], b, 0, st>>>(as);
    tmark(tm, DOF_K_MEDIAN_RT, st);
    tmark(tm, DOF_K_MIPS, st);
    const dim3 rg(A.start[SH_RECON][n]), rb(A.recon_w, A.recon_h);
    switch (image_storage_mode(A)) {
    case 0: k_recon<AS, 0><<<rg, rb, 0, st>>>(as); break;
    case 1: k_recon<AS, 1><<<rg, rb, 0, st>>>(as); break;
    default: k_recon<AS, 2><<<rg, rb, 0, st>>>(as); break;
    }
    count_launches(2);
    tmark(tm, DOF_K_RECON, st);
}

// the final TAA and the reconstruction's storage instances loaded now (a kernel first
// launched in a later frame would otherwise stall that frame on its load)
void preload_recon_kernels() {
    cudaFuncAttributes a;
    cudaFuncGetAttributes(&a, k_taa<BatchArgs>);
    cudaFuncGetAttributes(&a, k_taa<const BatchArgs *>);
    cudaFuncGetAttributes(&a, k_recon<BatchArgs, 0>);
    cudaFuncGetAttributes(&a, k_recon<BatchArgs, 1>);
    cudaFuncGetAttributes(&a, k_recon<BatchArgs, 2>);
    cudaFuncGetAttributes(&a, k_recon<const BatchArgs *, 0>);
    cudaFuncGetAttributes(&a, k_recon<const BatchArgs *, 1>);
    cudaFuncGetAttributes(&a, k_recon<const BatchArgs *, 2>);
    cudaGetLastError();
}

template <class AS>
void launch_composite_b(const BatchArgs &A, const AS &as, cudaStream_t st, DofHistory *tm) {
    const int n = A.ns;
    dim3 b(32, 8);
    k_composite<AS><<<A.start[SH_HPX][n], b, 0, st>>>(as);
    tmark(tm, DOF_K_COMPOSITE, st);
    const bool taa = any_taa(A);
    if (taa) k_taa<AS><<<A.start[SH_FPX][n], b, 0, st>>>(as);
    count_launches(taa ? 2 : 1);
    tmark(tm, DOF_K_TAA, st);
}

// the two argument forms: by value (a kernel parameter) and from device memory (graphs)
template void launch_recon_b<BatchArgs>(const BatchArgs &, const BatchArgs &, cudaStream_t, DofHistory *);
template void launch_recon_b<const BatchArgs *>(const BatchArgs &, const BatchArgs *const &, cudaStream_t, DofHistory *);
template void launch_composite_b<BatchArgs>(const BatchArgs &, const BatchArgs &, cudaStream_t, DofHistory *);
template void launch_composite_b<const BatchArgs *>(const BatchArgs &, const BatchArgs *const &, cudaStream_t, DofHistory *);

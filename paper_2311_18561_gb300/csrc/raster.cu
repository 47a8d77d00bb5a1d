// raster.cu -- per-tile compositing (stage c).
//
// Sec. 3.1, Eq. 3 with the depth and opacity channels Sec. 3.1 renders
// beside colour: one CTA per tile of TW x TH pixels, TW x TH/PX threads, each
// thread PX vertically adjacent pixels, each warp an 8 x 4 block of
// threads.  The tile's sorted list is walked front to back in batches of
// one record per thread, staged in shared memory as
//   s0 = (u, v, a', b')   projected mean, conic pre-scaled by -log2(e)
//   s1 = (c', o~)
//   s2 = (r, g, b, z)
// so a pixel's weight is one SFU ex2:
//   alpha = min(0.99, o~ 2^(a' dx^2 + b' dx dy + c' dy^2)).
// A pixel skips alpha < 1/255, stops before a blend that would leave
// T < 1e-4, and accumulates C += c alpha T, D += z alpha T, O += alpha T;
// the CTA leaves the list as soon as every pixel has stopped.  Several
// pixels per thread share each shared-memory load and the loop overhead.
// Every pixel's arithmetic is the same expression whatever TW, TH and PX,
// so images are bit-identical across tile shapes.
#include <type_traits>

#include "raster_common.cuh"

namespace pvg {
namespace {

// Writes the images (and the saved per-pixel state) of a thread's PX pixels.
template <int PX>
__device__ __forceinline__ void composite_epilogue(const Params &P, const ViewDesc &V, const TileGeom &G,
                                                   const float (&T)[PX], const float (&C0)[PX],
                                                   const float (&C1)[PX], const float (&C2)[PX],
                                                   const float (&D)[PX], const float (&O)[PX],
                                                   const uint32_t (&last)[PX]) {
    if (G.px >= V.W) return;
    const size_t HW = (size_t)V.W * V.H;
#pragma unroll
    for (int p = 0; p < PX; p++) {
        const int py = G.py0 + p;
        if (py >= V.H) break;
        const size_t pix = (size_t)py * V.W + G.px;
        if (V.sky) {  // C + (1 - O) f_sky(d)
            size_t ti[4];
            float tw[4];
            sky_texels(V, G.px, py, ti, tw);
            float f[3];
#pragma unroll
            for (int c = 0; c < 3; c++)
                f[c] = tw[0] * V.sky[ti[0] + c] + tw[1] * V.sky[ti[1] + c] + tw[2] * V.sky[ti[2] + c] +
                       tw[3] * V.sky[ti[3] + c];
            const float wo = 1.0f - O[p];
            V.out_rgb[pix] = C0[p] + wo * f[0];
            V.out_rgb[HW + pix] = C1[p] + wo * f[1];
            V.out_rgb[2 * HW + pix] = C2[p] + wo * f[2];
        } else {
            V.out_rgb[pix] = C0[p] + T[p] * V.bg[0];
            V.out_rgb[HW + pix] = C1[p] + T[p] * V.bg[1];
            V.out_rgb[2 * HW + pix] = C2[p] + T[p] * V.bg[2];
        }
        if (V.out_depth) V.out_depth[pix] = D[p];
        if (V.out_alpha) V.out_alpha[pix] = O[p];
        if (P.pix_T) {
            P.pix_T[V.pix_base + pix] = T[p];
            P.pix_last[V.pix_base + pix] = last[p];
        }
    }
}

// The tile's largest last-blend position (how far its adjoint walks),
// by every thread of the CTA once its pixels are written.
template <int PX>
__device__ __forceinline__ void tile_walk_record(const Params &P, const uint32_t (&last)[PX]) {
    __shared__ uint32_t s_walk;
    uint32_t m = last[0];
#pragma unroll
    for (int p = 1; p < PX; p++) m = max(m, last[p]);
    m = __reduce_max_sync(0xffffffffu, m);
    if (threadIdx.x == 0) s_walk = 0u;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&s_walk, m);
    __syncthreads();
    if (threadIdx.x == 0) P.tile_walk[P.tile_order ? P.tile_order[blockIdx.x] : blockIdx.x] = s_walk;
}

// kStats: instead of images, write per pixel the number of list entries
// whose footprint box contains the pixel, up to and including the one
// that stopped it (the compositing work E), and the number of those with
// alpha >= 1/255 (blended, or stopping the pixel).
template <int TW, int TH, int PX, bool kStats>
__global__ void __launch_bounds__(TW *TH / PX) k_composite(Params P) {
    pdl_enter();
    constexpr int BLOCK = TW * TH / PX;
    constexpr uint32_t ALL = (1u << PX) - 1u;
    __shared__ float4 s0[BLOCK];
    __shared__ float2 s1[BLOCK];
    __shared__ float4 s2[BLOCK];
    __shared__ float2 s_half[kStats ? BLOCK : 1];
    const TileGeom G = tile_geom<TW, TH, PX>(P);
    const ViewDesc &V = *G.V;
    const uint2 r = G.r;
    const int tid = threadIdx.x;
    const float fx = (float)G.px + 0.5f;
    float fy[PX];
    float T[PX], C0[PX], C1[PX], C2[PX], D[PX], O[PX];
    uint32_t last[PX], neval[PX], nblend[PX];
    uint32_t done = 0;
#pragma unroll
    for (int p = 0; p < PX; p++) {
        fy[p] = (float)(G.py0 + p) + 0.5f;
        T[p] = 1.0f;
        C0[p] = C1[p] = C2[p] = D[p] = O[p] = 0.f;
        last[p] = 0;
        neval[p] = 0;
        nblend[p] = 0;
        if (!(G.px < V.W && G.py0 + p < V.H)) done |= 1u << p;
    }
    for (uint32_t base = r.x; base < r.y; base += BLOCK) {
        if (__syncthreads_count(done != ALL) == 0) break;
        const uint32_t j = base + tid;
        if (j < r.y) {
            const uint32_t m = P.pair_vals[j];
            stage_record(P, m, s0, s1, s2, tid);
            if constexpr (kStats) s_half[tid] = make_float2(P.rec[3 * (size_t)m + 1].w, P.rec[3 * (size_t)m + 2].w);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)BLOCK, r.y - base);
        for (int k = 0; k < cnt && done != ALL; k++) {
            const float4 g = s0[k];
            const float2 q = s1[k];
            const float4 col = s2[k];
            const uint32_t pos = base + k + 1 - r.x;  // list position after this entry
            const float dx = __fsub_rn(fx, g.x);
            const FalloffColumn fc = falloff_column(g.z, g.w, dx);
            // entries whose o~ cannot reach the cap skip min(cap, .)
            auto pixels = [&](auto capped) {
                constexpr bool kCap = decltype(capped)::value;
#pragma unroll
                for (int p = 0; p < PX; p++) {
                    if (done & (1u << p)) continue;
                    const float dy = __fsub_rn(fy[p], g.y);
                    if constexpr (kStats) {
                        const float2 h = s_half[k];
                        if (fabsf(dx) <= h.x && fabsf(dy) <= h.y) neval[p]++;
                    }
                    const float e = falloff_exp2(fc, q.x, dy);
                    const float raw = __fmul_rn(q.y, ex2_approx(e));
                    if (!(raw >= kAlphaMin)) continue;  // = min(cap, raw) < 1/255, cap > 1/255
                    const float alpha = kCap ? fminf(kAlphaCap, raw) : raw;
                    if constexpr (kStats) nblend[p]++;
                    const float w = __fmul_rn(alpha, T[p]);
                    const float Tn = __fsub_rn(T[p], w);
                    if (Tn < kTStop) {
                        done |= 1u << p;
                        continue;
                    }
                    C0[p] = __fmaf_rn(col.x, w, C0[p]);
                    C1[p] = __fmaf_rn(col.y, w, C1[p]);
                    C2[p] = __fmaf_rn(col.z, w, C2[p]);
                    D[p] = __fmaf_rn(col.w, w, D[p]);
                    O[p] = __fadd_rn(O[p], w);
                    T[p] = Tn;
                    last[p] = pos;
                }
            };
            if (q.y > kUncappedOpacity) pixels(std::true_type{});
            else pixels(std::false_type{});
        }
    }
    if constexpr (kStats) {
        if (G.px >= V.W) return;
#pragma unroll
        for (int p = 0; p < PX; p++) {
            const int py = G.py0 + p;
            if (py >= V.H) break;
            const size_t pix = (size_t)py * V.W + G.px;
            P.pix_neval[V.pix_base + pix] = neval[p];
            P.pix_neval[P.total_pix + V.pix_base + pix] = nblend[p];
        }
    } else {
        composite_epilogue<PX>(P, V, G, T, C0, C1, C2, D, O, last);
        if (P.tile_walk) tile_walk_record<PX>(P, last);
    }
}

// The compositor for an even number of pixels per thread, on packed pairs
// of vertically adjacent pixels: the falloff, alpha, transmittance and
// accumulation of both pixels of a pair take one .f32x2 instruction each.
// The records are staged with their per-pixel operands duplicated into
// pairs.  A pixel of a pair that does not blend (alpha < 1/255, stopped,
// outside the image) adds a zero weight and keeps its T, which leaves its
// sums bit-identical to skipping it, so the images equal the scalar
// kernel's bit for bit.
template <int TW, int TH, int PX>
__global__ void __launch_bounds__(TW *TH / PX) k_composite_x2(Params P) {
    pdl_enter();
    static_assert(PX % 2 == 0, "pairs of pixels");
    constexpr int BLOCK = TW * TH / PX;
    constexpr int NP = PX / 2;
    constexpr uint32_t ALL = (1u << PX) - 1u;
    __shared__ float4 sA[BLOCK];  // (u, a', v, v)
    __shared__ float4 sB[BLOCK];  // (b', b', c', c')
    __shared__ float4 sC[BLOCK];  // (o~, o~, r, r)
    __shared__ float4 sD[BLOCK];  // (g, g, b, b)
    __shared__ float2 sE[BLOCK];  // (z, z)
    const TileGeom G = tile_geom<TW, TH, PX>(P);
    const ViewDesc &V = *G.V;
    const uint2 r = G.r;
    const int tid = threadIdx.x;
    const float fx = (float)G.px + 0.5f;
    const float2 one2 = make_float2(1.0f, 1.0f);
    float2 fy[NP], T[NP], C0[NP], C1[NP], C2[NP], D[NP], O[NP];
    uint32_t last[PX];
    uint32_t done = 0;
#pragma unroll
    for (int q = 0; q < NP; q++) {
        fy[q] = make_float2((float)(G.py0 + 2 * q) + 0.5f, (float)(G.py0 + 2 * q + 1) + 0.5f);
        T[q] = one2;
        C0[q] = C1[q] = C2[q] = D[q] = O[q] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int p = 0; p < PX; p++) {
        last[p] = 0;
        if (!(G.px < V.W && G.py0 + p < V.H)) done |= 1u << p;
    }
    // A pixel that is done (stopped, or outside the image) gets a row
    // coordinate far away: its falloff exponent is then -inf or NaN, its
    // alpha 0 or NaN, and the alpha test (false for NaN) never passes
    // again, so the loop needs no per-pixel done test.
#pragma unroll
    for (int q = 0; q < NP; q++) {
        if (done & (1u << (2 * q))) fy[q].x = kFarRow;
        if (done & (2u << (2 * q))) fy[q].y = kFarRow;
    }
    for (uint32_t base = r.x; base < r.y; base += BLOCK) {
        if (__syncthreads_count(done != ALL) == 0) break;
        const uint32_t j = base + tid;
        if (j < r.y) {
            float4 a, c;
            float2 b;
            record_terms(P.rec, P.pair_vals[j], a, b, c);
            sA[tid] = make_float4(a.x, a.z, a.y, a.y);
            sB[tid] = make_float4(a.w, a.w, b.x, b.x);
            sC[tid] = make_float4(b.y, b.y, c.x, c.x);
            sD[tid] = make_float4(c.y, c.y, c.z, c.z);
            sE[tid] = make_float2(c.w, c.w);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)BLOCK, r.y - base);
        for (int k = 0; k < cnt && done != ALL; k++) {
            const float4 A = sA[k], B = sB[k], Cq = sC[k], Dq = sD[k];
            const float2 E = sE[k];
            const uint32_t pos = base + k + 1 - r.x;  // list position after this entry
            const float dx = __fsub_rn(fx, A.x);
            const FalloffColumn fc = falloff_column(A.y, B.x, dx);
            const float2 A2 = make_float2(fc.A, fc.A), B2 = make_float2(fc.B, fc.B);
            const float2 v2 = make_float2(A.z, A.w), cp2 = make_float2(B.z, B.w);
            const float2 o2 = make_float2(Cq.x, Cq.y), r2 = make_float2(Cq.z, Cq.w);
            const float2 g2 = make_float2(Dq.x, Dq.y), b2 = make_float2(Dq.z, Dq.w);
            // entries whose o~ cannot reach the cap skip min(cap, .)
            auto pairs = [&](auto capped) {
                constexpr bool kCap = decltype(capped)::value;
#pragma unroll
                for (int q = 0; q < NP; q++) {
                    const float2 dy = sub2(fy[q], v2);
                    const float2 e = falloff_exp2_x2(A2, B2, cp2, dy);
                    const float2 a = mul2(o2, make_float2(ex2_approx(e.x), ex2_approx(e.y)));
                    // min(cap, a) >= 1/255 iff a >= 1/255 (cap > 1/255): the cap
                    // is applied to blending pixels only
                    // a done pixel (far row, c' <= -kMinRowCoef) has alpha 0
                    bool bx = a.x >= kAlphaMin, by = a.y >= kAlphaMin;
                    if (!(bx || by)) continue;
                    const float ax = kCap ? fminf(kAlphaCap, a.x) : a.x, ay = kCap ? fminf(kAlphaCap, a.y) : a.y;
                    const float2 al = make_float2(ax, ay);
                    const float2 wu = mul2(al, T[q]);
                    const float2 Tn = sub2(T[q], wu);
                    const bool sx = bx && Tn.x < kTStop, sy = by && Tn.y < kTStop;
                    if (sx || sy) {
                        done |= ((sx ? 1u : 0u) | (sy ? 2u : 0u)) << (2 * q);
                        if (sx) fy[q].x = kFarRow;
                        if (sy) fy[q].y = kFarRow;
                    }
                    bx = bx && !sx;
                    by = by && !sy;
                    // a pixel that does not blend takes w = +0 and T - 0 = T, bit
                    // for bit; a blending one gets the scalar kernel's w and T'
                    const float2 w = make_float2(bx ? wu.x : 0.f, by ? wu.y : 0.f);
                    C0[q] = fma2(r2, w, C0[q]);
                    C1[q] = fma2(g2, w, C1[q]);
                    C2[q] = fma2(b2, w, C2[q]);
                    D[q] = fma2(E, w, D[q]);
                    O[q] = add2(O[q], w);
                    T[q] = sub2(T[q], w);
                    last[2 * q] = bx ? pos : last[2 * q];
                    last[2 * q + 1] = by ? pos : last[2 * q + 1];
                }
            };
            if (Cq.x > kUncappedOpacity) pairs(std::true_type{});
            else pairs(std::false_type{});
        }
    }
    float Ts[PX], C0s[PX], C1s[PX], C2s[PX], Ds[PX], Os[PX];
#pragma unroll
    for (int q = 0; q < NP; q++) {
        Ts[2 * q] = T[q].x; Ts[2 * q + 1] = T[q].y;
        C0s[2 * q] = C0[q].x; C0s[2 * q + 1] = C0[q].y;
        C1s[2 * q] = C1[q].x; C1s[2 * q + 1] = C1[q].y;
        C2s[2 * q] = C2[q].x; C2s[2 * q + 1] = C2[q].y;
        Ds[2 * q] = D[q].x; Ds[2 * q + 1] = D[q].y;
        Os[2 * q] = O[q].x; Os[2 * q + 1] = O[q].y;
    }
    composite_epilogue<PX>(P, V, G, Ts, C0s, C1s, C2s, Ds, Os, last);
    if (P.tile_walk) tile_walk_record<PX>(P, last);
}

template <int TW, int TH, int PX>
void launch_fwd_t(const Params &p, cudaStream_t s) {
    note_launch();
    if constexpr (PX % 2 == 0)
        pdl_launch(k_composite_x2<TW, TH, PX>, p.total_tiles, TW * TH / PX, 0, s, p);
    else
        pdl_launch(k_composite<TW, TH, PX, false>, p.total_tiles, TW * TH / PX, 0, s, p);
}

template <int TW, int TH, int PX>
void launch_stats_t(const Params &p, cudaStream_t s) {
    note_launch();
    pdl_launch(k_composite<TW, TH, PX, true>, p.total_tiles, TW * TH / PX, 0, s, p);
}

}  // namespace

bool composite_supported(int tw, int th, int px) {
#define PVG_CHECK(W, H, X) if (tw == W && th == H && px == X) return true;
    PVG_TILE_CONFIGS(PVG_CHECK)
#undef PVG_CHECK
    return false;
}

#define PVG_DISPATCH_ONE_fwd(W, H, X) \
    if (p.tile_w == W && p.tile_h == H && p.px == X) return launch_fwd_t<W, H, X>(p, s);
#define PVG_DISPATCH_ONE_stats(W, H, X) \
    if (p.tile_w == W && p.tile_h == H && p.px == X) return launch_stats_t<W, H, X>(p, s);

void launch_composite(const Params &p, cudaStream_t s) {
    if (p.total_tiles == 0) return;
    PVG_TILE_CONFIGS(PVG_DISPATCH_ONE_fwd)
}

void launch_composite_stats(const Params &p, cudaStream_t s) {
    if (p.total_tiles == 0) return;
    PVG_TILE_CONFIGS(PVG_DISPATCH_ONE_stats)
}

}  // namespace pvg

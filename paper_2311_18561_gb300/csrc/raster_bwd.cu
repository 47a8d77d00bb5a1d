// raster_bwd.cu -- adjoint of the per-tile compositing (stage d1).
//
// The compositor's CTA shape walks the tile's list back to front from the
// last blended position of any pixel, rebuilding T_i = T_{i+1} / (1 -
// alpha_i).  With X_i = gC.c_i + gD z_i + gO (the pixel's output gradients
// against entry i's channels) and the scalar suffix sum
//   S_i = sum_{j > i} X_j alpha_j T_j  (+ T_final gC.bg),
// the derivative of the pixel's loss with respect to alpha_i is
//   dL/dalpha_i = T_i X_i - S_i / (1 - alpha_i),
// so one scalar per pixel carries what the colour, depth and opacity
// suffix sums would.  The 10 image-space gradient terms of an entry
// (moments of dL/dpower for u, v, conic a b c; o~; r g b; z) are summed
// over a thread's PX pixels, then over the warp by transposing butterflies
// (afterwards lane s holds term s), added to
// per-CTA shared accumulators by 10 lanes at once, and reach global memory with one
// atomic per (Gaussian, tile, term).  Alpha is the forward's expression
// (explicit roundings), so the blend decisions are the forward's; the rest
// of this file may contract a*b+c into fused multiply-adds.
#include <type_traits>

#include "raster_common.cuh"

namespace pvg {
namespace {

// Sum of v[0..NT-1] (NT = 9 or 10) over the warp, as transposing
// butterflies: terms 0..7 within groups of 8 lanes (4 + 2 + 1 exchanges,
// then two folds across the groups); for NT = 10 terms 8, 9 between lane
// pairs (1 exchange, four folds), for NT = 9 term 8 by a plain butterfly.
// On return lane L holds in .x the total of term L & 7 and in .y that of
// term 8 + (L & 1) (NT = 10) or term 8 (NT = 9); lanes 0..NT-1 therefore
// hold term L in .x (L < 8) or .y.  12 shuffles and 44 instructions for
// NT = 10 instead of one 16-slot butterfly's 62.
template <int NT>
__device__ __forceinline__ float2 warp_sum_terms(const float (&v)[10]) {
    static_assert(NT == 9 || NT == 10, "9 or 10 terms");
    const int lane = threadIdx.x & 31;
    bool hi = lane & 4;
    float b[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float send = hi ? v[i] : v[i + 4];
        b[i] = (hi ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    hi = lane & 2;
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float send = hi ? b[i] : b[i + 2];
        c[i] = (hi ? b[i + 2] : b[i]) + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    hi = lane & 1;
    float d = (hi ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, hi ? c[0] : c[1], 1);
    d += __shfl_xor_sync(0xffffffffu, d, 8);
    d += __shfl_xor_sync(0xffffffffu, d, 16);
    float e;
    if constexpr (NT == 10) {
        e = (hi ? v[9] : v[8]) + __shfl_xor_sync(0xffffffffu, hi ? v[8] : v[9], 1);
#pragma unroll
        for (int o = 2; o < 32; o <<= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    } else {
        e = v[8];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    return make_float2(d, e);
}

// Per-pixel state of the adjoint walk: final transmittance, last blended
// position, output gradients and the initial suffix sum (the background's
// share); with a sky map, its gradient is scattered here and its effect on
// dL/dO folded into gO.
struct PixelAdjoint {
    float T, gC0, gC1, gC2, gD, gO, S;
    uint32_t last;
};

__device__ __forceinline__ PixelAdjoint pixel_adjoint(const Params &P, const ViewDesc &V, int px, int py) {
    PixelAdjoint a;
    a.T = 1.0f;
    a.gC0 = a.gC1 = a.gC2 = a.gD = a.gO = 0.f;
    a.last = 0;
    const bool inside = px < V.W && py < V.H;
    if (inside) {
        const size_t HW = (size_t)V.W * V.H, pix = (size_t)py * V.W + px;
        a.T = P.pix_T[V.pix_base + pix];
        a.last = P.pix_last[V.pix_base + pix];
        if (V.dl_rgb) {
            a.gC0 = V.dl_rgb[pix];
            a.gC1 = V.dl_rgb[HW + pix];
            a.gC2 = V.dl_rgb[2 * HW + pix];
        }
        if (V.dl_depth) a.gD = V.dl_depth[pix];
        if (V.dl_alpha) a.gO = V.dl_alpha[pix];
    }
    a.S = a.T * (a.gC0 * V.bg[0] + a.gC1 * V.bg[1] + a.gC2 * V.bg[2]);
    if (V.sky && inside) {
        // colour = C + (1 - O) f: no constant background, dL/dO -= gC.f,
        // dL/df = (1 - O) gC scattered to the four texels
        size_t ti[4];
        float tw[4];
        sky_texels(V, px, py, ti, tw);
        const float gc[3] = {a.gC0, a.gC1, a.gC2};
        const float wo = a.T;  // 1 - O = T_final
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float f = tw[0] * V.sky[ti[0] + c] + tw[1] * V.sky[ti[1] + c] + tw[2] * V.sky[ti[2] + c] +
                            tw[3] * V.sky[ti[3] + c];
            a.gO -= gc[c] * f;
            if (V.g_sky && gc[c] != 0.f)
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (tw[q] != 0.f) atomicAdd(V.g_sky + ti[q] + c, tw[q] * wo * gc[c]);
        }
        a.S = 0.f;
    }
    return a;
}

// Image-space gradients of a staged entry from its CTA-summed terms:
//   d/da = -m_xx / 2, d/db = -m_xy, d/dc = -m_yy / 2,
//   d/du = (a m_x + b m_y) = -(2 a' m_x + b' m_y) / log2(e),
//   d/dv = (b m_x + c m_y) = -(b' m_x + 2 c' m_y) / log2(e);
// colour terms are zeroed where the forward clamped (col <= 0).
__device__ __forceinline__ void flush_entry(float *dst, const float *a, float ap, float bp, float cp, float r,
                                            float g, float b) {
    float gt[10];
    gt[0] = -0.6931471805599453f * (2.f * ap * a[0] + bp * a[1]);
    gt[1] = -0.6931471805599453f * (bp * a[0] + 2.f * cp * a[1]);
    gt[2] = -0.5f * a[2];
    gt[3] = -a[3];
    gt[4] = -0.5f * a[4];
    gt[5] = a[5];
    gt[6] = r > 0.f ? a[6] : 0.f;
    gt[7] = g > 0.f ? a[7] : 0.f;
    gt[8] = b > 0.f ? a[8] : 0.f;
    gt[9] = a[9];
#pragma unroll
    for (int c = 0; c < 10; c++)
        if (gt[c] != 0.f) atomicAdd(dst + c, gt[c]);
}

// kAux: the call has depth or opacity-map gradients or a sky map (dL/dO
// and the depth term of X can be non-zero); without them X = gC.c and the
// depth term is not reduced (9 terms).
template <int TW, int TH, int PX, bool kAux>
__global__ void __launch_bounds__(TW *TH / PX) k_composite_bwd(Params P) {
    pdl_enter();
    constexpr int BLOCK = TW * TH / PX;
    constexpr int NG = 10;               // shared accumulator stride
    constexpr int NT = kAux ? 10 : 9;    // terms reduced
    __shared__ float4 s0[BLOCK];
    __shared__ float2 s1[BLOCK];
    __shared__ float4 s2[BLOCK];
    __shared__ uint32_t s_m[BLOCK];
    __shared__ float s_acc[BLOCK * NG];
    __shared__ uint32_t s_maxlast;
    const TileGeom Gm = tile_geom<TW, TH, PX>(P);
    const ViewDesc &V = *Gm.V;
    const uint2 r = Gm.r;
    const int tid = threadIdx.x, lane = tid & 31;
    const float fx = (float)Gm.px + 0.5f;

    float fy[PX], T[PX], gC0[PX], gC1[PX], gC2[PX], gD[PX], gO[PX];
    float S[PX];  // suffix sum of X_j alpha_j T_j
    uint32_t last[PX];
    uint32_t maxlast = 0;
#pragma unroll
    for (int p = 0; p < PX; p++) {
        fy[p] = (float)(Gm.py0 + p) + 0.5f;
        PixelAdjoint a = pixel_adjoint(P, V, Gm.px, Gm.py0 + p);
        T[p] = a.T; last[p] = a.last; S[p] = a.S;
        gC0[p] = a.gC0; gC1[p] = a.gC1; gC2[p] = a.gC2; gD[p] = a.gD; gO[p] = a.gO;
        maxlast = max(maxlast, last[p]);
    }
    if (tid == 0) s_maxlast = 0;
    __syncthreads();
    if (maxlast) atomicMax(&s_maxlast, maxlast);
    __syncthreads();
    const uint32_t n = s_maxlast;
    // gv: an entry's 10 terms over this thread's pixels, zero between
    // entries (reset after each warp reduction).  The pixels share dx, so
    // the conic moments are kept as sum gpow (A0), sum gpow dy (gv[1]) and
    // sum gpow dy^2 (gv[4]) and expanded once: m_x = dx A0, m_xx = dx^2 A0,
    // m_xy = dx m_y.
    float gv[NG];
#pragma unroll
    for (int c = 0; c < NG; c++) gv[c] = 0.f;
    float A0 = 0.f;
    for (uint32_t end = r.x + n; end > r.x;) {
        const uint32_t start = end - r.x > (uint32_t)BLOCK ? end - BLOCK : r.x;
        const int cnt = (int)(end - start);
        __syncthreads();
        if (tid < cnt) {
            const uint32_t m = P.pair_vals[start + tid];
            stage_record(P, m, s0, s1, s2, tid);
            s_m[tid] = m;
        }
        for (int k = tid; k < BLOCK * NG; k += BLOCK) s_acc[k] = 0.f;
        __syncthreads();
        for (int k = cnt - 1; k >= 0; k--) {
            const uint32_t pos = start + k - r.x;  // list position
            bool contrib = false;
            if (pos < maxlast) {  // before the last blend of one of this thread's pixels
                const float4 g = s0[k];
                const float2 q = s1[k];
                const float4 col = s2[k];
                const float dx = __fsub_rn(fx, g.x);
                const FalloffColumn fc = falloff_column(g.z, g.w, dx);
                // entries whose o~ cannot reach the cap skip min(cap, .)
                auto pixels = [&](auto capped) {
                    constexpr bool kCap = decltype(capped)::value;
#pragma unroll
                    for (int p = 0; p < PX; p++) {
                        if (pos >= last[p]) continue;
                        const float dy = __fsub_rn(fy[p], g.y);
                        const float e = falloff_exp2(fc, q.x, dy);
                        const float G = ex2_approx(e);
                        const float raw = __fmul_rn(q.y, G);
                        if (!(raw >= kAlphaMin)) continue;  // = min(cap, raw) < 1/255, cap > 1/255
                        const float alpha = kCap ? fminf(kAlphaCap, raw) : raw;
                        contrib = true;
                        const float inv = rcp_approx(1.0f - alpha);
                        const float Ti = T[p] * inv;
                        const float w = alpha * Ti;
                        float X = gC0[p] * col.x + gC1[p] * col.y + gC2[p] * col.z;
                        if constexpr (kAux) X += gD[p] * col.w + gO[p];
                        const float ga = Ti * X - inv * S[p];
                        gv[6] += gC0[p] * w;
                        gv[7] += gC1[p] * w;
                        gv[8] += gC2[p] * w;
                        if constexpr (kAux) gv[9] += gD[p] * w;
                        if (!kCap || raw <= kAlphaCap) {
                            // moments of gpow = dL/dpower (d alpha / d power = alpha);
                            // the conic is applied once per Gaussian in the flush
                            gv[5] += ga * G;
                            const float gpow = ga * alpha;
                            const float my = gpow * dy;
                            A0 += gpow;
                            gv[1] += my;
                            gv[4] += my * dy;
                        }
                        S[p] += X * w;
                        T[p] = Ti;
                    }
                };
                if (q.y > kUncappedOpacity) pixels(std::true_type{});
                else pixels(std::false_type{});
                if (contrib) {
                    gv[0] = dx * A0;
                    gv[2] = dx * gv[0];
                    gv[3] = dx * gv[1];
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                const float2 tot = warp_sum_terms<NT>(gv);
                if (lane < NT) atomicAdd(&s_acc[k * NG + lane], lane < 8 ? tot.x : tot.y);
#pragma unroll
                for (int c = 0; c < NG; c++) gv[c] = 0.f;
                A0 = 0.f;
            }
        }
        __syncthreads();
        for (int k = tid; k < cnt; k += BLOCK)
            flush_entry(&P.g2d[10 * (size_t)s_m[k]], &s_acc[k * NG], s0[k].z, s0[k].w, s1[k].x, s2[k].x, s2[k].y,
                        s2[k].z);
        end = start;
    }
}

template <int TW, int TH, int PX>
void launch_bwd_t(const Params &p, cudaStream_t s) {
    note_launch();
    if (p.aux)
        pdl_launch(k_composite_bwd<TW, TH, PX, true>, p.total_tiles, TW * TH / PX, 0, s, p);
    else
        pdl_launch(k_composite_bwd<TW, TH, PX, false>, p.total_tiles, TW * TH / PX, 0, s, p);
}

}  // namespace

#define PVG_DISPATCH_ONE_bwd(W, H, X) \
    if (p.tile_w == W && p.tile_h == H && p.px == X) return launch_bwd_t<W, H, X>(p, s);

void launch_composite_bwd(const Params &p, cudaStream_t s) {
    if (p.total_tiles == 0) return;
    PVG_TILE_CONFIGS(PVG_DISPATCH_ONE_bwd)
}

}  // namespace pvg

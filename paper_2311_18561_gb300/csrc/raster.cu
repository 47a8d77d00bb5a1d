// raster.cu -- per-tile compositing (stage c) and its adjoint (stage d1).
//
// Forward (Sec. 3.1, Eq. 3 with the depth / opacity channels of "flexible
// rendering"): one CTA per tile of TW x TH pixels, TW x TH/PX threads, each
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
//
// Backward: the same CTA walks the list back to front from the last
// blended position of any pixel, rebuilding T_i = T_{i+1} / (1 - alpha_i)
// and the suffix sums S = sum_{j > i} x_j alpha_j T_j (+ T_final bg for
// colour), so dL/dalpha_i = T_i (gC.c_i + gD z_i + gO)
//                         - (gC.S_C + gD S_D + gO S_O) / (1 - alpha_i).
// The 10 image-space gradient terms of an entry (u, v, conic a b c, o~,
// r g b, z) are summed over a thread's PX pixels, then over the warp by a
// transposing butterfly (16 shuffles; afterwards lane 2s holds term s),
// added to per-CTA shared accumulators by 10 lanes at once, and reach
// global memory with one atomic per (Gaussian, tile, term).
#include "pvg_internal.cuh"

namespace pvg {
namespace {

struct TileGeom {
    const ViewDesc *V;
    int px, py0;  // this thread's first pixel (column px, rows py0 .. py0 + PX - 1)
    uint2 r;      // list range
};

template <int TW, int TH, int PX>
__device__ __forceinline__ TileGeom tile_geom(const Params &P) {
    static_assert(TW % 8 == 0 && (TH / PX) % 4 == 0 && TH % PX == 0, "tile must be whole 8x4-thread warps");
    TileGeom g;
    const uint32_t tile = P.tile_order ? P.tile_order[blockIdx.x] : blockIdx.x;
    const int view = view_of_tile(P.views, P.n_views, tile);
    g.V = &P.views[view];
    const uint32_t lt = tile - g.V->tile_base;
    const int tx = (int)(lt % (uint32_t)g.V->tiles_x), ty = (int)(lt / (uint32_t)g.V->tiles_x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wx = warp % (TW / 8), wy = warp / (TW / 8);
    g.px = tx * TW + wx * 8 + (lane & 7);
    g.py0 = ty * TH + (wy * 4 + (lane >> 3)) * PX;
    g.r = P.ranges[tile];
    return g;
}

__device__ __forceinline__ void stage_record(const Params &P, uint32_t m, float4 *s0, float2 *s1, float4 *s2,
                                             int slot) {
    float4 a, c;
    float2 b;
    record_terms(P.rec, m, a, b, c);
    s0[slot] = a;
    s1[slot] = b;
    s2[slot] = c;
}

// kStats: instead of images, write per pixel the number of list entries
// whose footprint box contains the pixel, up to and including the one
// that stopped it (the compositing work E), and the number of those with
// alpha >= 1/255 (blended, or stopping the pixel).
template <int TW, int TH, int PX, bool kStats>
__global__ void __launch_bounds__(TW *TH / PX) k_composite(Params P) {
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
            const float dx = __fsub_rn(fx, g.x);
#pragma unroll
            for (int p = 0; p < PX; p++) {
                if (done & (1u << p)) continue;
                const float dy = __fsub_rn(fy[p], g.y);
                if constexpr (kStats) {
                    const float2 h = s_half[k];
                    if (fabsf(dx) <= h.x && fabsf(dy) <= h.y) neval[p]++;
                }
                const float e = falloff_exp2(g.z, g.w, q.x, dx, dy);
                const float alpha = fminf(kAlphaCap, __fmul_rn(q.y, ex2_approx(e)));
                if (alpha < kAlphaMin) continue;
                if constexpr (kStats) nblend[p]++;
                const float Tn = __fmul_rn(T[p], __fsub_rn(1.0f, alpha));
                if (Tn < kTStop) {
                    done |= 1u << p;
                    continue;
                }
                const float w = __fmul_rn(alpha, T[p]);
                const float4 col = s2[k];
                C0[p] = __fmaf_rn(col.x, w, C0[p]);
                C1[p] = __fmaf_rn(col.y, w, C1[p]);
                C2[p] = __fmaf_rn(col.z, w, C2[p]);
                D[p] = __fmaf_rn(col.w, w, D[p]);
                O[p] = __fadd_rn(O[p], w);
                T[p] = Tn;
                last[p] = base + k + 1 - r.x;
            }
        }
    }
    if (G.px >= V.W) return;
    const size_t HW = (size_t)V.W * V.H;
#pragma unroll
    for (int p = 0; p < PX; p++) {
        const int py = G.py0 + p;
        if (py >= V.H) break;
        const size_t pix = (size_t)py * V.W + G.px;
        if (kStats) {
            P.pix_neval[V.pix_base + pix] = neval[p];
            P.pix_neval[P.total_pix + V.pix_base + pix] = nblend[p];
            continue;
        }
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

// Sum of v[0..9] over the warp.  On return lane L holds the total of term
// L >> 1 (terms 10..15 are padding and hold 0).
__device__ __forceinline__ float warp_sum10(const float (&v)[10]) {
    const int lane = threadIdx.x & 31;
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; i++) a[i] = i < 10 ? v[i] : 0.f;
    bool hi = lane & 16;
    float b[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const float send = hi ? a[i] : a[i + 8];
        b[i] = (hi ? a[i + 8] : a[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    hi = lane & 8;
    float c[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float send = hi ? b[i] : b[i + 4];
        c[i] = (hi ? b[i + 4] : b[i]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    hi = lane & 4;
    float d[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float send = hi ? c[i] : c[i + 2];
        d[i] = (hi ? c[i + 2] : c[i]) + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    hi = lane & 2;
    const float send = hi ? d[0] : d[1];
    float e = (hi ? d[1] : d[0]) + __shfl_xor_sync(0xffffffffu, send, 2);
    e += __shfl_xor_sync(0xffffffffu, e, 1);
    return e;
}

template <int TW, int TH, int PX>
__global__ void __launch_bounds__(TW *TH / PX) k_composite_bwd(Params P) {
    constexpr int BLOCK = TW * TH / PX;
    constexpr int NG = 10;
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
    const size_t HW = (size_t)V.W * V.H;

    float fy[PX], T[PX], gC0[PX], gC1[PX], gC2[PX], gD[PX], gO[PX];
    float sC0[PX], sC1[PX], sC2[PX], sD[PX], sO[PX];
    uint32_t last[PX];
    uint32_t maxlast = 0;
#pragma unroll
    for (int p = 0; p < PX; p++) {
        const int py = Gm.py0 + p;
        fy[p] = (float)py + 0.5f;
        T[p] = 1.0f;
        gC0[p] = gC1[p] = gC2[p] = gD[p] = gO[p] = 0.f;
        last[p] = 0;
        if (Gm.px < V.W && py < V.H) {
            const size_t pix = (size_t)py * V.W + Gm.px;
            T[p] = P.pix_T[V.pix_base + pix];
            last[p] = P.pix_last[V.pix_base + pix];
            if (V.dl_rgb) {
                gC0[p] = V.dl_rgb[pix];
                gC1[p] = V.dl_rgb[HW + pix];
                gC2[p] = V.dl_rgb[2 * HW + pix];
            }
            if (V.dl_depth) gD[p] = V.dl_depth[pix];
            if (V.dl_alpha) gO[p] = V.dl_alpha[pix];
        }
        sC0[p] = T[p] * V.bg[0];
        sC1[p] = T[p] * V.bg[1];
        sC2[p] = T[p] * V.bg[2];
        sD[p] = sO[p] = 0.f;
        if (V.sky && Gm.px < V.W && py < V.H) {
            // colour = C + (1 - O) f: no constant background, dL/dO -= gC.f,
            // dL/df = (1 - O) gC scattered to the four texels
            size_t ti[4];
            float tw[4];
            sky_texels(V, Gm.px, py, ti, tw);
            const float gc[3] = {gC0[p], gC1[p], gC2[p]};
            const float wo = T[p];  // 1 - O = T_final
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float f = tw[0] * V.sky[ti[0] + c] + tw[1] * V.sky[ti[1] + c] + tw[2] * V.sky[ti[2] + c] +
                                tw[3] * V.sky[ti[3] + c];
                gO[p] -= gc[c] * f;
                if (V.g_sky && gc[c] != 0.f)
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (tw[q] != 0.f) atomicAdd(V.g_sky + ti[q] + c, tw[q] * wo * gc[c]);
            }
            sC0[p] = sC1[p] = sC2[p] = 0.f;
        }
        maxlast = max(maxlast, last[p]);
    }
    if (tid == 0) s_maxlast = 0;
    __syncthreads();
    if (maxlast) atomicMax(&s_maxlast, maxlast);
    __syncthreads();
    const uint32_t n = s_maxlast;
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
            float gv[NG];
#pragma unroll
            for (int c = 0; c < NG; c++) gv[c] = 0.f;
            bool contrib = false;
            const float4 g = s0[k];
            const float2 q = s1[k];
            const float4 col = s2[k];
            const float dx = __fsub_rn(fx, g.x);
#pragma unroll
            for (int p = 0; p < PX; p++) {
                if (pos >= last[p]) continue;
                const float dy = __fsub_rn(fy[p], g.y);
                const float e = falloff_exp2(g.z, g.w, q.x, dx, dy);
                const float G = ex2_approx(e);
                const float raw = __fmul_rn(q.y, G);
                const float alpha = fminf(kAlphaCap, raw);
                if (alpha < kAlphaMin) continue;
                contrib = true;
                const float inv = __frcp_rn(1.0f - alpha);
                const float Ti = T[p] * inv;
                const float w = alpha * Ti;
                const float ga = Ti * (gC0[p] * col.x + gC1[p] * col.y + gC2[p] * col.z + gD[p] * col.w + gO[p]) -
                                 inv * (gC0[p] * sC0[p] + gC1[p] * sC1[p] + gC2[p] * sC2[p] + gD[p] * sD[p] +
                                        gO[p] * sO[p]);
                gv[6] += gC0[p] * w;
                gv[7] += gC1[p] * w;
                gv[8] += gC2[p] * w;
                gv[9] += gD[p] * w;
                if (raw <= kAlphaCap) {
                    // moments of gpow = dL/dpower (d alpha / d power = alpha);
                    // the conic is applied once per Gaussian in the flush
                    gv[5] += ga * G;
                    const float gpow = ga * alpha;
                    const float mx = gpow * dx, my = gpow * dy;
                    gv[0] += mx;
                    gv[1] += my;
                    gv[2] += mx * dx;
                    gv[3] += mx * dy;
                    gv[4] += my * dy;
                }
                sC0[p] += col.x * w;
                sC1[p] += col.y * w;
                sC2[p] += col.z * w;
                sD[p] += col.w * w;
                sO[p] += w;
                T[p] = Ti;
            }
            if (__any_sync(0xffffffffu, contrib)) {
                const float tot = warp_sum10(gv);
                if ((lane & 1) == 0 && (lane >> 1) < NG) atomicAdd(&s_acc[k * NG + (lane >> 1)], tot);
            }
        }
        __syncthreads();
        // image-space gradients of each staged Gaussian from its moments:
        //   d/da = -m_xx / 2, d/db = -m_xy, d/dc = -m_yy / 2,
        //   d/du = (a m_x + b m_y) = -(2 a' m_x + b' m_y) / log2(e),
        //   d/dv = (b m_x + c m_y) = -(b' m_x + 2 c' m_y) / log2(e)
        for (int k = tid; k < cnt; k += BLOCK) {
            const float *a = &s_acc[k * NG];
            const float ap = s0[k].z, bp = s0[k].w, cp = s1[k].x;
            float gt[NG];
            gt[0] = -0.6931471805599453f * (2.f * ap * a[0] + bp * a[1]);
            gt[1] = -0.6931471805599453f * (bp * a[0] + 2.f * cp * a[1]);
            gt[2] = -0.5f * a[2];
            gt[3] = -a[3];
            gt[4] = -0.5f * a[4];
#pragma unroll
            for (int c = 5; c < NG; c++) gt[c] = a[c];
            float *dst = &P.g2d[10 * (size_t)s_m[k]];
#pragma unroll
            for (int c = 0; c < NG; c++)
                if (gt[c] != 0.f) atomicAdd(dst + c, gt[c]);
        }
        end = start;
    }
}

template <int TW, int TH, int PX>
void launch_fwd_t(const Params &p, cudaStream_t s) {
    note_launch();
    k_composite<TW, TH, PX, false><<<p.total_tiles, TW * TH / PX, 0, s>>>(p);
}

template <int TW, int TH, int PX>
void launch_stats_t(const Params &p, cudaStream_t s) {
    note_launch();
    k_composite<TW, TH, PX, true><<<p.total_tiles, TW * TH / PX, 0, s>>>(p);
}

template <int TW, int TH, int PX>
void launch_bwd_t(const Params &p, cudaStream_t s) {
    note_launch();
    k_composite_bwd<TW, TH, PX><<<p.total_tiles, TW * TH / PX, 0, s>>>(p);
}

// Supported (tile width, tile height, pixels per thread) combinations.
#define PVG_TILE_CONFIGS(X)                                                                               \
    X(16, 16, 1) X(16, 16, 2) X(16, 16, 4) X(8, 8, 1) X(8, 8, 2) X(16, 8, 1) X(16, 8, 2) X(32, 8, 1)    \
    X(32, 16, 1) X(32, 16, 2) X(32, 16, 4) X(32, 32, 4) X(16, 32, 4)

}  // namespace

bool composite_supported(int tw, int th, int px) {
#define PVG_CHECK(W, H, X) if (tw == W && th == H && px == X) return true;
    PVG_TILE_CONFIGS(PVG_CHECK)
#undef PVG_CHECK
    return false;
}

#define PVG_DISPATCH(FN)        \
    if (p.total_tiles == 0) return; \
    PVG_TILE_CONFIGS(PVG_DISPATCH_ONE_##FN)

#define PVG_DISPATCH_ONE_fwd(W, H, X) \
    if (p.tile_w == W && p.tile_h == H && p.px == X) return launch_fwd_t<W, H, X>(p, s);
#define PVG_DISPATCH_ONE_stats(W, H, X) \
    if (p.tile_w == W && p.tile_h == H && p.px == X) return launch_stats_t<W, H, X>(p, s);
#define PVG_DISPATCH_ONE_bwd(W, H, X) \
    if (p.tile_w == W && p.tile_h == H && p.px == X) return launch_bwd_t<W, H, X>(p, s);

void launch_composite(const Params &p, cudaStream_t s) { PVG_DISPATCH(fwd) }

void launch_composite_stats(const Params &p, cudaStream_t s) { PVG_DISPATCH(stats) }

void launch_composite_bwd(const Params &p, cudaStream_t s) { PVG_DISPATCH(bwd) }

}  // namespace pvg

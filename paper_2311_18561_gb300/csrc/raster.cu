// raster.cu -- per-tile compositing (stage c) and its adjoint (stage d1).
//
// Forward (Sec. 3.1, Eq. 3 with the depth / opacity channels of "flexible
// rendering"): one CTA per tile, one thread per pixel.  The tile's sorted
// list is walked front to back in batches of one record per thread; each
// batch is staged in shared memory (the conic pre-scaled by -log2(e) so
// the falloff is a single SFU ex2) and every pixel evaluates
//   alpha = min(0.99, o~ 2^(a' dx^2 + b' dx dy + c' dy^2)),
// skips alpha < 1/255, stops before a blend that would leave T < 1e-4,
// and accumulates C += c alpha T, D += z alpha T, O += alpha T.  The CTA
// leaves the list as soon as every pixel has stopped.
//
// Backward: the same CTA walks the list back to front from the last
// blended position of any pixel, rebuilding T_i = T_{i+1} / (1 - alpha_i)
// and the suffix sums S = sum_{j > i} x_j alpha_j T_j (+ T_final bg for
// colour), so dL/dalpha_i = T_i (gC.c_i + gD z_i + gO)
//                         - (gC.S_C + gD S_D + gO S_O) / (1 - alpha_i).
// Per-Gaussian image-space gradients (u, v, conic, o~, rgb, z) are reduced
// over the warp with shuffles (skipped when no lane contributed), then over
// the CTA in shared memory, and reach global memory with one atomic per
// (Gaussian, tile, component).
#include "pvg_internal.cuh"

namespace pvg {
namespace {

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_composite(Params P) {
    constexpr int BLOCK = TW * TH;
    __shared__ float4 s0[BLOCK];  // u, v, a', b'
    __shared__ float4 s1[BLOCK];  // c', o~, z, -
    __shared__ float4 s2[BLOCK];  // r, g, b, -
    const uint32_t tile = blockIdx.x;
    const int view = view_of_tile(P.views, P.n_views, tile);
    const ViewDesc &V = P.views[view];
    const uint32_t lt = tile - V.tile_base;
    const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
    const int tid = threadIdx.x;
    const int px = tx * TW + tid % TW, py = ty * TH + tid / TW;
    const bool inside = px < V.W && py < V.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 r = P.ranges[tile];

    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, O = 0.f;
    uint32_t last = 0, neval = r.y - r.x;
    bool done = !inside;
    for (uint32_t base = r.x; base < r.y; base += BLOCK) {
        if (__syncthreads_count(!done) == 0) break;
        const uint32_t j = base + tid;
        if (j < r.y) {
            const uint32_t m = P.pair_vals[j];
            const float4 a = P.rec[3 * (size_t)m], b = P.rec[3 * (size_t)m + 1], c = P.rec[3 * (size_t)m + 2];
            s0[tid] = make_float4(a.x, a.y, -0.5f * kLog2e * a.z, -kLog2e * a.w);
            s1[tid] = make_float4(-0.5f * kLog2e * b.x, b.y, b.z, 0.f);
            s2[tid] = c;
        }
        __syncthreads();
        if (!done) {
            const int cnt = (int)min((uint32_t)BLOCK, r.y - base);
            for (int k = 0; k < cnt; k++) {
                const float4 g = s0[k];
                const float4 h = s1[k];
                const float dx = __fsub_rn(fx, g.x), dy = __fsub_rn(fy, g.y);
                const float e = falloff_exp2(g.z, g.w, h.x, dx, dy);
                const float alpha = fminf(kAlphaCap, __fmul_rn(h.y, ex2_approx(e)));
                if (alpha < kAlphaMin) continue;
                const float Tn = __fmul_rn(T, __fsub_rn(1.0f, alpha));
                if (Tn < kTStop) {
                    done = true;
                    neval = base + k + 1 - r.x;
                    break;
                }
                const float w = __fmul_rn(alpha, T);
                const float4 col = s2[k];
                C0 = __fmaf_rn(col.x, w, C0);
                C1 = __fmaf_rn(col.y, w, C1);
                C2 = __fmaf_rn(col.z, w, C2);
                D = __fmaf_rn(h.z, w, D);
                O = __fadd_rn(O, w);
                T = Tn;
                last = base + k + 1 - r.x;
            }
        }
    }
    if (inside) {
        const size_t HW = (size_t)V.W * V.H, pix = (size_t)py * V.W + px;
        V.out_rgb[pix] = C0 + T * V.bg[0];
        V.out_rgb[HW + pix] = C1 + T * V.bg[1];
        V.out_rgb[2 * HW + pix] = C2 + T * V.bg[2];
        if (V.out_depth) V.out_depth[pix] = D;
        if (V.out_alpha) V.out_alpha[pix] = O;
        if (P.pix_T) {
            P.pix_T[V.pix_base + pix] = T;
            P.pix_last[V.pix_base + pix] = last;
            P.pix_neval[V.pix_base + pix] = neval;
        }
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_composite_bwd(Params P) {
    constexpr int BLOCK = TW * TH;
    constexpr int NG = 10;
    __shared__ float4 s0[BLOCK];
    __shared__ float4 s1[BLOCK];
    __shared__ float4 s2[BLOCK];
    __shared__ uint32_t s_m[BLOCK];
    __shared__ float s_acc[BLOCK * NG];
    __shared__ uint32_t s_maxlast;
    const uint32_t tile = blockIdx.x;
    const int view = view_of_tile(P.views, P.n_views, tile);
    const ViewDesc &V = P.views[view];
    const uint32_t lt = tile - V.tile_base;
    const int tx = (int)(lt % (uint32_t)V.tiles_x), ty = (int)(lt / (uint32_t)V.tiles_x);
    const int tid = threadIdx.x, lane = tid & 31;
    const int px = tx * TW + tid % TW, py = ty * TH + tid / TW;
    const bool inside = px < V.W && py < V.H;
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint2 r = P.ranges[tile];
    const size_t HW = (size_t)V.W * V.H, pix = (size_t)py * V.W + px;

    float T = 1.0f, gC[3] = {0.f, 0.f, 0.f}, gD = 0.f, gO = 0.f;
    uint32_t last = 0;
    if (inside) {
        T = P.pix_T[V.pix_base + pix];
        last = P.pix_last[V.pix_base + pix];
        if (V.dl_rgb) {
            gC[0] = V.dl_rgb[pix];
            gC[1] = V.dl_rgb[HW + pix];
            gC[2] = V.dl_rgb[2 * HW + pix];
        }
        if (V.dl_depth) gD = V.dl_depth[pix];
        if (V.dl_alpha) gO = V.dl_alpha[pix];
    }
    float sC0 = T * V.bg[0], sC1 = T * V.bg[1], sC2 = T * V.bg[2], sD = 0.f, sO = 0.f;
    if (tid == 0) s_maxlast = 0;
    __syncthreads();
    if (last) atomicMax(&s_maxlast, last);
    __syncthreads();
    const uint32_t n = s_maxlast;
    for (uint32_t end = r.x + n; end > r.x;) {
        const uint32_t start = end - r.x > (uint32_t)BLOCK ? end - BLOCK : r.x;
        const int cnt = (int)(end - start);
        __syncthreads();
        if (tid < cnt) {
            const uint32_t m = P.pair_vals[start + tid];
            const float4 a = P.rec[3 * (size_t)m], b = P.rec[3 * (size_t)m + 1], c = P.rec[3 * (size_t)m + 2];
            s0[tid] = make_float4(a.x, a.y, -0.5f * kLog2e * a.z, -kLog2e * a.w);
            s1[tid] = make_float4(-0.5f * kLog2e * b.x, b.y, b.z, 0.f);
            s2[tid] = c;
            s_m[tid] = m;
        }
        for (int k = tid; k < BLOCK * NG; k += BLOCK) s_acc[k] = 0.f;
        __syncthreads();
        for (int k = cnt - 1; k >= 0; k--) {
            const uint32_t pos = start + k - r.x;  // list position
            float gv[NG];
            bool contrib = inside && pos < last;
            if (contrib) {
                const float4 g = s0[k];
                const float4 h = s1[k];
                const float dx = __fsub_rn(fx, g.x), dy = __fsub_rn(fy, g.y);
                const float e = falloff_exp2(g.z, g.w, h.x, dx, dy);
                const float G = ex2_approx(e);
                const float raw = __fmul_rn(h.y, G);
                const float alpha = fminf(kAlphaCap, raw);
                contrib = alpha >= kAlphaMin;
                if (contrib) {
                    const float4 col = s2[k];
                    const float oma = 1.0f - alpha;
                    const float inv = 1.0f / oma;
                    const float Ti = T * inv;
                    const float w = alpha * Ti;
                    const float ga = Ti * (gC[0] * col.x + gC[1] * col.y + gC[2] * col.z + gD * h.z + gO) -
                                     inv * (gC[0] * sC0 + gC[1] * sC1 + gC[2] * sC2 + gD * sD + gO * sO);
                    gv[6] = gC[0] * w;
                    gv[7] = gC[1] * w;
                    gv[8] = gC[2] * w;
                    gv[9] = gD * w;
                    if (raw <= kAlphaCap) {
                        gv[5] = ga * G;
                        const float gpow = ga * alpha;       // d alpha / d power = alpha
                        const float gpl = gpow * 0.6931471805599453f;  // gpow / log2(e)
                        gv[2] = -0.5f * gpow * dx * dx;
                        gv[3] = -gpow * dx * dy;
                        gv[4] = -0.5f * gpow * dy * dy;
                        // a dx + b dy = -(2 a' dx + b' dy) / log2(e)
                        gv[0] = -gpl * (2.f * g.z * dx + g.w * dy);
                        gv[1] = -gpl * (g.w * dx + 2.f * h.x * dy);
                    } else {
                        gv[0] = gv[1] = gv[2] = gv[3] = gv[4] = gv[5] = 0.f;
                    }
                    sC0 += col.x * w;
                    sC1 += col.y * w;
                    sC2 += col.z * w;
                    sD += h.z * w;
                    sO += w;
                    T = Ti;
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                if (!contrib)
                    for (int c = 0; c < NG; c++) gv[c] = 0.f;
#pragma unroll
                for (int c = 0; c < NG; c++) {
                    float v = gv[c];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    gv[c] = v;
                }
                if (lane == 0)
                    for (int c = 0; c < NG; c++) atomicAdd(&s_acc[k * NG + c], gv[c]);
            }
        }
        __syncthreads();
        for (int q = tid; q < cnt * NG; q += BLOCK) {
            const float v = s_acc[q];
            if (v != 0.f) atomicAdd(&P.g2d[10 * (size_t)s_m[q / NG] + (q % NG)], v);
        }
        end = start;
    }
}

template <int TW, int TH>
void launch_fwd_t(const Params &p, cudaStream_t s) {
    if (p.total_tiles == 0) return;
    note_launch();
    k_composite<TW, TH><<<p.total_tiles, TW * TH, 0, s>>>(p);
}

template <int TW, int TH>
void launch_bwd_t(const Params &p, cudaStream_t s) {
    if (p.total_tiles == 0) return;
    note_launch();
    k_composite_bwd<TW, TH><<<p.total_tiles, TW * TH, 0, s>>>(p);
}

}  // namespace

bool composite_supported(int tw, int th) {
    return (tw == 8 && th == 8) || (tw == 16 && th == 8) || (tw == 16 && th == 16) || (tw == 32 && th == 8) ||
           (tw == 32 && th == 16);
}

#define PVG_TILE_DISPATCH(FN)                                   \
    if (p.tile_w == 16 && p.tile_h == 16) FN<16, 16>(p, s);     \
    else if (p.tile_w == 8 && p.tile_h == 8) FN<8, 8>(p, s);    \
    else if (p.tile_w == 16 && p.tile_h == 8) FN<16, 8>(p, s);  \
    else if (p.tile_w == 32 && p.tile_h == 8) FN<32, 8>(p, s);  \
    else if (p.tile_w == 32 && p.tile_h == 16) FN<32, 16>(p, s);

void launch_composite(const Params &p, cudaStream_t s) { PVG_TILE_DISPATCH(launch_fwd_t) }

void launch_composite_bwd(const Params &p, cudaStream_t s) { PVG_TILE_DISPATCH(launch_bwd_t) }

}  // namespace pvg

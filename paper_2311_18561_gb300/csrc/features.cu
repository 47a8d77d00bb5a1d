// features.cu -- extra composited channels: the velocity, staticness and
// semantic maps (the adjoint is in features_bwd.cu).
//
// Each channel is a per-point value x_i composited with the colour's
// weights w_i = T_i alpha_i and no background:
//   v_bar = v exp(-rho / 2), rho = beta / l (Eq. 10)   velocity map, 3 ch.
//   min(rho, 2)                                         staticness map, 1 ch.
//   the point's semantic vector                         semantic map, n_sem ch.
// (Sec. 4: dynamic-element analysis and semantic rendering.)
//
// A pass of its own over the per-tile lists of the colour pass, so the
// colour compositor keeps its registers when no channel is asked for: one
// CTA of up to 256 threads per tile, one pixel per thread (tiles larger
// than the CTA are covered in rounds), the list staged in batches of kFB
// entries: the record's blending terms and the channel values, padded to
// float4 groups.  Alpha comes from record_terms / falloff_exp2 / ex2 with
// the colour pass's roundings, so the weights are the colour pass's bit
// for bit.
#include "features_common.cuh"

namespace pvg {

int feat_count(int mask, int n_sem) {
    return ((mask & kFeatVbar) ? 3 : 0) + ((mask & kFeatRho) ? 1 : 0) + ((mask & kFeatSem) ? n_sem : 0);
}

namespace {

template <int NG>
__global__ void __launch_bounds__(kFeatBlock) k_composite_feat(Params P) {
    pdl_enter();
    __shared__ float4 s0[kFB];
    __shared__ float2 s1[kFB];
    __shared__ float4 sf[kFB * NG];
    constexpr int kFPX = kFwdFPX;
    const int rounds = feat_rounds<kFPX>(P);
    constexpr uint32_t ALL = (1u << kFPX) - 1u;
    for (int round = 0; round < rounds; round++) {
        const FeatPixels<kFPX> Q = feat_pixels<kFPX>(P, round);
        const ViewDesc &V = *Q.V;
        const float fx = (float)Q.px + 0.5f;
        float fy[kFPX], T[kFPX], acc[kFPX][4 * NG];
        uint32_t done = 0;
#pragma unroll
        for (int p = 0; p < kFPX; p++) {
            fy[p] = (float)(Q.py0 + p) + 0.5f;
            T[p] = 1.0f;
#pragma unroll
            for (int c = 0; c < 4 * NG; c++) acc[p][c] = 0.f;
            if (!Q.inside[p]) done |= 1u << p;
        }
        for (uint32_t base = Q.r.x; base < Q.r.y; base += kFB) {
            if (__syncthreads_count(done != ALL) == 0) break;
            const int cnt = (int)min((uint32_t)kFB, Q.r.y - base);
            for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
                const uint32_t m = P.pair_vals[base + k];
                float4 a, c;
                float2 b;
                record_terms(P.rec, m, a, b, c);
                s0[k] = a;
                s1[k] = b;
                stage_feat<NG>(V, P.sgid[m], P.feat_mask, reinterpret_cast<float *>(&sf[k * NG]));
            }
            __syncthreads();
            for (int k = 0; k < cnt && done != ALL; k++) {
                const float4 g = s0[k];
                const float2 q = s1[k];
                const float dx = __fsub_rn(fx, g.x);
                const FalloffColumn fc = falloff_column(g.z, g.w, dx);
                float w[kFPX];
                bool any = false;
#pragma unroll
                for (int p = 0; p < kFPX; p++) {
                    w[p] = 0.f;
                    if (done & (1u << p)) continue;
                    const float dy = __fsub_rn(fy[p], g.y);
                    const float e = falloff_exp2(fc, q.x, dy);
                    const float raw = __fmul_rn(q.y, ex2_approx(e));
                    if (!(raw >= kAlphaMin)) continue;  // = min(cap, raw) < 1/255, cap > 1/255
                    const float alpha = fminf(kAlphaCap, raw);
                    const float wv = __fmul_rn(alpha, T[p]);
                    const float Tn = __fsub_rn(T[p], wv);
                    if (Tn < kTStop) {
                        done |= 1u << p;
                        continue;
                    }
                    w[p] = wv;
                    T[p] = Tn;
                    any = true;
                }
                if (!any) continue;
                // a pixel that did not blend adds a zero weight: its sums are unchanged
#pragma unroll
                for (int gi = 0; gi < NG; gi++) {
                    const float4 f = sf[k * NG + gi];
#pragma unroll
                    for (int p = 0; p < kFPX; p++) {
                        acc[p][4 * gi] = __fmaf_rn(f.x, w[p], acc[p][4 * gi]);
                        acc[p][4 * gi + 1] = __fmaf_rn(f.y, w[p], acc[p][4 * gi + 1]);
                        acc[p][4 * gi + 2] = __fmaf_rn(f.z, w[p], acc[p][4 * gi + 2]);
                        acc[p][4 * gi + 3] = __fmaf_rn(f.w, w[p], acc[p][4 * gi + 3]);
                    }
                }
            }
        }
        __syncthreads();  // the next round restages
        const size_t HW = (size_t)V.W * V.H;
#pragma unroll
        for (int p = 0; p < kFPX; p++) {
            if (!Q.inside[p]) continue;
            const size_t pix = (size_t)(Q.py0 + p) * V.W + Q.px;
#pragma unroll
            for (int c = 0; c < 4 * NG; c++)
                if (c < P.n_feat) V.out_feat[c * HW + pix] = acc[p][c];
        }
    }
}

}  // namespace

void launch_composite_feat(const Params &p, cudaStream_t s) {
    if (p.total_tiles == 0 || p.n_feat <= 0) return;
    note_launch();
    const int block = min(kFeatBlock, p.tile_w * p.tile_h / kFwdFPX);
    switch ((p.n_feat + 3) / 4) {
        case 1: pdl_launch(k_composite_feat<1>, p.total_tiles, block, 0, s, p); break;
        case 2: pdl_launch(k_composite_feat<2>, p.total_tiles, block, 0, s, p); break;
        case 3: pdl_launch(k_composite_feat<3>, p.total_tiles, block, 0, s, p); break;
        case 4: pdl_launch(k_composite_feat<4>, p.total_tiles, block, 0, s, p); break;
        case 5: pdl_launch(k_composite_feat<5>, p.total_tiles, block, 0, s, p); break;
        case 6: pdl_launch(k_composite_feat<6>, p.total_tiles, block, 0, s, p); break;
        case 7: pdl_launch(k_composite_feat<7>, p.total_tiles, block, 0, s, p); break;
        case 8: pdl_launch(k_composite_feat<8>, p.total_tiles, block, 0, s, p); break;
        default: pdl_launch(k_composite_feat<9>, p.total_tiles, block, 0, s, p); break;
    }
}

}  // namespace pvg

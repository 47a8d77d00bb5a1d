// features_bwd.cu -- adjoint of the extra composited channels.
//
// The walk of the colour adjoint, back to front from the pixel's final
// transmittance and last blended position, two vertically adjacent pixels
// per thread (their terms are summed before the warp reduction).  With X_i = gF.x_i and the
// scalar suffix sum S_i = sum_{j > i} X_j w_j,
//   dL/dalpha_i (channels) = T_i X_i - S_i / (1 - alpha_i),
// whose effect on (u, v, conic, o~) is added to the image-space gradient
// buffer in the colour adjoint's moment form, and dL/dx_i = sum gF w_i is
// accumulated per visible point.  k_feat_param_bwd then maps dL/dx to v,
// beta, l and the semantic vectors.  Blend decisions use the forward's
// explicitly rounded alpha.
#include "features_common.cuh"

namespace pvg {
namespace {

// Sum over the warp of N terms (N a power of two <= 32): afterwards lane L
// holds the total of term L & (N - 1).  Transposing butterfly: N - 1
// shuffles, then 5 - log2(N) to fold the lane groups.
template <int S, int N>
__device__ __forceinline__ void transpose_level(float (&a)[N], int lane) {
    if constexpr (S >= 1) {
        const bool hi = lane & S;
#pragma unroll
        for (int i = 0; i < S; i++) {
            const float send = hi ? a[i] : a[i + S];
            a[i] = (hi ? a[i + S] : a[i]) + __shfl_xor_sync(0xffffffffu, send, S);
        }
        transpose_level<S / 2, N>(a, lane);
    }
}

template <int N>
__device__ __forceinline__ float warp_transpose_sum(float (&a)[N]) {
    const int lane = threadIdx.x & 31;
    transpose_level<N / 2, N>(a, lane);
    float v = a[0];
#pragma unroll
    for (int s = N; s < 32; s <<= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    return v;
}

__host__ __device__ constexpr int pow2_at_least(int n) { return n <= 1 ? 1 : 2 * pow2_at_least((n + 1) / 2); }

// adds terms [B, B + N) of gv (N a power of two) into s_acc[k * NT + term]
template <int NT, int B, int N>
__device__ __forceinline__ void reduce_chunk(const float (&gv)[NT], float *s_acc, int k) {
    float a[N];
#pragma unroll
    for (int i = 0; i < N; i++) a[i] = B + i < NT ? gv[B + i] : 0.f;
    const float v = warp_transpose_sum<N>(a);
    const int lane = threadIdx.x & 31, term = B + (lane & (N - 1));
    if (lane < N && term < NT && v != 0.f) atomicAdd(&s_acc[k * NT + term], v);
}

template <int NG>
__global__ void __launch_bounds__(kFeatBlock) k_composite_feat_bwd(Params P) {
    pdl_enter();
    constexpr int F4 = 4 * NG;
    constexpr int NT = 6 + F4;  // moments x, y, xx, xy, yy; opacity; channels
    __shared__ float4 s0[kFB];
    __shared__ float2 s1[kFB];
    __shared__ float4 sf[kFB * NG];
    __shared__ uint32_t s_m[kFB];
    __shared__ float s_acc[kFB * NT];
    __shared__ uint32_t s_maxlast;
    constexpr int kFPX = kBwdFPX;
    const int rounds = feat_rounds<kFPX>(P);
    const int tid = threadIdx.x;
    for (int round = 0; round < rounds; round++) {
        const FeatPixels<kFPX> Q = feat_pixels<kFPX>(P, round);
        const ViewDesc &V = *Q.V;
        const float fx = (float)Q.px + 0.5f;
        float fy[kFPX], T[kFPX], S[kFPX], gF[kFPX][F4];  // S: suffix sum of X_j w_j (no background)
        uint32_t last[kFPX], maxlast = 0;
#pragma unroll
        for (int p = 0; p < kFPX; p++) {
            fy[p] = (float)(Q.py0 + p) + 0.5f;
            T[p] = 1.0f;
            S[p] = 0.f;
            last[p] = 0;
#pragma unroll
            for (int c = 0; c < F4; c++) gF[p][c] = 0.f;
            if (Q.inside[p] && V.dl_feat) {
                const size_t HW = (size_t)V.W * V.H, pix = (size_t)(Q.py0 + p) * V.W + Q.px;
                T[p] = P.pix_T[V.pix_base + pix];
                last[p] = P.pix_last[V.pix_base + pix];
#pragma unroll
                for (int c = 0; c < F4; c++)
                    if (c < P.n_feat) gF[p][c] = V.dl_feat[c * HW + pix];
            }
            maxlast = max(maxlast, last[p]);
        }
        __syncthreads();  // previous round done with the shared arrays
        if (tid == 0) s_maxlast = 0;
        __syncthreads();
        if (maxlast) atomicMax(&s_maxlast, maxlast);
        __syncthreads();
        const uint32_t n = s_maxlast;
        // gv: an entry's terms over this thread's pixels, zero between
        // entries (reset after each warp reduction); the conic moments as
        // in the colour adjoint (sum gpow in A0, expanded with the shared dx)
        float gv[NT];
#pragma unroll
        for (int c = 0; c < NT; c++) gv[c] = 0.f;
        float A0 = 0.f;
        for (uint32_t end = Q.r.x + n; end > Q.r.x;) {
            const uint32_t start = end - Q.r.x > (uint32_t)kFB ? end - kFB : Q.r.x;
            const int cnt = (int)(end - start);
            __syncthreads();
            for (int k = tid; k < cnt; k += blockDim.x) {
                const uint32_t m = P.pair_vals[start + k];
                float4 a, c;
                float2 b;
                record_terms(P.rec, m, a, b, c);
                s0[k] = a;
                s1[k] = b;
                s_m[k] = m;
                stage_feat<NG>(V, P.sgid[m], P.feat_mask, reinterpret_cast<float *>(&sf[k * NG]));
            }
            for (int k = tid; k < kFB * NT; k += blockDim.x) s_acc[k] = 0.f;
            __syncthreads();
            for (int k = cnt - 1; k >= 0; k--) {
                const uint32_t pos = start + k - Q.r.x;
                bool contrib = false;
                const float4 g = s0[k];
                const float2 q = s1[k];
                const float dx = __fsub_rn(fx, g.x);
                const FalloffColumn fc = falloff_column(g.z, g.w, dx);
#pragma unroll
                for (int p = 0; p < kFPX; p++) {
                    if (pos >= last[p]) continue;
                    const float dy = __fsub_rn(fy[p], g.y);
                    const float e = falloff_exp2(fc, q.x, dy);
                    const float G = ex2_approx(e);
                    const float raw = __fmul_rn(q.y, G);
                    if (!(raw >= kAlphaMin)) continue;  // = min(cap, raw) < 1/255, cap > 1/255
                    const float alpha = fminf(kAlphaCap, raw);
                    contrib = true;
                    const float inv = rcp_approx(1.0f - alpha);
                    const float Ti = T[p] * inv;
                    const float w = alpha * Ti;
                    float X = 0.f;
#pragma unroll
                    for (int gi = 0; gi < NG; gi++) {
                        const float4 f = sf[k * NG + gi];
                        const float fv[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const int c = 4 * gi + j;
                            X += gF[p][c] * fv[j];
                            gv[6 + c] += gF[p][c] * w;
                        }
                    }
                    if (raw <= kAlphaCap) {
                        const float ga = Ti * X - inv * S[p];
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
                if (__any_sync(0xffffffffu, contrib)) {
                    gv[0] = dx * A0;
                    gv[2] = dx * gv[0];
                    gv[3] = dx * gv[1];
                    constexpr int N0 = NT >= 32 ? 32 : pow2_at_least(NT);
                    reduce_chunk<NT, 0, N0>(gv, s_acc, k);
                    if constexpr (NT > 32) reduce_chunk<NT, 32, pow2_at_least(NT - 32)>(gv, s_acc, k);
#pragma unroll
                    for (int c = 0; c < NT; c++) gv[c] = 0.f;
                    A0 = 0.f;
                }
            }
            __syncthreads();
            // image-space terms from the moments (as in the colour adjoint)
            // and the channel gradients of each staged point
            for (int k = tid; k < cnt; k += blockDim.x) {
                const float *a = &s_acc[k * NT];
                const float ap = s0[k].z, bp = s0[k].w, cp = s1[k].x;
                float gt[6];
                gt[0] = -0.6931471805599453f * (2.f * ap * a[0] + bp * a[1]);
                gt[1] = -0.6931471805599453f * (bp * a[0] + 2.f * cp * a[1]);
                gt[2] = -0.5f * a[2];
                gt[3] = -a[3];
                gt[4] = -0.5f * a[4];
                gt[5] = a[5];
                float *dst = &P.g2d[10 * (size_t)s_m[k]];
#pragma unroll
                for (int c = 0; c < 6; c++)
                    if (gt[c] != 0.f) atomicAdd(dst + c, gt[c]);
                float *gf = &P.gfeat[(size_t)s_m[k] * P.n_feat];
                for (int c = 0; c < P.n_feat; c++)
                    if (a[6 + c] != 0.f) atomicAdd(gf + c, a[6 + c]);
            }
            end = start;
        }
    }
}

// dL/d(channel values) of each visible item -> v, beta, l, semantics
__global__ void k_feat_param_bwd(Params P) {
    pdl_enter();
    const uint32_t M = P.counters[0];
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const uint32_t gid = P.sgid[m];
        const ViewDesc &V = P.views[view_of_item(P.views, P.n_views, gid)];
        const uint32_t i = gid - V.item_base;
        const float *gf = &P.gfeat[(size_t)m * P.n_feat];
        const float beta = V.beta[i], l = V.period[i];
        const float rho = __fdiv_rn(beta, l);
        float grho = 0.f;  // dL/drho
        int c = 0;
        if (P.feat_mask & kFeatVbar) {
            // v_bar = v exp(-rho / 2): d/dv = exp(-rho / 2), d/drho = -v_bar / 2
            const float w = expf(-0.5f * rho);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (V.g_vel && gf[k] != 0.f) atomicAdd(V.g_vel + 3 * (size_t)i + k, gf[k] * w);
                grho -= 0.5f * gf[k] * V.vel[3 * (size_t)i + k] * w;
            }
            c = 3;
        }
        if (P.feat_mask & kFeatRho) {
            if (rho < 2.0f) grho += gf[c];
            c++;
        }
        if (grho != 0.f) {
            // rho = beta / l
            if (V.g_beta) atomicAdd(V.g_beta + i, grho / l);
            if (V.g_period) atomicAdd(V.g_period + i, -grho * beta / (l * l));
        }
        if ((P.feat_mask & kFeatSem) && V.g_sem)
            for (int k = 0; k < V.n_sem; k++)
                if (gf[c + k] != 0.f) atomicAdd(V.g_sem + (size_t)i * V.n_sem + k, gf[c + k]);
    }
}

}  // namespace

void launch_composite_feat_bwd(const Params &p, cudaStream_t s) {
    if (p.total_tiles == 0 || p.n_feat <= 0) return;
    note_launch();
    const int block = min(kFeatBlock, p.tile_w * p.tile_h / kBwdFPX);
    switch ((p.n_feat + 3) / 4) {
        case 1: pdl_launch(k_composite_feat_bwd<1>, p.total_tiles, block, 0, s, p); break;
        case 2: pdl_launch(k_composite_feat_bwd<2>, p.total_tiles, block, 0, s, p); break;
        case 3: pdl_launch(k_composite_feat_bwd<3>, p.total_tiles, block, 0, s, p); break;
        case 4: pdl_launch(k_composite_feat_bwd<4>, p.total_tiles, block, 0, s, p); break;
        case 5: pdl_launch(k_composite_feat_bwd<5>, p.total_tiles, block, 0, s, p); break;
        case 6: pdl_launch(k_composite_feat_bwd<6>, p.total_tiles, block, 0, s, p); break;
        case 7: pdl_launch(k_composite_feat_bwd<7>, p.total_tiles, block, 0, s, p); break;
        case 8: pdl_launch(k_composite_feat_bwd<8>, p.total_tiles, block, 0, s, p); break;
        default: pdl_launch(k_composite_feat_bwd<9>, p.total_tiles, block, 0, s, p); break;
    }
}

void launch_feat_param_bwd(const Params &p, cudaStream_t s) {
    if (p.n_items == 0 || p.n_feat <= 0) return;
    note_launch();
    pdl_launch(k_feat_param_bwd, 4 * device_sm_count(), 256, 0, s, p);
}

}  // namespace pvg

// features_common.cuh -- staging of the extra channels shared by their
// compositing pass (features.cu) and its adjoint (features_bwd.cu).
#pragma once
#include "pvg_internal.cuh"

namespace pvg {
namespace {

constexpr int kFB = 128;       // list entries staged per batch
constexpr int kFeatBlock = 256;  // threads per CTA (fewer for small tiles)

// channel values of item gid into dst[0 .. 4 NG) (zero padded)
template <int NG>
__device__ __forceinline__ void stage_feat(const ViewDesc &V, uint32_t gid, int mask, float *dst) {
#pragma unroll
    for (int c = 0; c < 4 * NG; c++) dst[c] = 0.f;
    const uint32_t i = gid - V.item_base;
    const float beta = V.beta[i], l = V.period[i];
    const float rho = __fdiv_rn(beta, l);
    int c = 0;
    if (mask & kFeatVbar) {
        const float w = expf(-0.5f * rho);
        dst[0] = V.vel[3 * (size_t)i] * w;
        dst[1] = V.vel[3 * (size_t)i + 1] * w;
        dst[2] = V.vel[3 * (size_t)i + 2] * w;
        c = 3;
    }
    if (mask & kFeatRho) dst[c++] = fminf(rho, 2.0f);
    if (mask & kFeatSem)
        for (int k = 0; k < V.n_sem; k++) dst[c + k] = V.sem[(size_t)i * V.n_sem + k];
}

// The FPX vertically adjacent pixels (column px, rows py0 .. py0 + FPX - 1)
// that thread threadIdx.x handles in `round` of its tile (pixel groups in
// row-major order), and the tile's list range.
template <int FPX>
struct FeatPixels {
    const ViewDesc *V;
    int px, py0;
    bool inside[FPX];
    uint2 r;
};

template <int FPX>
__device__ __forceinline__ FeatPixels<FPX> feat_pixels(const Params &P, int round) {
    FeatPixels<FPX> q;
    const uint32_t tile = P.tile_order ? P.tile_order[blockIdx.x] : blockIdx.x;
    q.V = &P.views[view_of_tile(P.views, P.n_views, tile)];
    const uint32_t lt = tile - q.V->tile_base;
    const int tx = (int)(lt % (uint32_t)q.V->tiles_x), ty = (int)(lt / (uint32_t)q.V->tiles_x);
    const int k = round * (int)blockDim.x + (int)threadIdx.x;  // pixel group of the tile
    const bool in_tile = k < P.tile_w * (P.tile_h / FPX);
    q.px = tx * P.tile_w + k % P.tile_w;
    q.py0 = ty * P.tile_h + (k / P.tile_w) * FPX;
#pragma unroll
    for (int p = 0; p < FPX; p++) q.inside[p] = in_tile && q.px < q.V->W && q.py0 + p < q.V->H;
    q.r = P.ranges[tile];
    return q;
}

template <int FPX>
__device__ __forceinline__ int feat_rounds(const Params &P) {
    const int groups = P.tile_w * (P.tile_h / FPX);
    return (groups + (int)blockDim.x - 1) / (int)blockDim.x;
}

// pixels per thread: the channel compositor keeps one (its per-pixel
// accumulators are many), its adjoint two (to amortise its warp reduction)
constexpr int kFwdFPX = 1, kBwdFPX = 2;

}  // namespace
}  // namespace pvg

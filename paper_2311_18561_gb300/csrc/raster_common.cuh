// raster_common.cuh -- tile geometry and record staging shared by the
// compositor (raster.cu) and its adjoint (raster_bwd.cu).
#pragma once
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


}  // namespace
}  // namespace pvg

// Supported (tile width, tile height, pixels per thread) combinations.
#define PVG_TILE_CONFIGS(X)                                                                               \
    X(16, 16, 1) X(16, 16, 2) X(16, 16, 4) X(8, 8, 1) X(8, 8, 2) X(16, 8, 1) X(16, 8, 2) X(32, 8, 1)    \
    X(32, 16, 1) X(32, 16, 2) X(32, 16, 4) X(32, 32, 4) X(16, 32, 4)

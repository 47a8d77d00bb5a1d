// pvg_internal.cuh -- device-side data layout shared by the kernels of the
// PVG rasterizer (sm_103a).  Not part of the ABI.
//
// Layout in HBM (per forward pass):
//   items     (view, Gaussian) pairs, gid = item_base[view] + i      [NV]
//   visible   depth-sorted visible items, position m                 [M]
//     sgid[m]   gid of the m-th visible item in (depth, gid) order
//     rec[m]    3 x float4 record read by the compositor:
//               (u, v, conic a, conic b) (conic c, o~, z, hx) (r, g, b, hy)
//               hx, hy: guarded half extents of the footprint box in pixels
//     rowtab[m] tiles of the footprint ellipse row by row, packed (items
//               of <= 8 rows x 255 columns)
//     ell[m]    2 x float4: the footprint ellipse in tile-row form (the
//               other items)
//     rect[m]   tile rectangle, packed (tx0 | ty0 << 16, tx1 | ty1 << 16)
//     vis_cnt[m] tiles of the rectangle that the footprint ellipse meets
//   pairs     (tile, m) pairs sorted by (tile, depth, gid)             [K]
//   ranges    [start, end) into the pairs per global tile             [tiles]
//   pixels    final transmittance and last blended list position      [sum HW]
#pragma once
#include <cstdint>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/pvg.h"

namespace pvg {

constexpr float kAlphaMin = 1.0f / 255.0f;  // skip gate
constexpr float kAlphaCap = 0.99f;          // alpha cap
// an entry whose o~ is at most this never reaches the cap: its alpha
// o~ 2^e (e <= 0 up to one rounding) stays below kAlphaCap, so the
// compositors take min(cap, .) only for the rare entries above it
constexpr float kUncappedOpacity = 0.9899f;
constexpr float kTStop = 1e-4f;             // transmittance stop
constexpr float kFarRow = 1e30f;            // row coordinate of a pixel that is done (packed compositor)
constexpr float kLog2e = 1.4426950408889634f;  // log2(e): e^x = 2^(x log2 e)
constexpr int kMaxViewsPerCall = 4096;

// Per-view description, uploaded once per call.
struct ViewDesc {
    float R[9], T[3];  // world->camera
    float fx, fy, cx, cy;
    float t, znear;
    float dt;          // temporal-smoothing shift (0: plain render)
    float bg[3];
    float campos[3];   // camera centre in world space, -R^T T
    float limx, limy;  // J clamp on x/z and y/z
    int32_t W, H;
    int32_t tiles_x, tiles_y;
    uint32_t tile_base;  // first global tile id of this view
    uint32_t pix_base;   // first pixel of this view in the per-pixel state
    uint32_t item_base;  // first gid of this view
    uint32_t n;          // Gaussians of this view's scene
    int32_t sh_degree;
    int32_t pad0;
    // scene
    const float *mu, *vel, *tau, *beta, *period, *scale, *quat, *opac, *sh;
    const float *sky;        // [6][R][R][3] cube map or NULL (constant bg)
    const float *sky_jitter; // [2][H][W] pixel offsets of the sky rays or NULL
    int32_t sky_res, pad1;
    const float *sem;        // [n][n_sem] semantic vectors or NULL
    int32_t n_sem, pad2;
    // outputs
    float *out_rgb, *out_depth, *out_alpha;
    float *out_feat;         // [F][H][W] extra channels or NULL
    // backward inputs / outputs
    const float *dl_rgb, *dl_depth, *dl_alpha, *dl_feat;
    float *g_mu, *g_vel, *g_tau, *g_beta, *g_period, *g_scale, *g_quat, *g_opac, *g_sh;
    float *g_sky, *g_sem;
};

// extra composited channels (bit mask): v_bar (3), min(rho, 2) (1), semantics (n_sem)
constexpr int kFeatVbar = 1, kFeatRho = 2, kFeatSem = 4;
constexpr int kMaxSem = 32;
constexpr int kMaxFeatGroups = 9;  // channels padded to float4 groups: 3 + 1 + 32 = 36

// Launch-wide parameters.
struct Params {
    const ViewDesc *views;
    int32_t n_views;
    int32_t sh_degree;       // of the call's scene (kernels are specialised on it)
    int32_t tile_w, tile_h;
    int32_t px;              // pixels per compositing thread
    float dilation;
    uint32_t n_items;        // NV
    uint32_t total_tiles;
    uint32_t total_pix;
    uint32_t pair_capacity;
    // device counters: [0] visible M, [1] pairs K, [2] overflow flag, [3] the
    // per-item adjoint's chunk ticket
    uint32_t *counters;
    // per-item scratch
    uint32_t *item_cnt;      // [NV] tiles touched (0 = invisible)
    uint32_t *item_zkey;     // [NV] depth bits (valid where item_cnt > 0)
    float4 *proj;            // [NV * 4] projection of each visible item (pass 1 -> pass 2)
    // visible
    uint32_t *sgid;          // [M]
    uint32_t *inv;           // [NV] depth position of each item, 0xffffffff if not visible
    uint32_t *szkey;         // [M]
    float4 *rec;             // [M*3]
    float4 *ell;             // [M*2] footprint ellipses (store_ellipse)
    uint4 *rowtab;           // [M] packed tile-row spans (has_row_table)
    uint2 *rect;             // [M]
    uint32_t *vis_cnt;       // [M] tiles per visible item
    uint32_t *vis_off;       // [M] first pair position of the item
    uint32_t *chunk_start;   // [K / 2048 + 1] first item of each pair chunk
    // pairs
    uint32_t *pair_keys;     // [K] tile ids (sorted in place via ping-pong)
    uint32_t *pair_vals;     // [K]
    uint2 *ranges;           // [total_tiles]
    uint32_t *tile_order;    // [total_tiles] tiles by decreasing list length (compositor launch order)
    uint32_t *tile_walk;     // [total_tiles] forward: largest pixel_last of the tile (the adjoint's walk)
    float *pix_T;            // [sum HW]
    uint32_t *pix_last;      // [sum HW] list position after the last blend
    uint32_t *pix_neval;     // [2][sum HW] stats pass: in-footprint entries up to the stop, and blended ones
    // backward
    float *g2d;              // [M*10] image-space gradients by depth position (u, v, conic a b c,
                             // o~, colour with the forward's clamp applied, z)
    int32_t aux;             // backward: some view has depth / opacity-map gradients or a sky map
    // extra channels
    int32_t feat_mask;       // kFeat* bits (0: none)
    int32_t n_feat;          // F
    float *gfeat;            // [M*F] dL/d(channel value) per visible item
};

// view of a global item / tile by binary search over the per-view bases
__device__ __forceinline__ int view_of_item(const ViewDesc *views, int nv, uint32_t gid) {
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].item_base <= gid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int view_of_tile(const ViewDesc *views, int nv, uint32_t tile) {
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// 2^x on the SFU (PTX ex2.approx.ftz.f32)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The compositor's terms of record m: (u, v, a', b'), (c', o~), (r, g, b, z)
// with the conic pre-scaled, (a', b', c') = -log2(e) (a/2, b, c/2).  Every
// kernel that blends takes its alpha from these terms, so the blending
// weights agree bit for bit across kernels.
// The row coefficient c' is kept at most -kMinRowCoef: a pixel moved to
// the far row (kFarRow, packed compositor) then always gets an exponent of
// -inf (alpha 0, never blends again), whatever its column; the bound only
// touches conics with c < 1.4e-20 px^-2 (a footprint over 1e10 pixels
// tall), and a NaN coefficient stays NaN.
constexpr float kMinRowCoef = 1e-20f;

__device__ __forceinline__ void record_terms(const float4 *rec, uint32_t m, float4 &s0, float2 &s1, float4 &s2) {
    const float4 a = rec[3 * (size_t)m], b = rec[3 * (size_t)m + 1], c = rec[3 * (size_t)m + 2];
    s0 = make_float4(a.x, a.y, -0.5f * kLog2e * a.z, -kLog2e * a.w);
    const float cp = -0.5f * kLog2e * b.x;
    s1 = make_float2(cp > -kMinRowCoef ? -kMinRowCoef : cp, b.y);
    s2 = make_float4(c.x, c.y, c.z, b.z);
}

// Kahan's difference of products a*b - c*d, accurate to a few ulp.
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

// Footprint of a record in one tile row.  The compositor blends a record at
// a pixel only where o~ G >= 1/255, i.e. where the pixel centre's offset d
// from (u, v) lies in the ellipse a dx^2 + 2 b dx dy + c dy^2 <= Q with
// Q = 2 ln(255 o~) (conic a b c).  Of the bounding rectangle's tiles, those
// of row ty whose pixel centres can reach that ellipse are the columns
// [c0, c1) returned here, computed for the widened level Q' = 1.01 Q + 1e-4
// and pixel-centre bands widened by 0.1 px: the widening covers the
// rounding of the compositor's own evaluation of the quadratic form, which
// for conics with (a + c)^2 > 1e4 (ac - b^2) (needle footprints, relative
// error above 0.4 %) is not assured: there the whole rectangle row is kept.
//   In a band of offsets y in [lo, hi] the left edge of the ellipse,
// x(y) = (-b y - sqrt(a Q' - D y^2)) / a with D = ac - b^2, is convex with
// its minimum at y_l = b sqrt(Q' / (c D)) (the right edge is concave with
// its maximum at -y_l), so the band's span is the edges evaluated at those
// points clamped into the band.  The tile count of a record (finalize pass)
// and the pair expansion both call this on the same stored floats, with
// explicitly rounded or hardware-approximate operations only, so the two
// agree bit for bit; the approximations' relative errors (a few ulp) are
// far inside the widening.
struct FootprintEllipse {
    float u, v, b, ia, aQ, D, ym, yl;
    bool exact;  // false: keep whole rectangle rows
};

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ FootprintEllipse footprint_ellipse(float u, float v, float a, float b, float c,
                                                              float ot) {
    // Q' = 1.01 * 2 ln(255 o~) + 1e-4 = 1.01 * 2 ln(2) log2(255 o~) + 1e-4
    const float Q = fmaxf(__fmul_rn(2.0f * 0.6931471805599453f, lg2_approx(__fmul_rn(255.0f, ot))), 0.0f);
    const float Qp = __fadd_rn(__fmul_rn(1.01f, Q), 1e-4f);
    FootprintEllipse E;
    E.u = u; E.v = v; E.b = b;
    E.D = diff_of_products(a, c, b, b);
    const float tr = __fadd_rn(a, c);
    E.exact = E.D > 0.0f && a > 0.0f && c > 0.0f && __fmul_rn(tr, tr) <= __fmul_rn(1e4f, E.D);
    const float iD = E.exact ? __frcp_rn(E.D) : 0.0f;
    E.ia = E.exact ? __frcp_rn(a) : 0.0f;
    E.exact = E.exact && E.ia > 0.0f;  // the stored form's flag
    if (!E.exact) E.ia = 0.0f;
    E.aQ = __fmul_rn(a, Qp);
    E.ym = sqrt_approx(__fmul_rn(E.aQ, iD));
    E.yl = __fmul_rn(b, sqrt_approx(__fmul_rn(Qp, __fmul_rn(iD, E.exact ? __frcp_rn(c) : 0.0f))));
    return E;
}

// The ellipse as stored per visible item without a row table (the finalize
// pass writes it and counts the tiles with the values it writes; the pair
// expansion reads it back), !exact encoded as ia = 0.
__device__ __forceinline__ void store_ellipse(float4 *ell, uint32_t m, const FootprintEllipse &E) {
    ell[2 * (size_t)m] = make_float4(E.u, E.v, E.b, E.ia);
    ell[2 * (size_t)m + 1] = make_float4(E.aQ, E.D, E.ym, E.yl);
}

__device__ __forceinline__ FootprintEllipse load_ellipse(const float4 *ell, uint32_t m) {
    const float4 p = ell[2 * (size_t)m], q = ell[2 * (size_t)m + 1];
    FootprintEllipse E;
    E.u = p.x; E.v = p.y; E.b = p.z; E.ia = p.w;
    E.aQ = q.x; E.D = q.y; E.ym = q.z; E.yl = q.w;
    E.exact = p.w > 0.0f;
    return E;
}

// Row table of an item whose rectangle has at most kTabRows rows and 255
// columns: row i's (c0 - tx0) | (c1 - c0) << 8 in bits [16 (i & 1), +16) of
// word i >> 1.
constexpr uint32_t kTabRows = 8;

__device__ __forceinline__ bool has_row_table(uint32_t tx0, uint32_t ty0, uint32_t tx1, uint32_t ty1) {
    return ty1 - ty0 <= kTabRows && tx1 - tx0 <= 255u;
}

// Pixel-centre columns [p0, p1] that the ellipse (widened by kPad) reaches
// within the pixel rows [ylo, yhi) (integer-valued floats); false when the
// rows miss it.  Only for E.exact.
__device__ __forceinline__ bool footprint_span(const FootprintEllipse &E, float ylo, float yhi, float &p0,
                                               float &p1) {
    constexpr float kPad = 0.1f;
    // offsets of the rows' pixel centres, py + 0.5 - v for py in [ylo, yhi)
    const float lo = fmaxf(__fsub_rn(ylo + (0.5f - kPad), E.v), -E.ym);
    const float hi = fminf(__fsub_rn(yhi - (0.5f - kPad), E.v), E.ym);
    if (!(lo <= hi)) return false;
    const float yl = fminf(fmaxf(E.yl, lo), hi);
    const float yr = fminf(fmaxf(-E.yl, lo), hi);
    const float wl = sqrt_approx(fmaxf(__fsub_rn(E.aQ, __fmul_rn(E.D, __fmul_rn(yl, yl))), 0.0f));
    const float wr = sqrt_approx(fmaxf(__fsub_rn(E.aQ, __fmul_rn(E.D, __fmul_rn(yr, yr))), 0.0f));
    const float xl = __fmul_rn(__fsub_rn(__fmul_rn(-E.b, yl), wl), E.ia);
    const float xr = __fmul_rn(__fadd_rn(__fmul_rn(-E.b, yr), wr), E.ia);
    // pixel columns px with px + 0.5 - u in [xl - pad, xr + pad]
    p0 = ceilf(__fadd_rn(__fsub_rn(E.u, 0.5f + kPad), xl));
    p1 = floorf(__fadd_rn(__fadd_rn(E.u, kPad - 0.5f), xr));
    return true;
}

// Columns [c0, c1) of tile row ty (tiles TW x TH, TW a power of two) within
// [tx0, tx1).
__device__ __forceinline__ uint2 footprint_cols(const FootprintEllipse &E, uint32_t ty, int TW, int TH,
                                                uint32_t tx0, uint32_t tx1) {
    if (!E.exact) return make_uint2(tx0, tx1);
    float p0, p1;
    if (!footprint_span(E, (float)(ty * TH), (float)((ty + 1) * TH), p0, p1)) return make_uint2(tx0, tx0);
    const float inv_w = __frcp_rn((float)TW);  // exact for a power of two
    const float c0 = fmaxf(floorf(__fmul_rn(p0, inv_w)), (float)tx0);
    const float c1 = fminf(__fadd_rn(floorf(__fmul_rn(p1, inv_w)), 1.0f), (float)tx1);
    if (!(c0 < c1)) return make_uint2(tx0, tx0);
    return make_uint2((uint32_t)c0, (uint32_t)c1);
}

// 1/x on the SFU (PTX rcp.approx.ftz.f32, within 1 ulp); the adjoints use it
// to walk the transmittance back, where no decision depends on the result
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Pairs of FP32 values in one instruction (PTX .f32x2 arithmetic, sm_100
// and later).  Each half is rounded exactly as the scalar __f*_rn
// intrinsic rounds it, so packed and scalar code give identical bits.
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Gaussian falloff exponent in base-2 units for the record's prescaled
// conic (a', b', c') = -log2(e) (a/2, b, c/2): the pixel weight is
// 2^(a' dx^2 + b' dx dy + c' dy^2) = 2^(A + dy (B + c' dy)) with the
// column terms A = a' dx^2 and B = b' dx computed once per entry and pixel
// column (a thread's pixels share dx), leaving two fused multiply-adds per
// pixel.  Written with explicit roundings so every kernel that evaluates
// it gets bit-identical results.
struct FalloffColumn {
    float A, B;
};

__device__ __forceinline__ FalloffColumn falloff_column(float ap, float bp, float dx) {
    FalloffColumn c;
    c.A = __fmul_rn(__fmul_rn(ap, dx), dx);
    c.B = __fmul_rn(bp, dx);
    return c;
}

__device__ __forceinline__ float falloff_exp2(const FalloffColumn &c, float cp, float dy) {
    return __fmaf_rn(__fmaf_rn(cp, dy, c.B), dy, c.A);
}

// falloff_exp2 for two pixels of one column (rows dy.x, dy.y), operands as
// pairs: A2 = (A, A), B2 = (B, B), cp2 = (c', c'); the same roundings in
// each half
__device__ __forceinline__ float2 falloff_exp2_x2(float2 A2, float2 B2, float2 cp2, float2 dy) {
    return fma2(fma2(cp2, dy, B2), dy, A2);
}

// Sky background (Sec. 3.4, C_f = C + (1 - O) f_sky(d)): the four texels
// (index of the texel's first channel) and bilinear weights that the ray of
// pixel (px, py) samples.  d = R^T ((x - cx)/fx, (y - cy)/fy, 1) at the
// (jittered) pixel centre; faces +X -X +Y -Y +Z -Z with the OpenGL
// cube-map face coordinates; bilinear inside the face, edges clamped.
__device__ __forceinline__ void sky_texels(const ViewDesc &V, int px, int py, size_t idx[4], float w[4]) {
    float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
    if (V.sky_jitter) {
        const size_t q = (size_t)py * V.W + px;
        sx += V.sky_jitter[q];
        sy += V.sky_jitter[(size_t)V.W * V.H + q];
    }
    const float dcx = (sx - V.cx) / V.fx, dcy = (sy - V.cy) / V.fy;
    float d[3];
    for (int k = 0; k < 3; k++) d[k] = V.R[k] * dcx + V.R[3 + k] * dcy + V.R[6 + k];
    const float ax = fabsf(d[0]), ay = fabsf(d[1]), az = fabsf(d[2]);
    int face;
    float sc, tc, ma;
    if (ax >= ay && ax >= az) {
        ma = ax;
        if (d[0] > 0.f) { face = 0; sc = -d[2]; tc = -d[1]; } else { face = 1; sc = d[2]; tc = -d[1]; }
    } else if (ay >= az) {
        ma = ay;
        if (d[1] > 0.f) { face = 2; sc = d[0]; tc = d[2]; } else { face = 3; sc = d[0]; tc = -d[2]; }
    } else {
        ma = az;
        if (d[2] > 0.f) { face = 4; sc = d[0]; tc = -d[1]; } else { face = 5; sc = -d[0]; tc = -d[1]; }
    }
    const int R = V.sky_res;
    const float x = 0.5f * (sc / ma + 1.0f) * R - 0.5f, y = 0.5f * (tc / ma + 1.0f) * R - 0.5f;
    const float x0f = floorf(x), y0f = floorf(y);
    const float fx = x - x0f, fy = y - y0f;
    const int x0 = min(max((int)x0f, 0), R - 1), x1 = min(max((int)x0f + 1, 0), R - 1);
    const int y0 = min(max((int)y0f, 0), R - 1), y1 = min(max((int)y0f + 1, 0), R - 1);
    const size_t base = (size_t)face * R * R;
    idx[0] = 3 * (base + (size_t)y0 * R + x0); w[0] = (1.f - fx) * (1.f - fy);
    idx[1] = 3 * (base + (size_t)y0 * R + x1); w[1] = fx * (1.f - fy);
    idx[2] = 3 * (base + (size_t)y1 * R + x0); w[2] = (1.f - fx) * fy;
    idx[3] = 3 * (base + (size_t)y1 * R + x1); w[3] = fx * fy;
}

// Programmatic dependent launch: a kernel started with pdl_launch may be
// scheduled while the kernel before it on the stream finishes, so that its
// launch and block dispatch overlap the previous kernel's last blocks.
// Every such kernel calls pdl_enter() first, which waits until the previous
// kernel has completed with all its writes visible (griddepcontrol.wait):
// no work overlaps.  Kernels do not signal their dependents early (the
// signal is implicit when their blocks exit): an early signal let waiting
// blocks of the next kernel sit beside the running one and made the
// captured steps 6 to 9 % slower.  For a kernel launched without the
// attribute the wait returns at once.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace pvg

// host-side launchers (one translation unit each)
namespace pvg {

// kernel<<<grid, block, smem, s>>>(args...) with programmatic stream
// serialization allowed (the kernel must begin with pdl_enter()); a launch
// error is left for cudaGetLastError, as with <<<>>>
template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// counts every kernel launch of the library (reported by pvg_kernel_launches)
void note_launch();
// streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// read once per device); grids of the grid-stride kernels are multiples of it
int device_sm_count();
// radix sort scratch: digit histograms of up to kMaxSortBlocks blocks (4 per
// SM on parts of up to 256 SMs; larger parts use kMaxSortBlocks blocks) and
// the scan partials
constexpr int kMaxSortBlocks = 1024;
constexpr int kSortRadix = 256;
constexpr int kMaxScanBlocks = 1024;
constexpr size_t kSortTempBytes = sizeof(uint32_t) * ((size_t)kSortRadix * kMaxSortBlocks + kMaxScanBlocks);
cudaError_t set_sh_constants();      // both copies of the SH constants
cudaError_t set_sh_constants_bwd();  // the adjoint's copy
void launch_project_count(const Params &p, cudaStream_t s);
void launch_finalize(const Params &p, cudaStream_t s);
void launch_preprocess_bwd(const Params &p, bool several_views, cudaStream_t s);
// sort / scan
size_t sort_temp_bytes();  // kSortTempBytes
// Compaction of the visible items (count > 0) into (depth key, gid) pairs
// in gid order; also writes inv[i] = 0xffffffff for the invisible items
// and the first digit pass's histogram of the depth sort that follows
// (radix_sort_pairs over capacity n_items, bits from 0, first_hist = true).
void compact_visible(const Params &p, uint32_t *keys_out, uint32_t *vals_out, uint32_t *inv, void *temp,
                     cudaStream_t s);
// inv_out (optional): the last pass also writes inv_out[value] = the
// value's final position.  first_hist: the first pass's digit histogram is
// already in the scratch (counted by the keys' producer), no upsweep.
void radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      const uint32_t *d_count, uint32_t capacity, int begin_bit, int end_bit, void *temp,
                      cudaStream_t s, bool *result_in_alt, uint32_t *inv_out = nullptr, bool first_hist = false);
void scan_count_pairs(const Params &p, void *temp, cudaStream_t s);
void scan_emit_pairs(const Params &p, void *temp, cudaStream_t s);
size_t emit_chunks(uint32_t capacity);
void launch_ranges(const Params &p, cudaStream_t s);
void launch_tile_order(const Params &p, cudaStream_t s);
// the adjoint's first kernel: p.g2d rows of the visible items zeroed, and
// the adjoint's tile order by walk[tile] (longest first) into order
void launch_bwd_prep(const Params &p, const uint32_t *walk, uint32_t *order, cudaStream_t s);
// raster
bool composite_supported(int tw, int th, int px);
void launch_composite(const Params &p, cudaStream_t s);
void launch_composite_stats(const Params &p, cudaStream_t s);
void launch_composite_bwd(const Params &p, cudaStream_t s);
// L1 loss with a fixed-order sum; scratch: l1_loss_scratch_bytes(), zeroed once
size_t l1_loss_scratch_bytes();
cudaError_t launch_l1_loss(const float *pred, const float *target, int64_t n, float scale, float *dl, float *loss,
                           void *scratch, cudaStream_t s);
// photometric loss (1 - lambda_r) L1 + lambda_r (1 - SSIM)
size_t rgb_loss_partials(int channels, int height, int width);
cudaError_t launch_rgb_loss(const float *pred, const float *target, int channels, int height, int width,
                            float lambda_r, float *dl, float *loss, void *partials, cudaStream_t s);
// render-server hooks (api.cu): one request's view descriptor built on the
// host (bases 0), workspace reservation, the views' device buffer of a
// frame, its counters (visible, pairs, overflow) and the forward launch
// sequence over descriptors written to that buffer on the stream
pvg_status_t serve_view_desc(pvg_ctx_t *x, const pvg_scene_t *scene, const pvg_camera_t *cam, const pvg_image_t *dst,
                             ViewDesc *out, uint32_t *tiles, uint32_t *pix);
pvg_status_t serve_reserve(pvg_ctx_t *x, pvg_frame_t *f, uint64_t items, uint64_t tiles, uint64_t pix,
                           uint64_t pairs, int max_views);
ViewDesc *serve_view_buffer(pvg_frame_t *f);
const uint32_t *serve_counters(pvg_frame_t *f);
pvg_status_t serve_forward(pvg_ctx_t *x, pvg_frame_t *f, std::vector<ViewDesc> &views, uint32_t NV, uint32_t tiles,
                           uint32_t pix, uint32_t pair_capacity, cudaStream_t s);
// extra channels
int feat_count(int mask, int n_sem);
void launch_composite_feat(const Params &p, cudaStream_t s);
void launch_composite_feat_bwd(const Params &p, cudaStream_t s);
void launch_feat_param_bwd(const Params &p, cudaStream_t s);
}  // namespace pvg

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
//     rect[m]   tile rectangle, packed (tx0 | ty0 << 16, tx1 | ty1 << 16)
//   pairs     (tile, m) pairs sorted by (tile, depth, gid)             [K]
//   ranges    [start, end) into the pairs per global tile             [tiles]
//   pixels    final transmittance and last blended list position      [sum HW]
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pvg {

constexpr float kAlphaMin = 1.0f / 255.0f;  // skip gate
constexpr float kAlphaCap = 0.99f;          // alpha cap
constexpr float kTStop = 1e-4f;             // transmittance stop
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
    // device counters: [0] visible M, [1] pairs K, [2] overflow flag
    uint32_t *counters;
    // per-item scratch
    uint32_t *item_cnt;      // [NV] tiles touched (0 = invisible)
    uint32_t *item_zkey;     // [NV] depth bits (valid where item_cnt > 0)
    // visible
    uint32_t *sgid;          // [M]
    uint32_t *inv;           // [NV] depth position of each item, 0xffffffff if not visible
    uint32_t *szkey;         // [M]
    float4 *rec;             // [M*3]
    uint2 *rect;             // [M]
    uint32_t *vis_cnt;       // [M] tiles per visible item
    uint32_t *vis_off;       // [M] first pair position of the item
    uint32_t *chunk_start;   // [K / 2048 + 1] first item of each pair chunk
    // pairs
    uint32_t *pair_keys;     // [K] tile ids (sorted in place via ping-pong)
    uint32_t *pair_vals;     // [K]
    uint2 *ranges;           // [total_tiles]
    uint32_t *tile_order;    // [total_tiles] tiles by decreasing list length (compositor launch order)
    float *pix_T;            // [sum HW]
    uint32_t *pix_last;      // [sum HW] list position after the last blend
    uint32_t *pix_neval;     // [2][sum HW] stats pass: in-footprint entries up to the stop, and blended ones
    // backward
    float *g2d;              // [M*10] image-space gradients by depth position (u, v, conic a b c,
                             // o~, colour with the forward's clamp applied, z)
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
__device__ __forceinline__ void record_terms(const float4 *rec, uint32_t m, float4 &s0, float2 &s1, float4 &s2) {
    const float4 a = rec[3 * (size_t)m], b = rec[3 * (size_t)m + 1], c = rec[3 * (size_t)m + 2];
    s0 = make_float4(a.x, a.y, -0.5f * kLog2e * a.z, -kLog2e * a.w);
    s1 = make_float2(-0.5f * kLog2e * b.x, b.y);
    s2 = make_float4(c.x, c.y, c.z, b.z);
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
// 2^(a' dx^2 + b' dx dy + c' dy^2).  Written with explicit roundings so
// every kernel that calls it gets bit-identical results.
__device__ __forceinline__ float falloff_exp2(float ap, float bp, float cp, float dx, float dy) {
    const float t = __fmaf_rn(bp, dy, __fmul_rn(ap, dx));
    return __fmaf_rn(__fmul_rn(cp, dy), dy, __fmul_rn(dx, t));
}

// falloff_exp2 for two pixels of one column (same dx, rows dy.x, dy.y),
// operands given as pairs: adx = (a' dx, a' dx), bp = (b', b'),
// cp = (c', c'), dx2 = (dx, dx); the same roundings in each half
__device__ __forceinline__ float2 falloff_exp2_x2(float2 adx, float2 bp, float2 cp, float2 dx2, float2 dy) {
    const float2 t = fma2(bp, dy, adx);
    return fma2(mul2(cp, dy), dy, mul2(dx2, t));
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

}  // namespace pvg

// host-side launchers (one translation unit each)
namespace pvg {
// counts every kernel launch of the library (reported by pvg_kernel_launches)
void note_launch();
cudaError_t set_sh_constants();      // both copies of the SH constants
cudaError_t set_sh_constants_bwd();  // the adjoint's copy
void launch_project_count(const Params &p, cudaStream_t s);
void launch_scatter_inv(const Params &p, cudaStream_t s);
void launch_finalize(const Params &p, cudaStream_t s);
void launch_preprocess_bwd(const Params &p, bool accumulate_atomic, cudaStream_t s);
// sort / scan
size_t sort_temp_bytes(uint32_t capacity);
void compact_visible(const Params &p, uint32_t *keys_out, uint32_t *vals_out, void *temp, cudaStream_t s);
void radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                      const uint32_t *d_count, uint32_t capacity, int begin_bit, int end_bit, void *temp,
                      cudaStream_t s, bool *result_in_alt);
void scan_count_pairs(const Params &p, void *temp, cudaStream_t s);
void scan_emit_pairs(const Params &p, void *temp, cudaStream_t s);
size_t emit_chunks(uint32_t capacity);
void launch_ranges(const Params &p, cudaStream_t s);
void launch_tile_order(const Params &p, cudaStream_t s);
// raster
bool composite_supported(int tw, int th, int px);
void launch_composite(const Params &p, cudaStream_t s);
void launch_composite_stats(const Params &p, cudaStream_t s);
void launch_composite_bwd(const Params &p, cudaStream_t s);
// photometric loss (1 - lambda_r) L1 + lambda_r (1 - SSIM)
size_t rgb_loss_partials(int channels, int height, int width);
cudaError_t launch_rgb_loss(const float *pred, const float *target, int channels, int height, int width,
                            float lambda_r, float *dl, float *loss, void *partials, cudaStream_t s);
// extra channels
int feat_count(int mask, int n_sem);
void launch_composite_feat(const Params &p, cudaStream_t s);
void launch_composite_feat_bwd(const Params &p, cudaStream_t s);
void launch_feat_param_bwd(const Params &p, cudaStream_t s);
}  // namespace pvg

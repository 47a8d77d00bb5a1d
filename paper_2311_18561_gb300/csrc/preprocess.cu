// preprocess.cu -- per-(view, Gaussian) kernels of the PVG rasterizer.
//
//   k_project_count  (stage a, pass 1) time evaluation (Sec. 3.2, Eq. 6-7),
//                    view transform and culls, 3D covariance from (s, q),
//                    EWA projection (Sec. 3.1, Eq. 2) and the tile
//                    footprint; writes the tile count and depth bits of
//                    every item.
//   k_finalize       (stage a, pass 2) for every visible item, in item
//                    order: the same projection plus the SH colour; writes
//                    the 48-byte compositing record, the tile rectangle and
//                    the tile count at the item's depth position m.
//   k_preprocess_bwd (stage d2) adjoint of both passes, in item order: from
//                    the image-space gradients of record m to dL/d{mu, v,
//                    tau, beta, l, s, q, o, sh}.
//
// All three recompute the projection with the same inline function and
// the library is built with --fmad=false, so pass 1 and pass 2 agree bit
// for bit.  Every kernel is HBM-bound: one thread per item, grid-stride.
#include "pvg_internal.cuh"

namespace pvg {

// Real SH normalisation constants, computed on the host from
// N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (x sqrt 2 for m != 0).
__constant__ float c_sh[10];

cudaError_t set_sh_constants() {
    const double pi = 3.14159265358979323846;
    const float h[10] = {
        (float)(0.5 * sqrt(1.0 / pi)),          // Y00
        (float)sqrt(3.0 / (4.0 * pi)),          // l = 1
        (float)(0.5 * sqrt(15.0 / pi)),         // xy, yz, xz
        (float)(0.25 * sqrt(5.0 / pi)),         // 2z^2 - x^2 - y^2
        (float)(0.25 * sqrt(15.0 / pi)),        // x^2 - y^2
        (float)(0.25 * sqrt(35.0 / (2.0 * pi))),// y(3x^2 - y^2), x(x^2 - 3y^2)
        (float)(0.5 * sqrt(105.0 / pi)),        // xyz
        (float)(0.25 * sqrt(21.0 / (2.0 * pi))),// y(4z^2 - x^2 - y^2), x(...)
        (float)(0.25 * sqrt(7.0 / pi)),         // z(2z^2 - 3x^2 - 3y^2)
        (float)(0.25 * sqrt(105.0 / pi)),       // z(x^2 - y^2)
    };
    return cudaMemcpyToSymbol(c_sh, h, sizeof(h));
}

namespace {

constexpr float kInv2Pi = 0.15915494309189535f;  // 1 / (2 pi)

struct Fwd {
    // time terms
    float delta, sn, cs, egate, amp;
    float vbw;          // exp(-beta / (2 l)) when the view has a flow shift
    float3 mut;
    float ot;
    // camera space
    float3 p;
    int clampx, clampy;
    float txc, tyc;
    // covariance
    float qn[4], qinv;  // normalised quaternion, 1/|q|
    float Rq[9];        // rotation of q^
    float s[3];
    float Sig[6];       // xx xy xz yy yz zz
    float J00, J02, J11, J12;
    float Tm[6];        // J W, 2x3 row-major
    float A, B, C, det;
    float ca, cb, cc;
    float u, v;
    // footprint: guarded half extents in pixels and the tile rectangle
    float hx, hy;
    uint32_t tx0, ty0, tx1, ty1, count;
};

__device__ __forceinline__ float3 ld3(const float *p, uint32_t i) {
    return make_float3(p[3 * (size_t)i], p[3 * (size_t)i + 1], p[3 * (size_t)i + 2]);
}

// n floats at src (item-strided, so 16-byte aligned when the base is and
// n is a multiple of 4) into registers / back, as float4 when possible
template <int NF>
__device__ __forceinline__ void load_floats(const float *src, float (&dst)[NF], bool vec) {
    if constexpr (NF % 4 == 0) {
        if (vec) {
            const float4 *p = reinterpret_cast<const float4 *>(src);
#pragma unroll
            for (int q = 0; q < NF / 4; q++) {
                const float4 v = p[q];
                dst[4 * q] = v.x; dst[4 * q + 1] = v.y; dst[4 * q + 2] = v.z; dst[4 * q + 3] = v.w;
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < NF; q++) dst[q] = src[q];
}

template <int NF>
__device__ __forceinline__ void store_floats(float *dst, const float (&src)[NF], bool vec) {
    if constexpr (NF % 4 == 0) {
        if (vec) {
            float4 *p = reinterpret_cast<float4 *>(dst);
#pragma unroll
            for (int q = 0; q < NF / 4; q++) p[q] = make_float4(src[4 * q], src[4 * q + 1], src[4 * q + 2], src[4 * q + 3]);
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < NF; q++) dst[q] = src[q];
}

__device__ __forceinline__ bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Kahan's difference of products a*b - c*d, accurate to a few ulp.
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

// Steps 1-3 + footprint for item (view V, index i).  Returns false if the
// item is culled (behind the near plane, o~ < 1/255, degenerate
// covariance, non-finite values or no tile covered).
__device__ __forceinline__ bool project(const ViewDesc &V, uint32_t i, float dilation, int TW, int TH,
                                        Fwd &F) {
    // Eq. 6 / Eq. 7
    const float tau = V.tau[i], l = V.period[i], beta = V.beta[i];
    // with dt != 0 the flow-translated state of Sec. 3.4: queried at t - dt,
    // moved by v_bar dt, v_bar = v exp(-rho / 2), rho = beta / l (Eq. 10)
    F.delta = (V.t - V.dt) - tau;
    sincospif(2.0f * F.delta / l, &F.sn, &F.cs);
    F.amp = l * F.sn * kInv2Pi;
    F.vbw = 0.f;
    if (V.dt != 0.f) {
        F.vbw = expf(-0.5f * beta / l);
        F.amp = F.amp + V.dt * F.vbw;
    }
    const float3 mu = ld3(V.mu, i), vel = ld3(V.vel, i);
    F.mut = make_float3(mu.x + F.amp * vel.x, mu.y + F.amp * vel.y, mu.z + F.amp * vel.z);
    F.egate = expf(-0.5f * (F.delta * F.delta) / (beta * beta));
    F.ot = V.opac[i] * F.egate;
    // view transform
    const float *R = V.R;
    F.p.x = R[0] * F.mut.x + R[1] * F.mut.y + R[2] * F.mut.z + V.T[0];
    F.p.y = R[3] * F.mut.x + R[4] * F.mut.y + R[5] * F.mut.z + V.T[1];
    F.p.z = R[6] * F.mut.x + R[7] * F.mut.y + R[8] * F.mut.z + V.T[2];
    if (!(F.p.z > V.znear)) return false;
    if (!(F.ot >= kAlphaMin)) return false;
    // Sigma = Rq diag(s)^2 Rq^T
    {
        const float *q = V.quat + 4 * (size_t)i;
        const float qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
        F.qinv = 1.0f / sqrtf(qq);
        for (int k = 0; k < 4; k++) F.qn[k] = q[k] * F.qinv;
        const float w = F.qn[0], x = F.qn[1], y = F.qn[2], z = F.qn[3];
        F.Rq[0] = 1.f - 2.f * (y * y + z * z); F.Rq[1] = 2.f * (x * y - w * z);       F.Rq[2] = 2.f * (x * z + w * y);
        F.Rq[3] = 2.f * (x * y + w * z);       F.Rq[4] = 1.f - 2.f * (x * x + z * z); F.Rq[5] = 2.f * (y * z - w * x);
        F.Rq[6] = 2.f * (x * z - w * y);       F.Rq[7] = 2.f * (y * z + w * x);       F.Rq[8] = 1.f - 2.f * (x * x + y * y);
        const float3 sc = ld3(V.scale, i);
        F.s[0] = sc.x; F.s[1] = sc.y; F.s[2] = sc.z;
        float M[9];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) M[3 * a + b] = F.Rq[3 * a + b] * F.s[b];
        F.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
        F.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
        F.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
        F.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
        F.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
        F.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    }
    // J (with the widened-frustum clamp) and Tm = J W
    {
        const float z = F.p.z, iz = 1.0f / z;
        float rx = F.p.x * iz, ry = F.p.y * iz;
        F.clampx = rx < -V.limx ? -1 : (rx > V.limx ? 1 : 0);
        F.clampy = ry < -V.limy ? -1 : (ry > V.limy ? 1 : 0);
        if (F.clampx) rx = F.clampx * V.limx;
        if (F.clampy) ry = F.clampy * V.limy;
        F.txc = rx * z;
        F.tyc = ry * z;
        F.J00 = V.fx * iz;
        F.J11 = V.fy * iz;
        F.J02 = -V.fx * F.txc * (iz * iz);
        F.J12 = -V.fy * F.tyc * (iz * iz);
        for (int k = 0; k < 3; k++) {
            F.Tm[k] = F.J00 * R[k] + F.J02 * R[6 + k];
            F.Tm[3 + k] = F.J11 * R[3 + k] + F.J12 * R[6 + k];
        }
        const float *S = F.Sig;
        // rows of Tm times Sigma
        const float a0 = F.Tm[0] * S[0] + F.Tm[1] * S[1] + F.Tm[2] * S[2];
        const float a1 = F.Tm[0] * S[1] + F.Tm[1] * S[3] + F.Tm[2] * S[4];
        const float a2 = F.Tm[0] * S[2] + F.Tm[1] * S[4] + F.Tm[2] * S[5];
        const float b0 = F.Tm[3] * S[0] + F.Tm[4] * S[1] + F.Tm[5] * S[2];
        const float b1 = F.Tm[3] * S[1] + F.Tm[4] * S[3] + F.Tm[5] * S[4];
        const float b2 = F.Tm[3] * S[2] + F.Tm[4] * S[4] + F.Tm[5] * S[5];
        F.A = a0 * F.Tm[0] + a1 * F.Tm[1] + a2 * F.Tm[2] + dilation;
        F.B = a0 * F.Tm[3] + a1 * F.Tm[4] + a2 * F.Tm[5];
        F.C = b0 * F.Tm[3] + b1 * F.Tm[4] + b2 * F.Tm[5] + dilation;
        F.det = diff_of_products(F.A, F.C, F.B, F.B);
        if (!(F.det > 0.0f)) return false;
        const float idet = 1.0f / F.det;
        F.ca = F.C * idet;
        F.cb = -F.B * idet;
        F.cc = F.A * idet;
        F.u = V.fx * (F.p.x * iz) + V.cx;
        F.v = V.fy * (F.p.y * iz) + V.cy;
    }
    // footprint: o~ G >= 1/255 inside the ellipse d^T conic d <= Q,
    // Q = 2 ln(255 o~), whose bounding box has half extents sqrt(Q A),
    // sqrt(Q C); widened by 0.1 % + 1 px against rounding
    {
        float Q = 2.0f * logf(255.0f * F.ot);
        Q = Q > 0.0f ? Q : 0.0f;
        const float rx = sqrtf(Q * F.A) * 1.001f + 1.0f;
        const float ry = sqrtf(Q * F.C) * 1.001f + 1.0f;
        if (!(isfinite(F.u) && isfinite(F.v)) || rx != rx || ry != ry) return false;
        F.hx = rx;
        F.hy = ry;
        const float x0 = fmaxf(ceilf(F.u - rx - 0.5f), 0.0f);
        const float x1 = fminf(floorf(F.u + rx - 0.5f), (float)(V.W - 1));
        const float y0 = fmaxf(ceilf(F.v - ry - 0.5f), 0.0f);
        const float y1 = fminf(floorf(F.v + ry - 0.5f), (float)(V.H - 1));
        if (x0 > x1 || y0 > y1) return false;
        F.tx0 = (uint32_t)x0 / TW;
        F.tx1 = (uint32_t)x1 / TW + 1;
        F.ty0 = (uint32_t)y0 / TH;
        F.ty1 = (uint32_t)y1 / TH + 1;
        F.count = (F.tx1 - F.tx0) * (F.ty1 - F.ty0);
    }
    return true;
}

// SH basis Y[k] at unit direction (x, y, z), k = l^2 + l + m, for degree
// D, and optionally the gradient of each polynomial.  D is a template
// argument so that every index is a constant and the arrays stay in
// registers.
template <int D, bool kGrad>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float (&Y)[16], float (&dY)[16][3]) {
    Y[0] = c_sh[0];
    if (kGrad) { dY[0][0] = dY[0][1] = dY[0][2] = 0.f; }
    if constexpr (D >= 1) {
        const float c1 = c_sh[1];
        Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
        if (kGrad) {
            dY[1][0] = 0.f; dY[1][1] = -c1; dY[1][2] = 0.f;
            dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = c1;
            dY[3][0] = -c1; dY[3][1] = 0.f; dY[3][2] = 0.f;
        }
    }
    if constexpr (D >= 2) {
        const float c2 = c_sh[2], c3 = c_sh[3], c4 = c_sh[4];
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = c2 * x * y;
        Y[5] = -c2 * y * z;
        Y[6] = c3 * (2.f * zz - xx - yy);
        Y[7] = -c2 * x * z;
        Y[8] = c4 * (xx - yy);
        if (kGrad) {
            dY[4][0] = c2 * y; dY[4][1] = c2 * x; dY[4][2] = 0.f;
            dY[5][0] = 0.f; dY[5][1] = -c2 * z; dY[5][2] = -c2 * y;
            dY[6][0] = -2.f * c3 * x; dY[6][1] = -2.f * c3 * y; dY[6][2] = 4.f * c3 * z;
            dY[7][0] = -c2 * z; dY[7][1] = 0.f; dY[7][2] = -c2 * x;
            dY[8][0] = 2.f * c4 * x; dY[8][1] = -2.f * c4 * y; dY[8][2] = 0.f;
        }
    }
    if constexpr (D >= 3) {
        const float c5 = c_sh[5], c6 = c_sh[6], c7 = c_sh[7], c8 = c_sh[8], c9 = c_sh[9];
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[9] = -c5 * y * (3.f * xx - yy);
        Y[10] = c6 * x * y * z;
        Y[11] = -c7 * y * (4.f * zz - xx - yy);
        Y[12] = c8 * z * (2.f * zz - 3.f * xx - 3.f * yy);
        Y[13] = -c7 * x * (4.f * zz - xx - yy);
        Y[14] = c9 * z * (xx - yy);
        Y[15] = -c5 * x * (xx - 3.f * yy);
        if (kGrad) {
            dY[9][0] = -6.f * c5 * x * y; dY[9][1] = -3.f * c5 * (xx - yy); dY[9][2] = 0.f;
            dY[10][0] = c6 * y * z; dY[10][1] = c6 * x * z; dY[10][2] = c6 * x * y;
            dY[11][0] = 2.f * c7 * x * y; dY[11][1] = -c7 * (4.f * zz - xx - 3.f * yy); dY[11][2] = -8.f * c7 * y * z;
            dY[12][0] = -6.f * c8 * x * z; dY[12][1] = -6.f * c8 * y * z; dY[12][2] = c8 * (6.f * zz - 3.f * xx - 3.f * yy);
            dY[13][0] = -c7 * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * c7 * x * y; dY[13][2] = -8.f * c7 * x * z;
            dY[14][0] = 2.f * c9 * x * z; dY[14][1] = -2.f * c9 * y * z; dY[14][2] = c9 * (xx - yy);
            dY[15][0] = -3.f * c5 * (xx - yy); dY[15][1] = 6.f * c5 * x * y; dY[15][2] = 0.f;
        }
    }
}

__global__ void __launch_bounds__(256) k_project_count(Params P) {
    const uint32_t n = P.n_items;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const int view = view_of_item(P.views, P.n_views, g);
        const ViewDesc &V = P.views[view];
        Fwd F;
        const bool vis = project(V, g - V.item_base, P.dilation, P.tile_w, P.tile_h, F);
        P.item_cnt[g] = vis ? F.count : 0u;
        if (vis) P.item_zkey[g] = __float_as_uint(F.p.z);
    }
}

// inverse of the depth order: inv[sgid[m]] = m (inv is 0xffffffff elsewhere)
__global__ void __launch_bounds__(256) k_scatter_inv(Params P) {
    const uint32_t M = P.counters[0];
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x)
        P.inv[P.sgid[m]] = m;
}

// Records in depth order, computed in item order (coalesced parameter
// reads; the 48-byte record goes to its depth position m = inv[g]).
template <int D>
__global__ void __launch_bounds__(256) k_finalize(Params P) {
    constexpr int K = (D + 1) * (D + 1);
    const uint32_t n = P.n_items;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const uint32_t m = P.inv[g];
        if (m == 0xffffffffu) continue;
        const int view = view_of_item(P.views, P.n_views, g);
        const ViewDesc &V = P.views[view];
        const uint32_t i = g - V.item_base;
        Fwd F;
        const bool vis = project(V, i, P.dilation, P.tile_w, P.tile_h, F);
        if (!vis) {  // cannot happen (same arithmetic as pass 1); stay safe
            P.vis_cnt[m] = 0u;
            P.rect[m] = make_uint2(0u, 0u);
            continue;
        }
        float dx = F.mut.x - V.campos[0], dy = F.mut.y - V.campos[1], dz = F.mut.z - V.campos[2];
        const float inv = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv; dy *= inv; dz *= inv;
        float Y[16], dY[16][3];
        sh_eval<D, false>(dx, dy, dz, Y, dY);
        float sh[3 * K];
        load_floats<3 * K>(V.sh + (size_t)i * K * 3, sh, aligned16(V.sh));
        float rgb[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int k = 0; k < K; k++) {
            rgb[0] += sh[3 * k] * Y[k];
            rgb[1] += sh[3 * k + 1] * Y[k];
            rgb[2] += sh[3 * k + 2] * Y[k];
        }
        const float z = __uint_as_float(P.szkey[m]);
        P.rec[3 * (size_t)m + 0] = make_float4(F.u, F.v, F.ca, F.cb);
        P.rec[3 * (size_t)m + 1] = make_float4(F.cc, F.ot, z, F.hx);
        P.rec[3 * (size_t)m + 2] = make_float4(fmaxf(rgb[0], 0.0f), fmaxf(rgb[1], 0.0f), fmaxf(rgb[2], 0.0f), F.hy);
        P.rect[m] = make_uint2(F.tx0 | (F.ty0 << 16), F.tx1 | (F.ty1 << 16));
        P.vis_cnt[m] = F.count;
    }
}

__device__ __forceinline__ void put(float *dst, size_t k, float v, bool atomic) {
    if (atomic) atomicAdd(dst + k, v);
    else dst[k] = v;
}

// Writes zero gradients for item g of view V (single-view calls, where
// this kernel writes every gradient entry instead of a separate memset).
template <int K>
__device__ __forceinline__ void zero_grads(const ViewDesc &V, uint32_t i) {
    if (V.g_mu) for (int k = 0; k < 3; k++) V.g_mu[3 * (size_t)i + k] = 0.f;
    if (V.g_vel) for (int k = 0; k < 3; k++) V.g_vel[3 * (size_t)i + k] = 0.f;
    if (V.g_scale) for (int k = 0; k < 3; k++) V.g_scale[3 * (size_t)i + k] = 0.f;
    if (V.g_quat) {
        const float z4[4] = {0.f, 0.f, 0.f, 0.f};
        store_floats<4>(V.g_quat + 4 * (size_t)i, z4, aligned16(V.g_quat));
    }
    if (V.g_tau) V.g_tau[i] = 0.f;
    if (V.g_beta) V.g_beta[i] = 0.f;
    if (V.g_period) V.g_period[i] = 0.f;
    if (V.g_opac) V.g_opac[i] = 0.f;
    if (V.g_sh) {
        float z[3 * K];
#pragma unroll
        for (int k = 0; k < 3 * K; k++) z[k] = 0.f;
        store_floats<3 * K>(V.g_sh + (size_t)i * 3 * K, z, aligned16(V.g_sh));
    }
}

// Adjoint of the projection and colour, in item order: item g reads the
// image-space gradients of its depth position m = inv[g].  With `atomic`
// (several views share the gradients) the gradients were zeroed before and
// are accumulated; otherwise every entry of item g is written, zeros for
// invisible items.
template <int D>
__global__ void __launch_bounds__(256) k_preprocess_bwd(Params P, bool atomic) {
    constexpr int K = (D + 1) * (D + 1);
    const uint32_t n = P.n_items;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const int view = view_of_item(P.views, P.n_views, g);
        const ViewDesc &V = P.views[view];
        const uint32_t i = g - V.item_base;
        const uint32_t m = P.inv[g];
        Fwd F;
        if (m == 0xffffffffu || !project(V, i, P.dilation, P.tile_w, P.tile_h, F)) {
            if (!atomic) zero_grads<K>(V, i);
            continue;
        }
        const float *G2 = P.g2d + 10 * (size_t)m;
        const float gu = G2[0], gv = G2[1], ga = G2[2], gb = G2[3], gc = G2[4];
        const float got = G2[5], gz = G2[9];
        float gmut[3] = {0.f, 0.f, 0.f};
        float gp[3] = {0.f, 0.f, 0.f};

        // ---- colour: rgb = max(0, sum_k sh_k Y_k(d) + 0.5)
        {
            float dx = F.mut.x - V.campos[0], dy = F.mut.y - V.campos[1], dz = F.mut.z - V.campos[2];
            const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
            const float inv = 1.0f / dist;
            dx *= inv; dy *= inv; dz *= inv;
            float Y[16], dY[16][3];
            sh_eval<D, true>(dx, dy, dz, Y, dY);
            float sh[3 * K];
            load_floats<3 * K>(V.sh + (size_t)i * K * 3, sh, aligned16(V.sh));
            float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
            for (int k = 0; k < K; k++)
#pragma unroll
                for (int c = 0; c < 3; c++) raw[c] += sh[3 * k + c] * Y[k];
            float gcol[3];
#pragma unroll
            for (int c = 0; c < 3; c++) gcol[c] = raw[c] > 0.0f ? G2[6 + c] : 0.0f;
            float gd[3] = {0.f, 0.f, 0.f};
            if (V.g_sh) {
                if (atomic) {
#pragma unroll
                    for (int k = 0; k < K; k++)
#pragma unroll
                        for (int c = 0; c < 3; c++) atomicAdd(V.g_sh + ((size_t)i * K + k) * 3 + c, gcol[c] * Y[k]);
                } else {
                    float gsh[3 * K];
#pragma unroll
                    for (int k = 0; k < K; k++)
#pragma unroll
                        for (int c = 0; c < 3; c++) gsh[3 * k + c] = gcol[c] * Y[k];
                    store_floats<3 * K>(V.g_sh + (size_t)i * K * 3, gsh, aligned16(V.g_sh));
                }
            }
#pragma unroll
            for (int k = 0; k < K; k++) {
                const float w = gcol[0] * sh[3 * k] + gcol[1] * sh[3 * k + 1] + gcol[2] * sh[3 * k + 2];
                gd[0] += w * dY[k][0];
                gd[1] += w * dY[k][1];
                gd[2] += w * dY[k][2];
            }
            const float dot = dx * gd[0] + dy * gd[1] + dz * gd[2];
            gmut[0] += (gd[0] - dx * dot) * inv;
            gmut[1] += (gd[1] - dy * dot) * inv;
            gmut[2] += (gd[2] - dz * dot) * inv;
        }

        // ---- conic = inverse(cov2): dL/dcov2 = -Q Ghat Q
        const float a = F.ca, b = F.cb, c = F.cc;
        const float gA = -(a * a * ga + a * b * gb + b * b * gc);
        const float gB = -(a * b * ga + 0.5f * (a * c + b * b) * gb + b * c * gc);  // symmetric entry
        const float gC = -(b * b * ga + b * c * gb + c * c * gc);
        // ---- cov2 = Tm Sigma Tm^T: G_Sigma = Tm^T G2 Tm, G_Tm = 2 G2 Tm Sigma
        const float *Tm = F.Tm, *S = F.Sig;
        float GS[6];  // xx xy xz yy yz zz of the symmetric gradient
        {
            float U[6];  // G2 Tm (2x3)
            for (int k = 0; k < 3; k++) {
                U[k] = gA * Tm[k] + gB * Tm[3 + k];
                U[3 + k] = gB * Tm[k] + gC * Tm[3 + k];
            }
            GS[0] = Tm[0] * U[0] + Tm[3] * U[3];
            GS[1] = Tm[0] * U[1] + Tm[3] * U[4];
            GS[2] = Tm[0] * U[2] + Tm[3] * U[5];
            GS[3] = Tm[1] * U[1] + Tm[4] * U[4];
            GS[4] = Tm[1] * U[2] + Tm[4] * U[5];
            GS[5] = Tm[2] * U[2] + Tm[5] * U[5];
            // G_Tm = 2 U Sigma
            float GT[6];
            for (int r = 0; r < 2; r++) {
                const float *u = U + 3 * r;
                GT[3 * r + 0] = 2.f * (u[0] * S[0] + u[1] * S[1] + u[2] * S[2]);
                GT[3 * r + 1] = 2.f * (u[0] * S[1] + u[1] * S[3] + u[2] * S[4]);
                GT[3 * r + 2] = 2.f * (u[0] * S[2] + u[1] * S[4] + u[2] * S[5]);
            }
            // Tm = J W: dL/dJ = G_Tm W^T (only J00, J02, J11, J12 are free)
            const float *R = V.R;
            const float gJ00 = GT[0] * R[0] + GT[1] * R[1] + GT[2] * R[2];
            const float gJ02 = GT[0] * R[6] + GT[1] * R[7] + GT[2] * R[8];
            const float gJ11 = GT[3] * R[3] + GT[4] * R[4] + GT[5] * R[5];
            const float gJ12 = GT[3] * R[6] + GT[4] * R[7] + GT[5] * R[8];
            const float z = F.p.z, iz = 1.0f / z, iz2 = iz * iz, iz3 = iz2 * iz;
            gp[2] += gJ00 * (-V.fx * iz2) + gJ11 * (-V.fy * iz2);
            if (F.clampx == 0) {
                gp[0] += gJ02 * (-V.fx * iz2);
                gp[2] += gJ02 * (2.f * V.fx * F.p.x * iz3);
            } else {
                gp[2] += gJ02 * (V.fx * F.clampx * V.limx * iz2);
            }
            if (F.clampy == 0) {
                gp[1] += gJ12 * (-V.fy * iz2);
                gp[2] += gJ12 * (2.f * V.fy * F.p.y * iz3);
            } else {
                gp[2] += gJ12 * (V.fy * F.clampy * V.limy * iz2);
            }
            // projected mean and depth
            gp[0] += gu * V.fx * iz;
            gp[1] += gv * V.fy * iz;
            gp[2] += -(gu * V.fx * F.p.x + gv * V.fy * F.p.y) * iz2 + gz;
        }
        // ---- Sigma = M M^T, M = Rq diag(s): G_M = 2 G_Sigma M
        {
            float M[9];
            for (int r = 0; r < 3; r++)
                for (int k = 0; k < 3; k++) M[3 * r + k] = F.Rq[3 * r + k] * F.s[k];
            const float Gs[9] = {GS[0], GS[1], GS[2], GS[1], GS[3], GS[4], GS[2], GS[4], GS[5]};
            float GM[9];
            for (int r = 0; r < 3; r++)
                for (int k = 0; k < 3; k++)
                    GM[3 * r + k] = 2.f * (Gs[3 * r] * M[k] + Gs[3 * r + 1] * M[3 + k] + Gs[3 * r + 2] * M[6 + k]);
            float gsc[3], GR[9];
            for (int k = 0; k < 3; k++) gsc[k] = GM[k] * F.Rq[k] + GM[3 + k] * F.Rq[3 + k] + GM[6 + k] * F.Rq[6 + k];
            for (int r = 0; r < 3; r++)
                for (int k = 0; k < 3; k++) GR[3 * r + k] = GM[3 * r + k] * F.s[k];
            const float w = F.qn[0], x = F.qn[1], y = F.qn[2], zq = F.qn[3];
            // dR/dw, dR/dx, dR/dy, dR/dz contracted with GR
            const float gw = 2.f * (-zq * GR[1] + y * GR[2] + zq * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
            const float gx = 2.f * (y * GR[1] + zq * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + zq * GR[6] +
                                    w * GR[7] - 2.f * x * GR[8]);
            const float gy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + zq * GR[5] - w * GR[6] +
                                    zq * GR[7] - 2.f * y * GR[8]);
            const float gzq = 2.f * (-2.f * zq * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * zq * GR[4] +
                                     y * GR[5] + x * GR[6] + y * GR[7]);
            const float dot = F.qn[0] * gw + F.qn[1] * gx + F.qn[2] * gy + F.qn[3] * gzq;
            if (V.g_quat) {
                const float gq[4] = {(gw - F.qn[0] * dot) * F.qinv, (gx - F.qn[1] * dot) * F.qinv,
                                     (gy - F.qn[2] * dot) * F.qinv, (gzq - F.qn[3] * dot) * F.qinv};
                if (atomic) {
                    for (int k = 0; k < 4; k++) atomicAdd(V.g_quat + 4 * (size_t)i + k, gq[k]);
                } else {
                    store_floats<4>(V.g_quat + 4 * (size_t)i, gq, aligned16(V.g_quat));
                }
            }
            if (V.g_scale)
                for (int k = 0; k < 3; k++) put(V.g_scale, 3 * (size_t)i + k, gsc[k], atomic);
        }
        // ---- p = W mu~ + T
        {
            const float *R = V.R;
            for (int k = 0; k < 3; k++) gmut[k] += R[k] * gp[0] + R[3 + k] * gp[1] + R[6 + k] * gp[2];
        }
        // ---- time evaluation (Eq. 6 / Eq. 7)
        {
            const float3 vel = ld3(V.vel, i);
            const float l = V.period[i], beta = V.beta[i];
            const float gvd = gmut[0] * vel.x + gmut[1] * vel.y + gmut[2] * vel.z;
            if (V.g_mu)
                for (int k = 0; k < 3; k++) put(V.g_mu, 3 * (size_t)i + k, gmut[k], atomic);
            if (V.g_vel)
                for (int k = 0; k < 3; k++) put(V.g_vel, 3 * (size_t)i + k, gmut[k] * F.amp, atomic);
            const float ib2 = 1.0f / (beta * beta);
            if (V.g_tau) put(V.g_tau, i, -F.cs * gvd + got * F.ot * F.delta * ib2, atomic);
            // flow shift dt v exp(-beta / (2 l)): its beta and l terms
            const float gsh = gvd * V.dt * F.vbw;
            if (V.g_period)
                put(V.g_period, i, gvd * (F.sn * kInv2Pi - F.delta / l * F.cs) + gsh * (0.5f * beta / (l * l)), atomic);
            if (V.g_opac) put(V.g_opac, i, got * F.egate, atomic);
            if (V.g_beta) put(V.g_beta, i, got * F.ot * F.delta * F.delta * ib2 / beta - gsh * (0.5f / l), atomic);
        }
    }
}

int grid_for(uint32_t n) {
    uint32_t g = (n + 255) / 256;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}

}  // namespace

void launch_project_count(const Params &p, cudaStream_t s) {
    note_launch();
    k_project_count<<<grid_for(p.n_items), 256, 0, s>>>(p);
}

void launch_scatter_inv(const Params &p, cudaStream_t s) {
    note_launch();
    k_scatter_inv<<<grid_for(p.n_items), 256, 0, s>>>(p);
}

void launch_finalize(const Params &p, cudaStream_t s) {
    note_launch();
    switch (p.sh_degree) {
        case 0: k_finalize<0><<<grid_for(p.n_items), 256, 0, s>>>(p); break;
        case 1: k_finalize<1><<<grid_for(p.n_items), 256, 0, s>>>(p); break;
        case 2: k_finalize<2><<<grid_for(p.n_items), 256, 0, s>>>(p); break;
        default: k_finalize<3><<<grid_for(p.n_items), 256, 0, s>>>(p); break;
    }
}

void launch_preprocess_bwd(const Params &p, bool accumulate_atomic, cudaStream_t s) {
    note_launch();
    switch (p.sh_degree) {
        case 0: k_preprocess_bwd<0><<<grid_for(p.n_items), 256, 0, s>>>(p, accumulate_atomic); break;
        case 1: k_preprocess_bwd<1><<<grid_for(p.n_items), 256, 0, s>>>(p, accumulate_atomic); break;
        case 2: k_preprocess_bwd<2><<<grid_for(p.n_items), 256, 0, s>>>(p, accumulate_atomic); break;
        default: k_preprocess_bwd<3><<<grid_for(p.n_items), 256, 0, s>>>(p, accumulate_atomic); break;
    }
}

}  // namespace pvg

// preprocess_common.cuh -- projection, SH basis and load helpers shared by
// the per-item forward kernels (preprocess.cu) and their adjoint
// (preprocess_bwd.cu).
#pragma once
#include <cmath>

#include "pvg_internal.cuh"

namespace pvg {

// Real SH normalisation constants (one copy per translation unit, set by
// set_sh_constants), computed on the host from
// N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (x sqrt 2 for m != 0).
static __constant__ float c_sh[10];

static inline void sh_constant_values(float h[10]) {
    const double pi = 3.14159265358979323846;
    h[0] = (float)(0.5 * std::sqrt(1.0 / pi));            // Y00
    h[1] = (float)std::sqrt(3.0 / (4.0 * pi));            // l = 1
    h[2] = (float)(0.5 * std::sqrt(15.0 / pi));           // xy, yz, xz
    h[3] = (float)(0.25 * std::sqrt(5.0 / pi));           // 2z^2 - x^2 - y^2
    h[4] = (float)(0.25 * std::sqrt(15.0 / pi));          // x^2 - y^2
    h[5] = (float)(0.25 * std::sqrt(35.0 / (2.0 * pi)));  // y(3x^2 - y^2), x(x^2 - 3y^2)
    h[6] = (float)(0.5 * std::sqrt(105.0 / pi));          // xyz
    h[7] = (float)(0.25 * std::sqrt(21.0 / (2.0 * pi)));  // y(4z^2 - x^2 - y^2), x(...)
    h[8] = (float)(0.25 * std::sqrt(7.0 / pi));           // z(2z^2 - 3x^2 - 3y^2)
    h[9] = (float)(0.25 * std::sqrt(105.0 / pi));         // z(x^2 - y^2)
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

int grid_for(uint32_t n) {
    uint32_t g = (n + 255) / 256;
    if (g < 1) g = 1;
    const uint32_t cap = 16u * (uint32_t)device_sm_count();
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace
}  // namespace pvg

// preprocess_bwd.cu -- adjoint of the per-item projection and colour
// (stage d2): for the visible items in gid order, from the image-space
// gradients of record m = inv[g] to dL/d{mu, v, tau, beta, l, s, q, o, sh}
// (Sec. 3.1, Eq. 2-4;
// Sec. 3.2, Eq. 6-8; the flow shift of Sec. 3.4).  Visibility comes from
// inv[]; the projection is recomputed for its intermediate terms only, so
// this file may contract a*b+c into fused multiply-adds.
#include "preprocess_common.cuh"

namespace pvg {

cudaError_t set_sh_constants_bwd() {
    float h[10];
    sh_constant_values(h);
    return cudaMemcpyToSymbol(c_sh, h, sizeof(h));
}

namespace {

__device__ __forceinline__ void put(float *dst, size_t k, float v, bool atomic) {
    if (atomic) atomicAdd(dst + k, v);
    else dst[k] = v;
}

// dL/dsh[k][c] = gcol[c] Y_k(d), written (or accumulated) in groups of four
// basis functions (three float4) when the rows allow it
template <int D>
__device__ __forceinline__ void sh_coef_adjoint(float x, float y, float z, const float (&gcol)[3], float *gsh,
                                                bool vec, bool atomic) {
    constexpr int K = (D + 1) * (D + 1);
    float Y[16], dY[16][3];
    sh_eval<D, false>(x, y, z, Y, dY);
    if constexpr (K % 4 == 0) {
        if (vec && !atomic) {
            float4 *g4 = reinterpret_cast<float4 *>(gsh);
#pragma unroll
            for (int q = 0; q < K / 4; q++) {
                float g[12];
#pragma unroll
                for (int j = 0; j < 4; j++)
#pragma unroll
                    for (int c = 0; c < 3; c++) g[3 * j + c] = gcol[c] * Y[4 * q + j];
                g4[3 * q] = make_float4(g[0], g[1], g[2], g[3]);
                g4[3 * q + 1] = make_float4(g[4], g[5], g[6], g[7]);
                g4[3 * q + 2] = make_float4(g[8], g[9], g[10], g[11]);
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
        for (int c = 0; c < 3; c++) put(gsh, 3 * (size_t)k + c, gcol[c] * Y[k], atomic);
}

// dL/dsh[k][c] += gcol[c] Y_k(d) into acc[(3 k + c) * stride] (shared
// memory, one column per thread)
template <int D>
__device__ __forceinline__ void sh_coef_accumulate(float x, float y, float z, const float (&gcol)[3], float *acc,
                                                   int stride) {
    constexpr int K = (D + 1) * (D + 1);
    float Y[16], dY[16][3];
    sh_eval<D, false>(x, y, z, Y, dY);
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
        for (int c = 0; c < 3; c++) acc[(3 * k + c) * stride] += gcol[c] * Y[k];
}

// dL/ddir = sum_k (gcol . sh_k) dY_k(d), reading the coefficients in
// groups of four basis functions (three float4) when the rows allow it
template <int D>
__device__ __forceinline__ void sh_dir_adjoint(float x, float y, float z, const float (&gcol)[3], const float *sh,
                                               bool vec, float (&gd)[3]) {
    constexpr int K = (D + 1) * (D + 1);
    float Y[16], dY[16][3];
    sh_eval<D, true>(x, y, z, Y, dY);
    gd[0] = gd[1] = gd[2] = 0.f;
    if constexpr (K % 4 == 0) {
        if (vec) {
            const float4 *s4 = reinterpret_cast<const float4 *>(sh);
#pragma unroll
            for (int q = 0; q < K / 4; q++) {
                const float4 a = s4[3 * q], b = s4[3 * q + 1], c = s4[3 * q + 2];
                const float s[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const float w = gcol[0] * s[3 * j] + gcol[1] * s[3 * j + 1] + gcol[2] * s[3 * j + 2];
                    gd[0] += w * dY[4 * q + j][0];
                    gd[1] += w * dY[4 * q + j][1];
                    gd[2] += w * dY[4 * q + j][2];
                }
            }
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
        const float w = gcol[0] * sh[3 * k] + gcol[1] * sh[3 * k + 1] + gcol[2] * sh[3 * k + 2];
        gd[0] += w * dY[k][0];
        gd[1] += w * dY[k][1];
        gd[2] += w * dY[k][2];
    }
}

// The per-item gradients other than the SH coefficients' (17 floats).
struct SmallGrads {
    float mu[3], vel[3], scale[3], quat[4], tau, beta, period, opac;
};
constexpr int kSmall = 17;

// Adjoint of the projection and colour of visible item i of view V, from
// the image-space gradients of its depth position m.  The SH coefficients'
// gradients go to V.g_sh directly (written, or accumulated with `atomic`),
// or, with sh_acc, are added to sh_acc[(3 k + c) * sh_stride]; the others
// are returned.  False if the projection culls the item (then nothing is
// written).
template <int D>
__device__ __forceinline__ bool item_adjoint(const Params &P, const ViewDesc &V, uint32_t i, uint32_t m,
                                             bool atomic, SmallGrads &out, float *sh_acc = nullptr,
                                             int sh_stride = 0) {
    constexpr int K = (D + 1) * (D + 1);
    Fwd F;
    if (!project(V, i, P.dilation, P.tile_w, P.tile_h, F)) return false;
    const float *G2 = P.g2d + 10 * (size_t)m;
    const float gu = G2[0], gv = G2[1], ga = G2[2], gb = G2[3], gc = G2[4];
    const float got = G2[5], gz = G2[9];
    float gmut[3] = {0.f, 0.f, 0.f};
    float gp[3] = {0.f, 0.f, 0.f};
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
        out.quat[0] = (gw - F.qn[0] * dot) * F.qinv;
        out.quat[1] = (gx - F.qn[1] * dot) * F.qinv;
        out.quat[2] = (gy - F.qn[2] * dot) * F.qinv;
        out.quat[3] = (gzq - F.qn[3] * dot) * F.qinv;
        for (int k = 0; k < 3; k++) out.scale[k] = gsc[k];
    }
    // ---- p = W mu~ + T
    {
        const float *R = V.R;
        for (int k = 0; k < 3; k++) gmut[k] += R[k] * gp[0] + R[3 + k] * gp[1] + R[6 + k] * gp[2];
    }
    // ---- colour: rgb = max(0, sum_k sh_k Y_k(d) + 0.5).  The compositor's
    // adjoint already zeroed the colour terms where the forward clamped;
    // two streaming passes over the coefficients (dL/dsh from Y, then
    // dL/ddir from dY) keep few values live at a time.
    {
        const float gcol[3] = {G2[6], G2[7], G2[8]};
        float dx = F.mut.x - V.campos[0], dy = F.mut.y - V.campos[1], dz = F.mut.z - V.campos[2];
        const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
        const float inv = 1.0f / dist;
        dx *= inv; dy *= inv; dz *= inv;
        const float *shp = V.sh + (size_t)i * K * 3;
        const bool vec = aligned16(V.sh) && (!V.g_sh || aligned16(V.g_sh));
        if (sh_acc) sh_coef_accumulate<D>(dx, dy, dz, gcol, sh_acc, sh_stride);
        else if (V.g_sh) sh_coef_adjoint<D>(dx, dy, dz, gcol, V.g_sh + (size_t)i * K * 3, vec, atomic);
        float gd[3];
        sh_dir_adjoint<D>(dx, dy, dz, gcol, shp, vec, gd);
        const float dot = dx * gd[0] + dy * gd[1] + dz * gd[2];
        gmut[0] += (gd[0] - dx * dot) * inv;
        gmut[1] += (gd[1] - dy * dot) * inv;
        gmut[2] += (gd[2] - dz * dot) * inv;
    }
    // ---- time evaluation (Eq. 6 / Eq. 7)
    {
        const float3 vel = ld3(V.vel, i);
        const float l = V.period[i], beta = V.beta[i];
        const float gvd = gmut[0] * vel.x + gmut[1] * vel.y + gmut[2] * vel.z;
        for (int k = 0; k < 3; k++) {
            out.mu[k] = gmut[k];
            out.vel[k] = gmut[k] * F.amp;
        }
        const float ib2 = 1.0f / (beta * beta);
        out.tau = -F.cs * gvd + got * F.ot * F.delta * ib2;
        // flow shift dt v exp(-beta / (2 l)): its beta and l terms
        const float gsh = gvd * V.dt * F.vbw;
        out.period = gvd * (F.sn * kInv2Pi - F.delta / l * F.cs) + gsh * (0.5f * beta / (l * l));
        out.opac = got * F.egate;
        out.beta = got * F.ot * F.delta * F.delta * ib2 / beta - gsh * (0.5f / l);
    }
    return true;
}

// Several views of one scene: one thread per Gaussian walks the views
// that see it (found 64 at a time from the inverse map, coalesced across
// the warp), accumulates the item adjoints over those views -- the 17 small
// gradients in registers, the SH-coefficient gradients in a column of
// shared memory -- and writes every gradient entry once: no atomics and no
// zeroing pass.  Warps take 32 consecutive Gaussians at a time.
constexpr int kViewsThreads = 128;

template <int D>
__global__ void __launch_bounds__(kViewsThreads) k_preprocess_bwd_views(Params P) {
    pdl_enter();
    constexpr int K = (D + 1) * (D + 1);
    extern __shared__ float s_sh[];  // [3 K][kViewsThreads]
    const int tid = threadIdx.x;
    const ViewDesc &V0 = P.views[0];  // every view renders the same scene (gradient pointers too)
    const uint32_t n = V0.n;
    float *col = V0.g_sh ? s_sh + tid : nullptr;
    // a warp's first 32 Gaussians by its index, the next ones from a ticket
    // (counters[3], reset by the adjoint's first kernel): the Gaussians seen
    // by more views cost more, and the warps done first take more
    constexpr uint32_t kWarps = kViewsThreads / 32;
    const int lane = tid & 31;
    uint32_t w = blockIdx.x * kWarps + (uint32_t)(tid >> 5);
    for (;;) {
        const uint32_t i = w * 32u + (uint32_t)lane;
        if (w * 32u >= n) break;
        {
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(&P.counters[3], 1u);
            w = __shfl_sync(0xffffffffu, t, 0) + gridDim.x * kWarps;
        }
        if (i >= n) continue;
        SmallGrads acc = SmallGrads{};
        if (col)
#pragma unroll
            for (int c = 0; c < 3 * K; c++) col[c * kViewsThreads] = 0.f;
        for (int v0 = 0; v0 < P.n_views; v0 += 64) {
            const int vn = min(64, P.n_views - v0);
            unsigned long long mask = 0ull;
            for (int v = 0; v < vn; v++)
                if (P.inv[P.views[v0 + v].item_base + i] != 0xffffffffu) mask |= 1ull << v;
            while (mask) {
                const int v = __ffsll((long long)mask) - 1;
                mask &= mask - 1ull;
                const ViewDesc &V = P.views[v0 + v];
                SmallGrads q;
                if (!item_adjoint<D>(P, V, i, P.inv[V.item_base + i], false, q, col, kViewsThreads)) continue;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    acc.mu[k] += q.mu[k];
                    acc.vel[k] += q.vel[k];
                    acc.scale[k] += q.scale[k];
                }
#pragma unroll
                for (int k = 0; k < 4; k++) acc.quat[k] += q.quat[k];
                acc.tau += q.tau;
                acc.beta += q.beta;
                acc.period += q.period;
                acc.opac += q.opac;
            }
        }
        if (V0.g_mu) for (int k = 0; k < 3; k++) V0.g_mu[3 * (size_t)i + k] = acc.mu[k];
        if (V0.g_vel) for (int k = 0; k < 3; k++) V0.g_vel[3 * (size_t)i + k] = acc.vel[k];
        if (V0.g_scale) for (int k = 0; k < 3; k++) V0.g_scale[3 * (size_t)i + k] = acc.scale[k];
        if (V0.g_quat) for (int k = 0; k < 4; k++) V0.g_quat[4 * (size_t)i + k] = acc.quat[k];
        if (V0.g_tau) V0.g_tau[i] = acc.tau;
        if (V0.g_beta) V0.g_beta[i] = acc.beta;
        if (V0.g_period) V0.g_period[i] = acc.period;
        if (V0.g_opac) V0.g_opac[i] = acc.opac;
        if (col) {
            float g[3 * K];
#pragma unroll
            for (int c = 0; c < 3 * K; c++) g[c] = col[c * kViewsThreads];
            store_floats<3 * K>(V0.g_sh + (size_t)i * 3 * K, g, aligned16(V0.g_sh));
        }
    }
}

// One view: every gradient entry is written once, with no block barrier.
// A warp takes chunks of kWarpChunk consecutive items (its first by its
// index, the others from a ticket): their visibility by ballot, the
// visible items compacted onto its lanes, the 17 small gradients of the
// chunk staged in the warp's shared memory in the global arrays' own
// layout (zeros for the invisible items) and copied out as float4, so that
// each 32-byte sector is written whole and no index is divided.
// SH-coefficient rows (192 bytes at degree 3) are written by the visible
// item's lane, and zeroed warp-wide as float4 for the invisible items.
constexpr int kWarpChunk = 64;
constexpr int kWarpPer = kWarpChunk / 32;
// offsets of the staged fields in a warp's buffer (floats): mu, v, s (3 per
// item), q (4), tau, beta, l, o (1)
constexpr int kStMu = 0, kStVel = 3 * kWarpChunk, kStScale = 6 * kWarpChunk, kStQuat = 9 * kWarpChunk,
              kStOne = 13 * kWarpChunk;

// dst[0, n) = src[0, n) by one warp (float4 where both allow it)
__device__ __forceinline__ void warp_copy_out(float *dst, const float *src, uint32_t n, int lane) {
    if (!dst) return;
    if (aligned16(dst) && (n & 3u) == 0) {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (uint32_t e = lane; e < n / 4; e += 32) d4[e] = s4[e];
    } else {
        for (uint32_t e = lane; e < n; e += 32) dst[e] = src[e];
    }
}

__device__ __forceinline__ void stage_small(float *st, int idx, const SmallGrads &q) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        st[kStMu + 3 * idx + c] = q.mu[c];
        st[kStVel + 3 * idx + c] = q.vel[c];
        st[kStScale + 3 * idx + c] = q.scale[c];
    }
#pragma unroll
    for (int c = 0; c < 4; c++) st[kStQuat + 4 * idx + c] = q.quat[c];
    st[kStOne + idx] = q.tau;
    st[kStOne + kWarpChunk + idx] = q.beta;
    st[kStOne + 2 * kWarpChunk + idx] = q.period;
    st[kStOne + 3 * kWarpChunk + idx] = q.opac;
}

template <int D>
__global__ void __launch_bounds__(256, 3) k_preprocess_bwd(Params P) {
    pdl_enter();
    constexpr int K = (D + 1) * (D + 1);
    __shared__ __align__(16) float s_gw[8][kSmall * kWarpChunk];
    __shared__ uint32_t s_mw[8][kWarpChunk];  // depth positions of the compacted items
    __shared__ uint8_t s_lw[8][kWarpChunk];   // their places in the chunk
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *st = s_gw[warp];
    uint32_t *s_mpos = s_mw[warp];
    uint8_t *s_list = s_lw[warp];
    const ViewDesc &V = P.views[0];  // one view: item g is Gaussian g (item_base 0)
    constexpr bool kRows4 = (3 * K) % 4 == 0;
    const bool rows4 = kRows4 && V.g_sh && aligned16(V.g_sh);
    const uint32_t n = P.n_items;
    const uint32_t lmask = (1u << lane) - 1u;
    const uint32_t n_chunks = (n + kWarpChunk - 1) / kWarpChunk;
    const SmallGrads zero{};
    // A warp's first chunk is blockIdx.x * 8 + warp; after that it takes
    // the next untaken one from a ticket (counters[3], reset by the
    // adjoint's first kernel), so that warps whose chunks hold fewer visible
    // items take more of them.  The inverse map of a warp's next chunk is
    // loaded while it works on the current one (its depth positions start
    // the chunk's dependent loads).
    uint32_t m_next[kWarpPer];
    auto load_inv = [&](uint32_t c, uint32_t (&m)[kWarpPer]) {
#pragma unroll
        for (int q = 0; q < kWarpPer; q++) {
            const uint32_t g = c * kWarpChunk + 32 * q + lane;
            m[q] = g < n ? P.inv[g] : 0xffffffffu;
        }
    };
    auto take = [&]() {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&P.counters[3], 1u);
        return __shfl_sync(0xffffffffu, t, 0) + gridDim.x * 8u;
    };
    uint32_t c = blockIdx.x * 8u + warp;
    if (c < n_chunks) load_inv(c, m_next);
    while (c < n_chunks) {
        const uint32_t base = c * kWarpChunk;
        uint32_t m_cur[kWarpPer];
#pragma unroll
        for (int q = 0; q < kWarpPer; q++) m_cur[q] = m_next[q];
        const uint32_t c_next = take();
        if (c_next < n_chunks) load_inv(c_next, m_next);
        uint64_t vis = 0;  // bit k: item base + k is visible
        uint32_t nvis = 0;
#pragma unroll
        for (int q = 0; q < kWarpPer; q++) {
            const uint32_t g = base + 32 * q + lane;
            const uint32_t m = m_cur[q];
            const bool v = m != 0xffffffffu;
            const uint32_t b = __ballot_sync(0xffffffffu, v);
            vis |= (uint64_t)b << (32 * q);
            if (v) {
                const uint32_t r = nvis + __popc(b & lmask);
                s_mpos[r] = m;
                s_list[r] = (uint8_t)(32 * q + lane);
            } else {
                stage_small(st, 32 * q + lane, zero);
                if (g < n && V.g_sh && !rows4) {
                    float z[3 * K];
#pragma unroll
                    for (int k = 0; k < 3 * K; k++) z[k] = 0.f;
                    store_floats<3 * K>(V.g_sh + (size_t)g * 3 * K, z, aligned16(V.g_sh));
                }
            }
            nvis += __popc(b);
        }
        if constexpr (kRows4) {
            if (rows4) {  // SH rows of the invisible items, warp-wide; float4 e is row e / R4
                constexpr uint32_t R4 = 3 * K / 4;
                float4 *sh4 = reinterpret_cast<float4 *>(V.g_sh + (size_t)base * 3 * K);
                const uint32_t cn4 = min((uint32_t)kWarpChunk, n - base) * R4;
                uint32_t item = (uint32_t)lane / R4, rem = (uint32_t)lane % R4;
                for (uint32_t e = lane; e < cn4; e += 32) {
                    if (!((vis >> item) & 1u)) sh4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
                    item += 32u / R4;
                    rem += 32u % R4;
                    if (rem >= R4) {
                        rem -= R4;
                        item++;
                    }
                }
            }
        }
        __syncwarp();
        // the visible items, compacted
        for (uint32_t k = lane; k < nvis; k += 32) {
            const int idx = s_list[k];
            const uint32_t i = base + idx;
            SmallGrads q;
            if (!item_adjoint<D>(P, V, i, s_mpos[k], false, q)) {  // culled after all: zeros
                q = zero;
                if (V.g_sh) {
                    float z[3 * K];
#pragma unroll
                    for (int cc = 0; cc < 3 * K; cc++) z[cc] = 0.f;
                    store_floats<3 * K>(V.g_sh + (size_t)i * 3 * K, z, aligned16(V.g_sh));
                }
            }
            stage_small(st, idx, q);
        }
        __syncwarp();
        // the chunk's small gradients, copied out
        const uint32_t cn = min((uint32_t)kWarpChunk, n - base);
        warp_copy_out(V.g_mu ? V.g_mu + 3 * (size_t)base : nullptr, st + kStMu, 3 * cn, lane);
        warp_copy_out(V.g_vel ? V.g_vel + 3 * (size_t)base : nullptr, st + kStVel, 3 * cn, lane);
        warp_copy_out(V.g_scale ? V.g_scale + 3 * (size_t)base : nullptr, st + kStScale, 3 * cn, lane);
        warp_copy_out(V.g_quat ? V.g_quat + 4 * (size_t)base : nullptr, st + kStQuat, 4 * cn, lane);
        float *const one[4] = {V.g_tau, V.g_beta, V.g_period, V.g_opac};
#pragma unroll
        for (int f = 0; f < 4; f++)
            warp_copy_out(one[f] ? one[f] + base : nullptr, st + kStOne + f * kWarpChunk, cn, lane);
        __syncwarp();  // the next chunk restages
        c = c_next;
    }
}

}  // namespace

void launch_preprocess_bwd(const Params &p, bool several_views, cudaStream_t s) {
    note_launch();
    if (several_views) {
        // the host copy of the views: every view has the scene's n items
        const uint32_t n = p.n_views > 0 ? p.n_items / (uint32_t)p.n_views : 0u;
        uint32_t grid = (n + kViewsThreads - 1) / kViewsThreads;
        const uint32_t cap = 16u * (uint32_t)device_sm_count();
        if (grid > cap) grid = cap;
        if (grid < 1) grid = 1;
        const size_t smem = sizeof(float) * 3 * (p.sh_degree + 1) * (p.sh_degree + 1) * kViewsThreads;
        switch (p.sh_degree) {
            case 0: pdl_launch(k_preprocess_bwd_views<0>, grid, kViewsThreads, smem, s, p); break;
            case 1: pdl_launch(k_preprocess_bwd_views<1>, grid, kViewsThreads, smem, s, p); break;
            case 2: pdl_launch(k_preprocess_bwd_views<2>, grid, kViewsThreads, smem, s, p); break;
            default: pdl_launch(k_preprocess_bwd_views<3>, grid, kViewsThreads, smem, s, p); break;
        }
        return;
    }
    // persistent: three blocks of 8 warps per SM
    const uint32_t chunks = (p.n_items + kWarpChunk - 1) / kWarpChunk;
    int grid = (int)((chunks + 7) / 8);
    if (grid > 3 * device_sm_count()) grid = 3 * device_sm_count();
    if (grid < 1) grid = 1;
    switch (p.sh_degree) {
        case 0: pdl_launch(k_preprocess_bwd<0>, grid, 256, 0, s, p); break;
        case 1: pdl_launch(k_preprocess_bwd<1>, grid, 256, 0, s, p); break;
        case 2: pdl_launch(k_preprocess_bwd<2>, grid, 256, 0, s, p); break;
        default: pdl_launch(k_preprocess_bwd<3>, grid, 256, 0, s, p); break;
    }
}

}  // namespace pvg

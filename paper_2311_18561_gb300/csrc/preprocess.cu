// preprocess.cu -- per-(view, Gaussian) kernels of the PVG rasterizer.
//
//   k_project_count  (stage a, pass 1) time evaluation (Sec. 3.2, Eq. 6-7),
//                    view transform and culls, 3D covariance from (s, q),
//                    EWA projection (Sec. 3.1, Eq. 2) and the tile
//                    footprint; writes the tile count and depth bits of
//                    every item.
//   k_finalize       (stage a, pass 2) for every visible item, in depth
//                    order: pass 1's stored projection plus the SH colour; writes
//                    the 48-byte compositing record, the tile rectangle and
//                    the count of its tiles that the footprint ellipse
//                    meets, at the item's depth position m.
//
// Pass 1 stores each visible item's projection (64 bytes, item order) and
// pass 2 reads it back, so both use the same bits.  Every kernel is HBM-bound: one
// thread per item, grid-stride.  The adjoint is in preprocess_bwd.cu.
#include "preprocess_common.cuh"

namespace pvg {

cudaError_t set_sh_constants() {
    float h[10];
    sh_constant_values(h);
    const cudaError_t e = cudaMemcpyToSymbol(c_sh, h, sizeof(h));
    return e != cudaSuccess ? e : set_sh_constants_bwd();
}

namespace {

__global__ void __launch_bounds__(256) k_project_count(Params P) {
    pdl_enter();
    const uint32_t n = P.n_items;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const int view = view_of_item(P.views, P.n_views, g);
        const ViewDesc &V = P.views[view];
        Fwd F;
        const bool vis = project(V, g - V.item_base, P.dilation, P.tile_w, P.tile_h, F);
        P.item_cnt[g] = vis ? F.count : 0u;
        if (vis) {
            P.item_zkey[g] = __float_as_uint(F.p.z);
            // what the finalize pass needs of the projection, so that it
            // reads 64 bytes instead of the item's parameters again
            float4 *q = P.proj + 4 * (size_t)g;
            q[0] = make_float4(F.u, F.v, F.ca, F.cb);
            q[1] = make_float4(F.cc, F.ot, F.hx, F.hy);
            q[2] = make_float4(F.mut.x, F.mut.y, F.mut.z, __uint_as_float(F.tx0 | (F.ty0 << 16)));
            q[3] = make_float4(__uint_as_float(F.tx1 | (F.ty1 << 16)), 0.f, 0.f, 0.f);
        }
    }
}

// Records in depth order, one thread per depth position m (item g =
// sgid[m]): the writes are coalesced, and the reads of g's stored
// projection (64 bytes) and SH row (192 bytes at degree 3) are whole
// sectors in any order.
template <int D>
__global__ void __launch_bounds__(256, 4) k_finalize(Params P) {
    pdl_enter();
    constexpr int K = (D + 1) * (D + 1);
    const uint32_t M = P.counters[0];
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const uint32_t g = P.sgid[m];
        const int view = view_of_item(P.views, P.n_views, g);
        const ViewDesc &V = P.views[view];
        const uint32_t i = g - V.item_base;
        // the projection as pass 1 computed and stored it
        const float4 *pq = P.proj + 4 * (size_t)g;
        const float4 q0 = pq[0], q1 = pq[1], q2 = pq[2], q3 = pq[3];
        Fwd F;
        F.u = q0.x; F.v = q0.y; F.ca = q0.z; F.cb = q0.w;
        F.cc = q1.x; F.ot = q1.y; F.hx = q1.z; F.hy = q1.w;
        F.mut = make_float3(q2.x, q2.y, q2.z);
        const uint32_t r0 = __float_as_uint(q2.w), r1 = __float_as_uint(q3.x);
        F.tx0 = r0 & 0xffffu; F.ty0 = r0 >> 16; F.tx1 = r1 & 0xffffu; F.ty1 = r1 >> 16;
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
        // tiles of the rectangle that the footprint ellipse meets
        const FootprintEllipse E = footprint_ellipse(F.u, F.v, F.ca, F.cb, F.cc, F.ot);
        const bool tab = has_row_table(F.tx0, F.ty0, F.tx1, F.ty1);
        if (!tab) store_ellipse(P.ell, m, E);  // the expansion recomputes these rows
        uint32_t cnt = 0, w0 = 0, w1 = 0, w2 = 0, w3 = 0;
        for (uint32_t ty = F.ty0; ty < F.ty1; ty++) {
            const uint2 c = footprint_cols(E, ty, P.tile_w, P.tile_h, F.tx0, F.tx1);
            cnt += c.y - c.x;
            const uint32_t i = ty - F.ty0;
            const uint32_t v = ((c.x - F.tx0) | ((c.y - c.x) << 8)) << (16 * (i & 1));
            w0 |= i >> 1 == 0 ? v : 0u;
            w1 |= i >> 1 == 1 ? v : 0u;
            w2 |= i >> 1 == 2 ? v : 0u;
            w3 |= i >> 1 == 3 ? v : 0u;
        }
        if (tab) P.rowtab[m] = make_uint4(w0, w1, w2, w3);
        P.vis_cnt[m] = cnt;
    }
}

}  // namespace

void launch_project_count(const Params &p, cudaStream_t s) {
    note_launch();
    pdl_launch(k_project_count, grid_for(p.n_items), 256, 0, s, p);
}

void launch_finalize(const Params &p, cudaStream_t s) {
    note_launch();
    switch (p.sh_degree) {
        case 0: pdl_launch(k_finalize<0>, grid_for(p.n_items), 256, 0, s, p); break;
        case 1: pdl_launch(k_finalize<1>, grid_for(p.n_items), 256, 0, s, p); break;
        case 2: pdl_launch(k_finalize<2>, grid_for(p.n_items), 256, 0, s, p); break;
        default: pdl_launch(k_finalize<3>, grid_for(p.n_items), 256, 0, s, p); break;
    }
}

}  // namespace pvg

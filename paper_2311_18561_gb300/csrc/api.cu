// api.cu -- the C ABI of include/pvg.h: contexts, frames and the forward /
// backward orchestration of the four stages.
//
// Forward pass on one stream (no host round trip except the optional pair
// count read-back that sizes the pair buffers):
//   a  k_project_count      items -> tile count, depth bits, projection
//      compact_visible      visible items in gid order -> (zbits, gid), M
//   b  radix sort           by depth bits (4 passes of <= 8 bits); the last
//                           pass also writes inv[gid] = depth position
//   a  k_finalize           records, rects, counts in depth order
//   b  scan + emit          (tile, m) pairs in depth order, K
//      radix sort           by tile id (ceil(log2 tiles) bits)
//      k_ranges             [start, end) per tile
//   c  k_composite          images + per-pixel T and last position
// Backward: k_composite_bwd (image-space gradients per record) and
// k_preprocess_bwd (parameter gradients).
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pvg.h"
#include "pvg_internal.cuh"

using namespace pvg;

namespace pvg {
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static constexpr int kMaxSmDevices = 64;
static std::atomic<int> g_sm_count[kMaxSmDevices];

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxSmDevices) {
        cudaGetLastError();
        return 1;
    }
    int v = g_sm_count[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 1;
        }
        g_sm_count[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}
}  // namespace pvg

namespace {

thread_local std::string g_last_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

void release(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// test hook: the next g_fail_allocs device allocations fail (PVG_ERR_OOM)
std::atomic<int> g_fail_allocs{0};

bool injected_alloc_failure() {
    int n = g_fail_allocs.load();
    while (n > 0)
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) return true;
    return false;
}

// grow to at least `bytes` (x1.25 headroom); contents are not kept
pvg_status_t ensure(DevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return PVG_OK;
    release(b);
    if (injected_alloc_failure()) {
        g_last_error = "device allocation failed (injected)";
        return PVG_ERR_OOM;
    }
    const size_t want = bytes + bytes / 4;
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return PVG_ERR_OOM;
        }
        b.bytes = bytes;
        return PVG_OK;
    }
    b.bytes = want;
    return PVG_OK;
}

// ensure() that refuses to allocate while the stream is being captured
pvg_status_t ensure_c(DevBuf &b, size_t bytes, bool capturing) {
    if (capturing) return b.bytes >= (bytes ? bytes : 16) ? PVG_OK : PVG_ERR_INVALID;
    return ensure(b, bytes);
}

template <class T>
T *ptr(DevBuf &b) { return reinterpret_cast<T *>(b.p); }

pvg_status_t cuda_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return PVG_OK;
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return PVG_ERR_CUDA;
}

#define PVG_TRY(expr)                              \
    do {                                           \
        pvg_status_t _s = (expr);                  \
        if (_s != PVG_OK) return _s;               \
    } while (0)

#define PVG_CUDA(expr) PVG_TRY(cuda_status((expr), #expr))

// CUDA-event timing of the stages of each call, on the call's stream.
struct StageTimer {
    bool on = false;
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> pending;
    cudaEvent_t open[PVG_NUM_STAGES] = {};
    cudaEvent_t get() {
        cudaEvent_t e = nullptr;
        if (!pool.empty()) {
            e = pool.back();
            pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
        }
        return e;
    }
    void begin(int st, cudaStream_t s) {
        if (!on) return;
        open[st] = get();
        if (open[st]) cudaEventRecord(open[st], s);
    }
    void end(int st, cudaStream_t s) {
        if (!on || !open[st]) return;
        cudaEvent_t b = get();
        if (!b) return;
        cudaEventRecord(b, s);
        pending.push_back({st, open[st], b});
        open[st] = nullptr;
    }
    void destroy() {
        for (auto &r : pending) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
        pending.clear();
        pool.clear();
    }
};

}  // namespace

struct ViewStage;
void free_stage_ptr(ViewStage *st);
ViewStage *new_stage();

struct pvg_frame {
    int device = -1;
    ViewStage *stage_fwd = nullptr, *stage_bwd = nullptr;
    DevBuf counters;            // u32 [4]: M, K, overflow, the per-item adjoint's chunk ticket
    DevBuf sgid, szkey;         // [NV]
    DevBuf inv;                 // [NV] depth position per item
    DevBuf rec;                 // [NV * 3] float4
    DevBuf ell;                 // [NV * 2] float4 footprint ellipses
    DevBuf rowtab;              // [NV] uint4 packed tile rows
    DevBuf rect, vis_cnt;       // [NV]
    DevBuf pair_vals;           // [K]
    DevBuf ranges;              // [tiles]
    DevBuf tile_order;          // [tiles] compositor launch order
    DevBuf tile_walk;           // [tiles] largest last-blend position per tile (forward)
    DevBuf tile_order_bwd;      // [tiles] adjoint launch order (by walk)
    DevBuf pix_T, pix_last;     // [pixels]
    DevBuf pix_neval;           // [pixels]
    DevBuf g2d;                 // [NV * 10] image-space gradients by depth position
    DevBuf gfeat;               // [NV * F] dL/d(channel value)
    std::vector<ViewDesc> views;
    int feat_mask = 0, n_feat = 0, n_sem = 0;  // extra channels of the forward
    bool one_scene = true;      // every view renders the same scene
    uint32_t n_items = 0, total_tiles = 0, total_pix = 0, pair_capacity = 0;
    int tile_w = 0, tile_h = 0, px = 1;
    int64_t n = -1;
    int sh_degree = -1;
    float dilation = 0.f;
    cudaStream_t stream = nullptr;
    bool valid = false;
    bool has_state = false;     // the last forward kept what the backward needs
    uint32_t *h_counters = nullptr;  // pinned
};

struct pvg_ctx {
    int device = -1;
    pvg_config_t cfg;
    DevBuf views;
    DevBuf item_cnt, item_zkey;  // [NV]
    DevBuf proj;                 // [NV * 4] float4: projections from pass 1 to pass 2
    DevBuf alt_keys, alt_vals;   // [NV] depth sort ping-pong
    DevBuf pair_keys, pair_keys2, pair_vals2;  // [K]
    DevBuf vis_off;              // [NV]
    DevBuf chunk_start;          // [K / 2048 + 1]
    DevBuf temp;
    DevBuf sort_n;               // u32: element count of pvg_sort_pairs
    DevBuf loss_partials;        // float2 per CTA of pvg_rgb_loss
    DevBuf l1_scratch;           // pvg_l1_loss: ticket counter + per-block partial sums
    uint32_t *h_pinned = nullptr;
    pvg_frame *own_frame = nullptr;
    StageTimer timer;
};

// ------------------------------------------------------------------ misc

extern "C" const char *pvg_status_str(pvg_status_t s) {
    switch (s) {
        case PVG_OK: return "PVG_OK";
        case PVG_ERR_INVALID: return "PVG_ERR_INVALID";
        case PVG_ERR_OOM: return "PVG_ERR_OOM";
        case PVG_ERR_BUSY: return "PVG_ERR_BUSY";
        case PVG_ERR_TIMEOUT: return "PVG_ERR_TIMEOUT";
        case PVG_ERR_CUDA: return "PVG_ERR_CUDA";
        case PVG_ERR_OVERFLOW: return "PVG_ERR_OVERFLOW";
        case PVG_ERR_NOT_FOUND: return "PVG_ERR_NOT_FOUND";
    }
    return "PVG_ERR_UNKNOWN";
}

extern "C" const char *pvg_last_error(void) { return g_last_error.c_str(); }

extern "C" int pvg_version(void) { return 100; }

extern "C" void pvg_debug_fail_allocations(int32_t n) { g_fail_allocs.store(n > 0 ? n : 0); }

extern "C" void pvg_config_default(pvg_config_t *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->pixels_per_thread = 1;
    cfg->sync_sizes = 1;
    cfg->pair_capacity = 1 << 24;
    cfg->dilation = 0.3f;
    cfg->fov_clamp = 1.3f;
}

static pvg_status_t check_config(const pvg_config_t *c) {
    const int px = c->pixels_per_thread ? c->pixels_per_thread : 1;
    if (!composite_supported(c->tile_w, c->tile_h, px)) return PVG_ERR_INVALID;
    if (!(c->dilation >= 0.f) || !(c->fov_clamp > 0.f)) return PVG_ERR_INVALID;
    if (!c->sync_sizes && (c->pair_capacity <= 0 || c->pair_capacity > 0xfffffff0LL)) return PVG_ERR_INVALID;
    return PVG_OK;
}

extern "C" pvg_status_t pvg_frame_create(pvg_frame_t **frame) {
    if (!frame) return PVG_ERR_INVALID;
    pvg_frame *f = new pvg_frame();
    PVG_CUDA(cudaGetDevice(&f->device));
    f->stage_fwd = new_stage();
    f->stage_bwd = new_stage();
    if (cudaMallocHost(&f->h_counters, 4 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        delete f;
        return PVG_ERR_OOM;
    }
    if (ensure(f->counters, 4 * sizeof(uint32_t)) != PVG_OK) {
        cudaFreeHost(f->h_counters);
        delete f;
        return PVG_ERR_OOM;
    }
    *frame = f;
    return PVG_OK;
}

extern "C" void pvg_frame_destroy(pvg_frame_t *f) {
    if (!f) return;
    if (f->stream) cudaStreamSynchronize(f->stream);
    for (DevBuf *b : {&f->counters, &f->sgid, &f->inv, &f->szkey, &f->rec, &f->ell, &f->rowtab, &f->rect, &f->vis_cnt, &f->pair_vals,
                      &f->ranges, &f->tile_order, &f->tile_walk, &f->tile_order_bwd, &f->pix_T, &f->pix_last, &f->pix_neval, &f->g2d, &f->gfeat})
        release(*b);
    if (f->h_counters) cudaFreeHost(f->h_counters);
    free_stage_ptr(f->stage_fwd);
    free_stage_ptr(f->stage_bwd);
    delete f;
}

extern "C" pvg_status_t pvg_create(pvg_ctx_t **ctx, const pvg_config_t *cfg) {
    if (!ctx) return PVG_ERR_INVALID;
    pvg_config_t c;
    if (cfg) c = *cfg; else pvg_config_default(&c);
    PVG_TRY(check_config(&c));
    pvg_ctx *x = new pvg_ctx();
    x->cfg = c;
    if (cudaGetDevice(&x->device) != cudaSuccess || set_sh_constants() != cudaSuccess) {
        g_last_error = cudaGetErrorString(cudaGetLastError());
        delete x;
        return PVG_ERR_CUDA;
    }
    if (cudaMallocHost(&x->h_pinned, 16) != cudaSuccess) {
        cudaGetLastError();
        delete x;
        return PVG_ERR_OOM;
    }
    if (ensure(x->temp, sort_temp_bytes()) != PVG_OK || pvg_frame_create(&x->own_frame) != PVG_OK) {
        cudaFreeHost(x->h_pinned);
        release(x->temp);
        delete x;
        return PVG_ERR_OOM;
    }
    *ctx = x;
    return PVG_OK;
}

extern "C" void pvg_destroy(pvg_ctx_t *x) {
    if (!x) return;
    cudaDeviceSynchronize();
    for (DevBuf *b : {&x->views, &x->item_cnt, &x->item_zkey, &x->proj, &x->alt_keys, &x->alt_vals, &x->pair_keys,
                      &x->pair_keys2, &x->pair_vals2, &x->temp, &x->sort_n, &x->vis_off, &x->chunk_start,
                      &x->loss_partials, &x->l1_scratch})
        release(*b);
    if (x->h_pinned) cudaFreeHost(x->h_pinned);
    pvg_frame_destroy(x->own_frame);
    x->timer.destroy();
    delete x;
}

extern "C" pvg_status_t pvg_set_config(pvg_ctx_t *x, const pvg_config_t *cfg) {
    if (!x || !cfg) return PVG_ERR_INVALID;
    PVG_TRY(check_config(cfg));
    x->cfg = *cfg;
    return PVG_OK;
}

// ------------------------------------------------------------------ views

static bool finite3x4(const float *m) {
    for (int k = 0; k < 12; k++)
        if (!std::isfinite(m[k])) return false;
    return true;
}

static pvg_status_t validate_scene(const pvg_scene_t *sc) {
    if (!sc || sc->n < 0 || sc->sh_degree < 0 || sc->sh_degree > 3) return PVG_ERR_INVALID;
    if (sc->sky && (sc->sky_res < 1 || sc->sky_res > 16384)) return PVG_ERR_INVALID;
    if (sc->sem && (sc->n_sem < 1 || sc->n_sem > kMaxSem)) return PVG_ERR_INVALID;
    if (sc->n > 0 && (!sc->mu || !sc->vel || !sc->tau || !sc->beta || !sc->period || !sc->scale || !sc->quat ||
                      !sc->opacity || !sc->sh))
        return PVG_ERR_INVALID;
    return PVG_OK;
}

// Per-view descriptors.  Scene of view v = scenes[v * scene_stride]
// (stride 0: one scene for every view).  Items of view v are
// [item_base, item_base + n_v), item_base = sum of the earlier views' n.
static pvg_status_t build_views(const pvg_ctx *x, const pvg_scene_t *scenes, int scene_stride,
                                const pvg_camera_t *cams, int nv, std::vector<ViewDesc> &out, uint32_t *n_items,
                                uint32_t *total_tiles, uint32_t *total_pix) {
    if (!cams || !scenes || nv < 1 || nv > kMaxViewsPerCall) return PVG_ERR_INVALID;
    const int TW = x->cfg.tile_w, TH = x->cfg.tile_h;
    out.assign(nv, ViewDesc());
    uint64_t tiles = 0, pix = 0, items = 0;
    for (int v = 0; v < nv; v++) {
        const pvg_scene_t *sc = &scenes[(size_t)v * scene_stride];
        PVG_TRY(validate_scene(sc));
        if (sc->sh_degree != scenes[0].sh_degree) return PVG_ERR_INVALID;
        const pvg_camera_t &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384) return PVG_ERR_INVALID;
        if (!(c.fx > 0.f) || !(c.fy > 0.f) || !std::isfinite(c.fx) || !std::isfinite(c.fy) ||
            !std::isfinite(c.cx) || !std::isfinite(c.cy) || !std::isfinite(c.t) || !(c.z_near >= 0.f) ||
            !std::isfinite(c.z_near) || !finite3x4(c.viewmat))
            return PVG_ERR_INVALID;
        ViewDesc &d = out[v];
        for (int r = 0; r < 3; r++) {
            for (int k = 0; k < 3; k++) d.R[3 * r + k] = c.viewmat[4 * r + k];
            d.T[r] = c.viewmat[4 * r + 3];
        }
        for (int k = 0; k < 3; k++)
            d.campos[k] = -(d.R[k] * d.T[0] + d.R[3 + k] * d.T[1] + d.R[6 + k] * d.T[2]);
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        d.t = c.t; d.znear = c.z_near;
        if (!std::isfinite(c.dt)) return PVG_ERR_INVALID;
        d.dt = c.dt;
        d.bg[0] = c.bg[0]; d.bg[1] = c.bg[1]; d.bg[2] = c.bg[2];
        d.limx = x->cfg.fov_clamp * 0.5f * (float)c.width / c.fx;
        d.limy = x->cfg.fov_clamp * 0.5f * (float)c.height / c.fy;
        d.W = c.width; d.H = c.height;
        d.tiles_x = (c.width + TW - 1) / TW;
        d.tiles_y = (c.height + TH - 1) / TH;
        d.tile_base = (uint32_t)tiles;
        d.pix_base = (uint32_t)pix;
        d.item_base = (uint32_t)items;
        d.n = (uint32_t)sc->n;
        d.sh_degree = sc->sh_degree;
        d.mu = sc->mu; d.vel = sc->vel; d.tau = sc->tau; d.beta = sc->beta; d.period = sc->period;
        d.scale = sc->scale; d.quat = sc->quat; d.opac = sc->opacity; d.sh = sc->sh;
        d.sky = sc->sky;
        d.sky_res = sc->sky_res;
        d.sky_jitter = c.sky_jitter;
        d.sem = sc->sem;
        d.n_sem = sc->n_sem;
        tiles += (uint64_t)d.tiles_x * d.tiles_y;
        pix += (uint64_t)c.width * c.height;
        items += (uint64_t)sc->n;
        if (items >= (1ull << 31)) return PVG_ERR_INVALID;
    }
    if (tiles >= (1ull << 31) || pix >= (1ull << 32)) return PVG_ERR_INVALID;
    *n_items = (uint32_t)items;
    *total_tiles = (uint32_t)tiles;
    *total_pix = (uint32_t)pix;
    return PVG_OK;
}

// Copies the view descriptors to the device through pinned staging owned
// by `stage` (so that the copy can be captured in a CUDA graph).  Outside
// capture, waits for the previous copy from the same staging first.  A
// captured copy reads its source at every replay, so each capture stages
// into a pinned buffer of its own that nothing writes afterwards: later
// uncaptured calls on the frame and later captures (other cameras or
// output images) do not change what an earlier graph renders.  An
// uncaptured call keeps one spare buffer of its size ready, which the next
// capture takes (a capture must follow an uncaptured call of the same
// size); the taken buffers (a few hundred bytes per view) are freed with
// the frame.
struct ViewStage {
    ViewDesc *host = nullptr;  // pinned, uncaptured calls
    size_t cap = 0;
    ViewDesc *spare = nullptr;  // pinned, for the next capture
    size_t spare_cap = 0;
    std::vector<ViewDesc *> captured;  // pinned, one per capture taken so far
    DevBuf dev;
    cudaEvent_t done = nullptr;
    bool pending = false;
};

static pvg_status_t pinned_views(ViewDesc **p, size_t n) {
    if (cudaMallocHost(p, sizeof(ViewDesc) * n) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return PVG_ERR_OOM;
    }
    return PVG_OK;
}

static pvg_status_t stage_views(ViewStage &st, const std::vector<ViewDesc> &views, cudaStream_t s,
                                bool capturing) {
    const size_t n = views.size();
    const size_t bytes = sizeof(ViewDesc) * n;
    ViewDesc *src;
    if (capturing) {  // no allocation while capturing
        if (!st.spare || st.spare_cap < n || st.dev.bytes < bytes || !st.done) return PVG_ERR_INVALID;
        src = st.spare;
        st.captured.push_back(st.spare);
        st.spare = nullptr;
        st.spare_cap = 0;
    } else {
        if (st.pending) {
            PVG_CUDA(cudaEventSynchronize(st.done));
            st.pending = false;
        }
        if (st.cap < n) {
            if (st.host) cudaFreeHost(st.host);
            st.host = nullptr;
            st.cap = 0;
            PVG_TRY(pinned_views(&st.host, n));
            st.cap = n;
        }
        if (st.spare_cap < n) {
            if (st.spare) cudaFreeHost(st.spare);
            st.spare = nullptr;
            st.spare_cap = 0;
            PVG_TRY(pinned_views(&st.spare, n));
            st.spare_cap = n;
        }
        PVG_TRY(ensure(st.dev, bytes));
        if (!st.done) PVG_CUDA(cudaEventCreateWithFlags(&st.done, cudaEventDisableTiming));
        src = st.host;
    }
    std::memcpy(src, views.data(), bytes);
    PVG_CUDA(cudaMemcpyAsync(st.dev.p, src, bytes, cudaMemcpyHostToDevice, s));
    if (!capturing) {
        PVG_CUDA(cudaEventRecord(st.done, s));
        st.pending = true;
    }
    return PVG_OK;
}

ViewStage *new_stage() { return new ViewStage(); }

static void free_stage(ViewStage &st);
void free_stage_ptr(ViewStage *st) {
    if (!st) return;
    free_stage(*st);
    delete st;
}

static void free_stage(ViewStage &st) {
    if (st.pending) cudaEventSynchronize(st.done);
    if (st.host) cudaFreeHost(st.host);
    if (st.spare) cudaFreeHost(st.spare);
    for (ViewDesc *c : st.captured) cudaFreeHost(c);
    if (st.done) cudaEventDestroy(st.done);
    release(st.dev);
    st = ViewStage();
}

static bool is_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

static int bits_for(uint32_t n) {
    if (n <= 1) return 1;
    int b = 0;
    while ((1ull << b) < n) b++;
    return b;
}

// ------------------------------------------------------------------ forward

// The forward launch sequence for views whose host copies are `views`
// (sizes and bases set).  dev_views: NULL stages the host copies into the
// frame (pinned staging, one copy); otherwise the descriptors were already
// written to dev_views on stream s (the render server's gather kernel).
// no_alloc: every buffer must already be large enough (graph capture, or a
// workspace reserved in advance); PVG_ERR_INVALID otherwise.
static pvg_status_t enqueue_forward(pvg_ctx_t *x, pvg_frame *f, std::vector<ViewDesc> &views,
                                    const ViewDesc *dev_views, uint32_t NV, uint32_t tiles, uint32_t pix, int fmask,
                                    int nsem, bool keep_state, bool no_alloc, cudaStream_t s) {
    const bool capturing = no_alloc;
    const int n_views = (int)views.size();
    const int n_feat = fmask ? feat_count(fmask, nsem) : 0;
    // workspace
    PVG_TRY(ensure_c(x->item_cnt, sizeof(uint32_t) * NV, capturing));
    PVG_TRY(ensure_c(x->item_zkey, sizeof(uint32_t) * NV, capturing));
    PVG_TRY(ensure_c(x->proj, sizeof(float4) * 4 * (size_t)NV, capturing));
    PVG_TRY(ensure_c(x->alt_keys, sizeof(uint32_t) * NV, capturing));
    PVG_TRY(ensure_c(x->alt_vals, sizeof(uint32_t) * NV, capturing));
    PVG_TRY(ensure_c(x->vis_off, sizeof(uint32_t) * NV, capturing));
    PVG_TRY(ensure_c(f->sgid, sizeof(uint32_t) * NV, capturing));
    PVG_TRY(ensure_c(f->inv, sizeof(uint32_t) * NV, capturing));
    PVG_TRY(ensure_c(f->szkey, sizeof(uint32_t) * NV, capturing));
    PVG_TRY(ensure_c(f->rec, sizeof(float4) * 3 * (size_t)NV, capturing));
    PVG_TRY(ensure_c(f->ell, sizeof(float4) * 2 * (size_t)NV, capturing));
    PVG_TRY(ensure_c(f->rowtab, sizeof(uint4) * (size_t)NV, capturing));
    PVG_TRY(ensure_c(f->rect, sizeof(uint2) * NV, capturing));
    PVG_TRY(ensure_c(f->vis_cnt, sizeof(uint32_t) * NV, capturing));
    PVG_TRY(ensure_c(f->ranges, sizeof(uint2) * tiles, capturing));
    PVG_TRY(ensure_c(f->tile_order, sizeof(uint32_t) * tiles, capturing));
    PVG_TRY(ensure_c(f->tile_walk, sizeof(uint32_t) * tiles, capturing));
    PVG_TRY(ensure_c(f->tile_order_bwd, sizeof(uint32_t) * tiles, capturing));
    PVG_TRY(ensure_c(f->pix_T, sizeof(float) * pix, capturing));
    PVG_TRY(ensure_c(f->pix_last, sizeof(uint32_t) * pix, capturing));
    PVG_TRY(ensure_c(f->pix_neval, sizeof(uint32_t) * 2 * (size_t)pix, capturing));
    uint32_t pair_cap;
    if (x->cfg.sync_sizes) {
        pair_cap = (uint32_t)(f->pair_vals.bytes / sizeof(uint32_t));
    } else {
        pair_cap = (uint32_t)x->cfg.pair_capacity;
        PVG_TRY(ensure_c(f->pair_vals, sizeof(uint32_t) * (size_t)pair_cap, capturing));
        PVG_TRY(ensure_c(x->pair_keys, sizeof(uint32_t) * (size_t)pair_cap, capturing));
        PVG_TRY(ensure_c(x->pair_keys2, sizeof(uint32_t) * (size_t)pair_cap, capturing));
        PVG_TRY(ensure_c(x->pair_vals2, sizeof(uint32_t) * (size_t)pair_cap, capturing));
        PVG_TRY(ensure_c(x->chunk_start, sizeof(uint32_t) * emit_chunks(pair_cap), capturing));
    }
    f->views = views;
    f->one_scene = true;
    for (int v = 1; v < n_views; v++)
        if (views[v].mu != views[0].mu || views[v].n != views[0].n) f->one_scene = false;
    f->n_items = NV;
    f->total_tiles = tiles;
    f->total_pix = pix;
    f->tile_w = x->cfg.tile_w;
    f->tile_h = x->cfg.tile_h;
    f->px = x->cfg.pixels_per_thread ? x->cfg.pixels_per_thread : 1;
    f->n = views[0].n;
    f->sh_degree = views[0].sh_degree;
    f->dilation = x->cfg.dilation;
    f->stream = s;
    f->valid = false;
    f->has_state = false;
    f->feat_mask = fmask;
    f->n_feat = n_feat;
    f->n_sem = nsem;

    if (!dev_views) PVG_TRY(stage_views(*f->stage_fwd, views, s, capturing));
    PVG_CUDA(cudaMemsetAsync(f->counters.p, 0, 4 * sizeof(uint32_t), s));

    Params p;
    std::memset(&p, 0, sizeof(p));
    p.views = dev_views ? dev_views : ptr<ViewDesc>(f->stage_fwd->dev);
    p.n_views = n_views;
    p.sh_degree = views[0].sh_degree;
    p.tile_w = x->cfg.tile_w;
    p.tile_h = x->cfg.tile_h;
    p.px = f->px;
    p.dilation = x->cfg.dilation;
    p.n_items = NV;
    p.total_tiles = tiles;
    p.counters = ptr<uint32_t>(f->counters);
    p.item_cnt = ptr<uint32_t>(x->item_cnt);
    p.item_zkey = ptr<uint32_t>(x->item_zkey);
    p.proj = ptr<float4>(x->proj);
    p.sgid = ptr<uint32_t>(f->sgid);
    p.inv = ptr<uint32_t>(f->inv);
    p.szkey = ptr<uint32_t>(f->szkey);
    p.rec = ptr<float4>(f->rec);
    p.ell = ptr<float4>(f->ell);
    p.rowtab = ptr<uint4>(f->rowtab);
    p.rect = ptr<uint2>(f->rect);
    p.vis_cnt = ptr<uint32_t>(f->vis_cnt);
    p.ranges = ptr<uint2>(f->ranges);
    p.tile_order = ptr<uint32_t>(f->tile_order);
    p.pix_T = ptr<float>(f->pix_T);
    p.pix_last = ptr<uint32_t>(f->pix_last);
    p.pix_neval = ptr<uint32_t>(f->pix_neval);
    p.vis_off = ptr<uint32_t>(x->vis_off);
    p.feat_mask = fmask;
    p.n_feat = n_feat;
    StageTimer &tm = x->timer;
    const bool timer_on = tm.on;
    if (capturing) tm.on = false;

    if (NV > 0) {
        // (a) project + count, (b) depth sort of the visible items
        tm.begin(PVG_STAGE_PROJECT, s);
        launch_project_count(p, s);
        tm.end(PVG_STAGE_PROJECT, s);
        tm.begin(PVG_STAGE_DEPTH_SORT, s);
        // the inverse map inv[gid] = depth position: 0xffffffff for the
        // invisible items from the compaction, the visible ones' from the
        // sort's last pass; the compaction also counts the sort's first
        // digit histogram
        compact_visible(p, p.szkey, p.sgid, p.inv, x->temp.p, s);
        bool in_alt = false;
        radix_sort_pairs(p.szkey, p.sgid, ptr<uint32_t>(x->alt_keys), ptr<uint32_t>(x->alt_vals), &p.counters[0], NV,
                         0, 31, x->temp.p, s, &in_alt, p.inv, true);
        if (in_alt) {  // 31 bits = 4 passes: never taken, kept for safety
            PVG_CUDA(cudaMemcpyAsync(p.szkey, x->alt_keys.p, sizeof(uint32_t) * NV, cudaMemcpyDeviceToDevice, s));
            PVG_CUDA(cudaMemcpyAsync(p.sgid, x->alt_vals.p, sizeof(uint32_t) * NV, cudaMemcpyDeviceToDevice, s));
        }
        tm.end(PVG_STAGE_DEPTH_SORT, s);
        // (a) records in depth order, (b) pair count
        tm.begin(PVG_STAGE_FINALIZE, s);
        launch_finalize(p, s);
        tm.end(PVG_STAGE_FINALIZE, s);
        tm.begin(PVG_STAGE_PAIRS, s);
        p.pair_capacity = x->cfg.sync_sizes ? 0xffffffffu : pair_cap;
        scan_count_pairs(p, x->temp.p, s);
        if (x->cfg.sync_sizes) {
            PVG_CUDA(cudaMemcpyAsync(x->h_pinned, &p.counters[1], sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            PVG_CUDA(cudaStreamSynchronize(s));
            const uint32_t K = x->h_pinned[0];
            PVG_TRY(ensure_c(f->pair_vals, sizeof(uint32_t) * (size_t)K, capturing));
            PVG_TRY(ensure_c(x->pair_keys, sizeof(uint32_t) * (size_t)K, capturing));
            PVG_TRY(ensure_c(x->pair_keys2, sizeof(uint32_t) * (size_t)K, capturing));
            PVG_TRY(ensure_c(x->pair_vals2, sizeof(uint32_t) * (size_t)K, capturing));
            PVG_TRY(ensure_c(x->chunk_start, sizeof(uint32_t) * emit_chunks(K), capturing));
            pair_cap = K;
        }
        p.pair_capacity = pair_cap;
        p.chunk_start = ptr<uint32_t>(x->chunk_start);
        // emission target so that an odd/even number of tile passes ends in f->pair_vals
        const int tbits = bits_for(tiles);
        const int tpasses = (tbits + 7) / 8;
        uint32_t *E_keys = ptr<uint32_t>(x->pair_keys), *F_keys = ptr<uint32_t>(x->pair_keys2);
        uint32_t *E_vals, *F_vals;
        if (tpasses % 2 == 0) {
            E_vals = ptr<uint32_t>(f->pair_vals);
            F_vals = ptr<uint32_t>(x->pair_vals2);
        } else {
            E_vals = ptr<uint32_t>(x->pair_vals2);
            F_vals = ptr<uint32_t>(f->pair_vals);
        }
        p.pair_keys = E_keys;
        p.pair_vals = E_vals;
        scan_emit_pairs(p, x->temp.p, s);
        tm.end(PVG_STAGE_PAIRS, s);
        tm.begin(PVG_STAGE_TILE_SORT, s);
        bool t_alt = false;
        // the first digit pass's histogram was counted by the expansion
        radix_sort_pairs(E_keys, E_vals, F_keys, F_vals, &p.counters[1], pair_cap, 0, tbits, x->temp.p, s, &t_alt,
                         nullptr, true);
        p.pair_keys = t_alt ? F_keys : E_keys;
        p.pair_vals = ptr<uint32_t>(f->pair_vals);
        launch_ranges(p, s);
        launch_tile_order(p, s);
        tm.end(PVG_STAGE_TILE_SORT, s);
    } else {
        PVG_CUDA(cudaMemsetAsync(p.ranges, 0, sizeof(uint2) * tiles, s));
        launch_tile_order(p, s);
    }
    f->pair_capacity = pair_cap;
    p.pair_vals = ptr<uint32_t>(f->pair_vals);
    if (!keep_state) p.pix_T = nullptr;  // inference only: no state for a backward pass
    // with state: each tile's walk length, from which the adjoint orders its tiles
    p.tile_walk = keep_state ? ptr<uint32_t>(f->tile_walk) : nullptr;
    tm.begin(PVG_STAGE_COMPOSITE, s);
    launch_composite(p, s);
    if (n_feat) launch_composite_feat(p, s);
    tm.end(PVG_STAGE_COMPOSITE, s);
    tm.on = timer_on;
    PVG_CUDA(cudaGetLastError());
    f->valid = true;
    f->has_state = keep_state;
    return PVG_OK;
}

static pvg_status_t render_fwd_impl(pvg_ctx_t *x, const pvg_scene_t *scenes, int scene_stride,
                                    const pvg_camera_t *cams, int32_t n_views, const pvg_image_t *out,
                                    pvg_frame_t *frame, void *stream_) {
    if (!x || !out || !scenes) return PVG_ERR_INVALID;
    for (int v = 0; v < n_views; v++)
        if (!out[v].rgb) return PVG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream_;
    const bool capturing = is_capturing(s);
    if (capturing && x->cfg.sync_sizes) return PVG_ERR_INVALID;  // a graph cannot hold the size read-back
    pvg_frame *f = frame ? frame : x->own_frame;
    std::vector<ViewDesc> views;
    uint32_t NV, tiles, pix;
    PVG_TRY(build_views(x, scenes, scene_stride, cams, n_views, views, &NV, &tiles, &pix));
    const pvg_scene_t *scene = &scenes[0];
    // extra channels: one mask for the call, channel values of every scene
    const int fmask = out[0].feat_mask;
    if (fmask & ~(kFeatVbar | kFeatRho | kFeatSem)) return PVG_ERR_INVALID;
    const int nsem = (fmask & kFeatSem) ? scene->n_sem : 0;
    if ((fmask & kFeatSem) && (nsem < 1 || nsem > kMaxSem)) return PVG_ERR_INVALID;
    for (int v = 0; v < n_views; v++) {
        if (out[v].feat_mask != fmask || (fmask && !out[v].feat)) return PVG_ERR_INVALID;
        if ((fmask & kFeatSem) && ((views[v].n > 0 && !views[v].sem) || views[v].n_sem != nsem))
            return PVG_ERR_INVALID;
    }
    for (int v = 0; v < n_views; v++) {
        views[v].out_rgb = out[v].rgb;
        views[v].out_depth = out[v].depth;
        views[v].out_alpha = out[v].alpha;
        views[v].out_feat = fmask ? out[v].feat : nullptr;
    }
    return enqueue_forward(x, f, views, nullptr, NV, tiles, pix, fmask, nsem, frame != nullptr, capturing, s);
}

// ------------------------------------------------------------------ render-server hooks (serve.cu)

namespace pvg {

pvg_status_t serve_view_desc(pvg_ctx_t *x, const pvg_scene_t *scene, const pvg_camera_t *cam, const pvg_image_t *dst,
                             ViewDesc *out, uint32_t *tiles, uint32_t *pix) {
    if (!x || !dst || !dst->rgb || dst->feat_mask) return PVG_ERR_INVALID;
    std::vector<ViewDesc> v;
    uint32_t NV = 0, T = 0, P = 0;
    PVG_TRY(build_views(x, scene, 0, cam, 1, v, &NV, &T, &P));
    v[0].out_rgb = dst->rgb;
    v[0].out_depth = dst->depth;
    v[0].out_alpha = dst->alpha;
    v[0].out_feat = nullptr;
    *out = v[0];
    *tiles = T;
    *pix = P;
    return PVG_OK;
}

pvg_status_t serve_reserve(pvg_ctx_t *x, pvg_frame_t *f, uint64_t items, uint64_t tiles, uint64_t pix,
                           uint64_t pairs, int max_views) {
    if (!x || !f || items >= (1ull << 31) || tiles >= (1ull << 31) || pix >= (1ull << 32) || pairs > 0xfffffff0ull)
        return PVG_ERR_INVALID;
    for (DevBuf *b : {&x->item_cnt, &x->item_zkey, &x->alt_keys, &x->alt_vals, &x->vis_off, &f->sgid, &f->inv,
                      &f->szkey, &f->vis_cnt})
        PVG_TRY(ensure(*b, sizeof(uint32_t) * items));
    PVG_TRY(ensure(x->proj, sizeof(float4) * 4 * items));
    PVG_TRY(ensure(f->rec, sizeof(float4) * 3 * items));
    PVG_TRY(ensure(f->ell, sizeof(float4) * 2 * items));
    PVG_TRY(ensure(f->rowtab, sizeof(uint4) * items));
    PVG_TRY(ensure(f->rect, sizeof(uint2) * items));
    PVG_TRY(ensure(f->ranges, sizeof(uint2) * tiles));
    PVG_TRY(ensure(f->tile_order, sizeof(uint32_t) * tiles));
    PVG_TRY(ensure(f->tile_walk, sizeof(uint32_t) * tiles));
    PVG_TRY(ensure(f->tile_order_bwd, sizeof(uint32_t) * tiles));
    PVG_TRY(ensure(f->pix_T, sizeof(float) * pix));
    PVG_TRY(ensure(f->pix_last, sizeof(uint32_t) * pix));
    PVG_TRY(ensure(f->pix_neval, sizeof(uint32_t) * 2 * pix));
    for (DevBuf *b : {&f->pair_vals, &x->pair_keys, &x->pair_keys2, &x->pair_vals2})
        PVG_TRY(ensure(*b, sizeof(uint32_t) * pairs));
    PVG_TRY(ensure(x->chunk_start, sizeof(uint32_t) * emit_chunks((uint32_t)pairs)));
    PVG_TRY(ensure(f->stage_fwd->dev, sizeof(ViewDesc) * (size_t)max_views));
    return PVG_OK;
}

ViewDesc *serve_view_buffer(pvg_frame_t *f) { return ptr<ViewDesc>(f->stage_fwd->dev); }

const uint32_t *serve_counters(pvg_frame_t *f) { return ptr<uint32_t>(f->counters); }

pvg_status_t serve_forward(pvg_ctx_t *x, pvg_frame_t *f, std::vector<ViewDesc> &views, uint32_t NV, uint32_t tiles,
                           uint32_t pix, uint32_t pair_capacity, cudaStream_t s) {
    if (!x || !f || views.empty() || x->cfg.sync_sizes || pair_capacity == 0 || pair_capacity > 0xfffffff0u)
        return PVG_ERR_INVALID;
    PVG_TRY(ensure(f->stage_fwd->dev, sizeof(ViewDesc) * views.size()));
    x->cfg.pair_capacity = pair_capacity;
    return enqueue_forward(x, f, views, ptr<ViewDesc>(f->stage_fwd->dev), NV, tiles, pix, 0, 0, false, false, s);
}

}  // namespace pvg

extern "C" pvg_status_t pvg_render_fwd(pvg_ctx_t *x, const pvg_scene_t *scene, const pvg_camera_t *cams,
                                       int32_t n_views, const pvg_image_t *out, pvg_frame_t *frame,
                                       void *stream) {
    return render_fwd_impl(x, scene, 0, cams, n_views, out, frame, stream);
}

extern "C" pvg_status_t pvg_render_fwd_multi(pvg_ctx_t *x, const pvg_scene_t *scenes, const pvg_camera_t *cams,
                                             int32_t n_views, const pvg_image_t *out, pvg_frame_t *frame,
                                             void *stream) {
    return render_fwd_impl(x, scenes, 1, cams, n_views, out, frame, stream);
}

// ------------------------------------------------------------------ backward

// zeroes rows [0, *d_m) of a [*, per] array (the visible items' rows)
__global__ static void k_zero_rows(float *a, const uint32_t *d_m, int per) {
    pdl_enter();
    const size_t n = (size_t)per * *d_m;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        a[k] = 0.f;
}

extern "C" pvg_status_t pvg_render_bwd(pvg_ctx_t *x, const pvg_scene_t *scene, const pvg_camera_t *cams,
                                       int32_t n_views, pvg_frame_t *frame, const pvg_image_grad_t *dL,
                                       const pvg_scene_grad_t *grads, void *stream_) {
    if (!x || !dL || !grads) return PVG_ERR_INVALID;
    PVG_TRY(validate_scene(scene));
    pvg_frame *f = frame ? frame : x->own_frame;
    // the forward must have kept its state (a frame passed to it; NULL
    // rendered into the context's own frame for inference only)
    if (!f->valid || !f->has_state || !f->one_scene || f->n != scene->n || f->sh_degree != scene->sh_degree ||
        (int)f->views.size() != n_views)
        return PVG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream_;
    const bool capturing = is_capturing(s);
    std::vector<ViewDesc> views = f->views;
    bool feat_bwd = false;
    if ((f->feat_mask & kFeatSem) && ((scene->n > 0 && !scene->sem) || scene->n_sem != f->n_sem))
        return PVG_ERR_INVALID;
    for (int v = 0; v < n_views; v++) {
        if (!cams || cams[v].width != views[v].W || cams[v].height != views[v].H) return PVG_ERR_INVALID;
        if (dL[v].feat) {
            if (!f->feat_mask) return PVG_ERR_INVALID;  // the forward rendered no extra channel
            feat_bwd = true;
        }
        ViewDesc &d = views[v];
        d.mu = scene->mu; d.vel = scene->vel; d.tau = scene->tau; d.beta = scene->beta; d.period = scene->period;
        d.scale = scene->scale; d.quat = scene->quat; d.opac = scene->opacity; d.sh = scene->sh;
        d.sky = scene->sky; d.sky_res = scene->sky_res;
        d.g_sky = scene->sky ? grads->sky : nullptr;
        d.dl_rgb = dL[v].rgb; d.dl_depth = dL[v].depth; d.dl_alpha = dL[v].alpha;
        d.g_mu = grads->mu; d.g_vel = grads->vel; d.g_tau = grads->tau; d.g_beta = grads->beta;
        d.g_period = grads->period; d.g_scale = grads->scale; d.g_quat = grads->quat; d.g_opac = grads->opacity;
        d.g_sh = grads->sh;
        d.sem = scene->sem;
        d.n_sem = scene->n_sem;
        d.dl_feat = dL[v].feat;
        d.g_sem = (f->feat_mask & kFeatSem) ? grads->sem : nullptr;
    }
    const size_t N = (size_t)scene->n, K = (size_t)(scene->sh_degree + 1) * (scene->sh_degree + 1);
    struct { float *p; size_t n; } zero[] = {
        {grads->mu, 3 * N}, {grads->vel, 3 * N}, {grads->tau, N}, {grads->beta, N}, {grads->period, N},
        {grads->scale, 3 * N}, {grads->quat, 4 * N}, {grads->opacity, N}, {grads->sh, 3 * K * N}};
    // k_preprocess_bwd (one view) and k_preprocess_bwd_views (several views
    // of the scene) write every entry, zeros for the Gaussians no view sees;
    // without visible items nothing runs, so the arrays are zeroed here
    if (f->n_items == 0)
        for (auto &z : zero)
            if (z.p && z.n) PVG_CUDA(cudaMemsetAsync(z.p, 0, sizeof(float) * z.n, s));
    if (scene->sky && grads->sky)
        PVG_CUDA(cudaMemsetAsync(grads->sky, 0, sizeof(float) * 18 * (size_t)scene->sky_res * scene->sky_res, s));
    if ((f->feat_mask & kFeatSem) && grads->sem)
        PVG_CUDA(cudaMemsetAsync(grads->sem, 0, sizeof(float) * N * (size_t)f->n_sem, s));
    if (f->n_items == 0 && !scene->sky) return PVG_OK;
    PVG_TRY(ensure_c(f->g2d, sizeof(float) * 10 * (size_t)f->n_items, capturing));
    if (feat_bwd) PVG_TRY(ensure_c(f->gfeat, sizeof(float) * f->n_feat * (size_t)f->n_items, capturing));
    PVG_TRY(stage_views(*f->stage_bwd, views, s, capturing));

    Params p;
    std::memset(&p, 0, sizeof(p));
    p.views = ptr<ViewDesc>(f->stage_bwd->dev);
    p.n_views = n_views;
    p.sh_degree = scene->sh_degree;
    p.tile_w = f->tile_w;
    p.tile_h = f->tile_h;
    p.px = f->px;
    p.dilation = f->dilation;
    p.n_items = f->n_items;
    p.total_tiles = f->total_tiles;
    p.pair_capacity = f->pair_capacity;
    p.counters = ptr<uint32_t>(f->counters);
    p.sgid = ptr<uint32_t>(f->sgid);
    p.inv = ptr<uint32_t>(f->inv);
    p.szkey = ptr<uint32_t>(f->szkey);
    p.rec = ptr<float4>(f->rec);
    p.rect = ptr<uint2>(f->rect);
    p.vis_cnt = ptr<uint32_t>(f->vis_cnt);
    p.pair_vals = ptr<uint32_t>(f->pair_vals);
    p.ranges = ptr<uint2>(f->ranges);
    p.tile_order = ptr<uint32_t>(f->tile_order);
    p.pix_T = ptr<float>(f->pix_T);
    p.pix_last = ptr<uint32_t>(f->pix_last);
    p.g2d = ptr<float>(f->g2d);
    for (const ViewDesc &d : views) p.aux |= (d.dl_depth || d.dl_alpha || d.sky) ? 1 : 0;
    if (feat_bwd) {
        p.feat_mask = f->feat_mask;
        p.n_feat = f->n_feat;
        p.gfeat = ptr<float>(f->gfeat);
    }
    StageTimer &tm = x->timer;
    const bool timer_on = tm.on;
    if (capturing) tm.on = false;
    tm.begin(PVG_STAGE_COMPOSITE_BWD, s);
    // g2d zeroed, and the adjoint's tiles ordered longest walk first (the
    // forward recorded each tile's largest last-blend position)
    launch_bwd_prep(p, ptr<uint32_t>(f->tile_walk), ptr<uint32_t>(f->tile_order_bwd), s);
    p.tile_order = ptr<uint32_t>(f->tile_order_bwd);
    launch_composite_bwd(p, s);
    if (feat_bwd && f->n_items) {
        note_launch();
        pdl_launch(k_zero_rows, device_sm_count() * 4, 256, 0, s, p.gfeat, &p.counters[0], p.n_feat);
        launch_composite_feat_bwd(p, s);
    }
    tm.end(PVG_STAGE_COMPOSITE_BWD, s);
    tm.begin(PVG_STAGE_PREPROCESS_BWD, s);
    launch_preprocess_bwd(p, n_views > 1, s);
    if (feat_bwd) launch_feat_param_bwd(p, s);
    tm.end(PVG_STAGE_PREPROCESS_BWD, s);
    tm.on = timer_on;
    PVG_CUDA(cudaGetLastError());
    return PVG_OK;
}

// ------------------------------------------------------------------ loss

extern "C" pvg_status_t pvg_rgb_loss(pvg_ctx_t *x, const float *pred, const float *target, int32_t channels,
                                     int32_t height, int32_t width, float lambda_r, float *dl, float *loss,
                                     void *stream) {
    if (!x || !pred || !target || !loss || channels < 1 || height < 1 || width < 1 || channels > 65535 ||
        height > 16384 || width > 16384 || !(lambda_r >= 0.f && lambda_r <= 1.f))
        return PVG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const bool capturing = is_capturing(s);
    PVG_TRY(ensure_c(x->loss_partials, 2 * sizeof(float) * rgb_loss_partials(channels, height, width), capturing));
    PVG_CUDA(launch_rgb_loss(pred, target, channels, height, width, lambda_r, dl, loss, x->loss_partials.p, s));
    return PVG_OK;
}

extern "C" pvg_status_t pvg_l1_loss(pvg_ctx_t *x, const float *pred, const float *target, int64_t n, float scale,
                                    float *dl, float *loss, void *stream) {
    if (!x || !loss || n < 0 || (n > 0 && (!pred || !target))) return PVG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t need = l1_loss_scratch_bytes();
    if (x->l1_scratch.bytes < need) {
        if (is_capturing(s)) return PVG_ERR_INVALID;
        PVG_TRY(ensure(x->l1_scratch, need));
        PVG_CUDA(cudaMemsetAsync(x->l1_scratch.p, 0, x->l1_scratch.bytes, s));  // the ticket starts at 0
    }
    PVG_CUDA(launch_l1_loss(pred, target, n, scale, dl, loss, x->l1_scratch.p, s));
    return PVG_OK;
}

// ------------------------------------------------------------------ introspection

extern "C" pvg_status_t pvg_frame_stats(pvg_frame_t *f, int64_t *n_visible, int64_t *n_pairs, int32_t *overflowed) {
    if (!f) return PVG_ERR_INVALID;
    PVG_CUDA(cudaMemcpyAsync(f->h_counters, f->counters.p, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, f->stream));
    PVG_CUDA(cudaStreamSynchronize(f->stream));
    if (n_visible) *n_visible = f->h_counters[0];
    if (n_pairs) *n_pairs = f->h_counters[1];
    if (overflowed) *overflowed = (int32_t)f->h_counters[2];
    return PVG_OK;
}

__global__ static void k_export_rect(const uint2 *rect, const uint32_t *d_m, int32_t *out) {
    const uint32_t M = *d_m;
    for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const uint2 r = rect[m];
        out[4 * m + 0] = (int32_t)(r.x & 0xffffu);
        out[4 * m + 1] = (int32_t)(r.x >> 16);
        out[4 * m + 2] = (int32_t)(r.y & 0xffffu);
        out[4 * m + 3] = (int32_t)(r.y >> 16);
    }
}

extern "C" pvg_status_t pvg_frame_export(pvg_frame_t *f, uint32_t *sorted_gid, uint32_t *depth_key, int32_t *rect,
                                         float *records, uint32_t *pair_vals, uint32_t *ranges) {
    if (!f || !f->valid) return PVG_ERR_INVALID;
    int64_t M, K;
    int32_t ov;
    PVG_TRY(pvg_frame_stats(f, &M, &K, &ov));
    if (K > (int64_t)f->pair_capacity) K = f->pair_capacity;
    cudaStream_t s = f->stream;
    if (sorted_gid && M)
        PVG_CUDA(cudaMemcpyAsync(sorted_gid, f->sgid.p, 4 * M, cudaMemcpyDeviceToDevice, s));
    if (depth_key && M)
        PVG_CUDA(cudaMemcpyAsync(depth_key, f->szkey.p, 4 * M, cudaMemcpyDeviceToDevice, s));
    if (records && M)
        PVG_CUDA(cudaMemcpyAsync(records, f->rec.p, 48 * M, cudaMemcpyDeviceToDevice, s));
    if (pair_vals && K)
        PVG_CUDA(cudaMemcpyAsync(pair_vals, f->pair_vals.p, 4 * K, cudaMemcpyDeviceToDevice, s));
    if (ranges && f->total_tiles)
        PVG_CUDA(cudaMemcpyAsync(ranges, f->ranges.p, 8 * (size_t)f->total_tiles, cudaMemcpyDeviceToDevice, s));
    if (rect && M) {
        note_launch();
        k_export_rect<<<device_sm_count(), 256, 0, s>>>(ptr<uint2>(f->rect), ptr<uint32_t>(f->counters), rect);
    }
    PVG_CUDA(cudaGetLastError());
    PVG_CUDA(cudaStreamSynchronize(s));
    return PVG_OK;
}

// ------------------------------------------------------------------ measurement

extern "C" uint64_t pvg_kernel_launches(void) { return pvg::g_launches.load(); }

extern "C" pvg_status_t pvg_profile_enable(pvg_ctx_t *x, int on) {
    if (!x) return PVG_ERR_INVALID;
    x->timer.on = on != 0;
    return PVG_OK;
}

extern "C" pvg_status_t pvg_profile_read(pvg_ctx_t *x, double *ms, int64_t *calls) {
    if (!x || !ms || !calls) return PVG_ERR_INVALID;
    for (int k = 0; k < PVG_NUM_STAGES; k++) {
        ms[k] = 0.0;
        calls[k] = 0;
    }
    for (auto &r : x->timer.pending) {
        PVG_CUDA(cudaEventSynchronize(r.b));
        float e = 0.f;
        PVG_CUDA(cudaEventElapsedTime(&e, r.a, r.b));
        ms[r.stage] += e;
        calls[r.stage] += 1;
        x->timer.pool.push_back(r.a);
        x->timer.pool.push_back(r.b);
    }
    x->timer.pending.clear();
    return PVG_OK;
}

__global__ static void k_sum_u32(const uint32_t *v, uint32_t n, unsigned long long *out) {
    unsigned long long acc = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += v[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

extern "C" pvg_status_t pvg_frame_eval_count(pvg_ctx_t *x, pvg_frame_t *f, int64_t *evals, int64_t *blends) {
    if (!x || !f || !evals || !f->valid) return PVG_ERR_INVALID;
    cudaStream_t s = f->stream;
    const int nv = (int)f->views.size();
    PVG_TRY(ensure(x->views, sizeof(ViewDesc) * nv));
    PVG_TRY(ensure(x->sort_n, 2 * sizeof(unsigned long long)));
    PVG_CUDA(cudaMemcpyAsync(x->views.p, f->views.data(), sizeof(ViewDesc) * nv, cudaMemcpyHostToDevice, s));
    Params p;
    std::memset(&p, 0, sizeof(p));
    p.views = ptr<ViewDesc>(x->views);
    p.n_views = nv;
    p.tile_w = f->tile_w;
    p.tile_h = f->tile_h;
    p.px = f->px;
    p.total_tiles = f->total_tiles;
    p.total_pix = f->total_pix;
    p.rec = ptr<float4>(f->rec);
    p.pair_vals = ptr<uint32_t>(f->pair_vals);
    p.ranges = ptr<uint2>(f->ranges);
    p.tile_order = ptr<uint32_t>(f->tile_order);
    p.pix_neval = ptr<uint32_t>(f->pix_neval);
    PVG_CUDA(cudaMemsetAsync(f->pix_neval.p, 0, sizeof(uint32_t) * 2 * (size_t)f->total_pix, s));
    launch_composite_stats(p, s);
    unsigned long long h[2] = {0, 0};
    unsigned long long *d = ptr<unsigned long long>(x->sort_n);
    PVG_CUDA(cudaMemsetAsync(d, 0, sizeof(h), s));
    note_launch();
    k_sum_u32<<<device_sm_count() * 4, 256, 0, s>>>(ptr<uint32_t>(f->pix_neval), f->total_pix, d);
    note_launch();
    k_sum_u32<<<device_sm_count() * 4, 256, 0, s>>>(ptr<uint32_t>(f->pix_neval) + f->total_pix, f->total_pix, d + 1);
    PVG_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    PVG_CUDA(cudaStreamSynchronize(s));
    *evals = (int64_t)h[0];
    if (blends) *blends = (int64_t)h[1];
    return PVG_OK;
}

// ------------------------------------------------------------------ sorting

__global__ static void k_store_u32(uint32_t *dst, uint32_t v) { *dst = v; }

extern "C" pvg_status_t pvg_sort_pairs(pvg_ctx_t *x, uint32_t *keys, uint32_t *vals, int64_t n, int32_t begin_bit,
                                       int32_t end_bit, void *stream_) {
    if (!x || n < 0 || n >= (int64_t)0xffffffffLL || begin_bit < 0 || end_bit > 32 || begin_bit >= end_bit)
        return PVG_ERR_INVALID;
    if (n == 0) return PVG_OK;
    if (!keys || !vals) return PVG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream_;
    PVG_TRY(ensure(x->alt_keys, sizeof(uint32_t) * (size_t)n));
    PVG_TRY(ensure(x->alt_vals, sizeof(uint32_t) * (size_t)n));
    PVG_TRY(ensure(x->sort_n, sizeof(uint32_t)));
    note_launch();
    k_store_u32<<<1, 1, 0, s>>>(ptr<uint32_t>(x->sort_n), (uint32_t)n);
    bool in_alt = false;
    radix_sort_pairs(keys, vals, ptr<uint32_t>(x->alt_keys), ptr<uint32_t>(x->alt_vals), ptr<uint32_t>(x->sort_n),
                     (uint32_t)n, begin_bit, end_bit, x->temp.p, s, &in_alt);
    if (in_alt) {
        PVG_CUDA(cudaMemcpyAsync(keys, x->alt_keys.p, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        PVG_CUDA(cudaMemcpyAsync(vals, x->alt_vals.p, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    }
    PVG_CUDA(cudaGetLastError());
    return PVG_OK;
}

// serve.cu -- continuous-batching render server (pvg_serve_*).
//
// Requests live in a ring of slots in mapped pinned memory: submit writes
// a request's view descriptor (built on the host exactly as
// pvg_render_fwd builds it, so a served image equals a direct render bit
// for bit) into a free slot and then publishes the slot by storing its
// sequence number with release order.  Workers -- one thread, one CUDA
// stream, one workspace each -- take queued requests into batches and
// enqueue, per batch, one launch sequence that the host never waits for:
//
//   k_serve_gather    one thread per view: a bounded wait (globaltimer
//                     deadline and an iteration cap) for the view's slot to
//                     carry its sequence number, then the descriptor is
//                     copied into the workspace with this batch's tile /
//                     pixel / item bases; a slot that never appears gets a
//                     descriptor that renders nothing (every point behind
//                     the near plane) and its request the status
//                     PVG_ERR_TIMEOUT
//   the forward pass  of pvg_render_fwd over all the batch's views, with the
//                     pair capacity the batch reserved
//   k_serve_complete  per slot: status (TIMEOUT, OVERFLOW when the pair
//                     count of the batch exceeded its reservation, else
//                     OK), the batch's pair count and GPU timestamps, then
//                     the slot's done sequence number with release order
//
// A worker keeps up to pipeline_depth batches in flight on its stream
// (stream order keeps their use of the one workspace apart) and notices
// completion by reading the slots' done numbers.  Requests that arrive
// while batches are on the GPU form the next batch (continuous batching);
// workers on different streams overlap on the device.
//
// Admission: at creation the free device memory (cudaMemGetInfo) bounds
// the workers' arenas, reserved in advance so that nothing is allocated
// while serving; a batch takes requests while their Gaussians, pixels,
// tiles and estimated pairs fit its worker's arena.  The pair estimate of
// a request is its pixels times the pairs per pixel its scene produced in
// earlier batches.  After the GPU counted the pairs of a batch, a count
// above the reservation sends the batch's requests back to the head of the
// queue with the measured density (count, reserve, continue or requeue).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pvg.h"
#include "pvg_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
using pvg::ViewDesc;

constexpr int kServeMaxBatch = 64;
constexpr int kMaxScenes = 1024;
constexpr uint32_t kGatherSpinCap = 1u << 22;  // iterations of the gather wait (about 4 s of 1 us sleeps)
constexpr double kPairsPerPixelStart = 8.0;    // estimate for a scene before its first batch
constexpr int kMaxAttempts = 4;

// One request slot in mapped pinned memory.  The host writes `view` and
// then `seq`; the GPU writes the fields below `seq` and then `done_seq`.
struct alignas(128) Slot {
    ViewDesc view;
    uint32_t seq;
    uint32_t done_seq;
    int32_t status;
    uint32_t pairs;
    unsigned long long t_gather_ns, t_done_ns;
};

struct GatherView {
    uint32_t slot, seq, scene, tile_base, pix_base, item_base;
    int32_t W, H, tiles_x, tiles_y;
    float *rgb, *depth, *alpha;
};

struct GatherArgs {
    int32_t n;
    uint32_t pair_reservation;
    unsigned long long timeout_ns;
    GatherView v[kServeMaxBatch];
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_sys(uint32_t *p, uint32_t v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void k_serve_gather(Slot *ring, const ViewDesc *scene_tab, GatherArgs a, ViewDesc *views,
                               uint32_t *gate_ok) {
    const int v = threadIdx.x;
    if (v >= a.n) return;
    const GatherView &g = a.v[v];
    Slot *sl = &ring[g.slot];
    const unsigned long long t0 = globaltimer_ns();
    bool ok = false;
    for (uint32_t it = 0; it < kGatherSpinCap; ++it) {
        if (ld_acquire_sys(&sl->seq) == g.seq) {
            ok = true;
            break;
        }
        if (globaltimer_ns() - t0 > a.timeout_ns) break;
        __nanosleep(1000);
    }
    ViewDesc d;
    if (ok) {
        d = sl->view;
    } else {
        // the request never appeared: its scene, no visible point
        d = scene_tab[g.scene];
        for (int k = 0; k < 9; k++) d.R[k] = (k % 4 == 0) ? 1.f : 0.f;
        d.T[0] = d.T[1] = d.T[2] = 0.f;
        d.campos[0] = d.campos[1] = d.campos[2] = 0.f;
        d.fx = d.fy = 1.f;
        d.cx = d.cy = 0.f;
        d.t = 0.f;
        d.dt = 0.f;
        d.znear = INFINITY;
        d.bg[0] = d.bg[1] = d.bg[2] = 0.f;
        d.limx = d.limy = 1.f;
        d.sky_jitter = nullptr;
    }
    d.W = g.W;
    d.H = g.H;
    d.tiles_x = g.tiles_x;
    d.tiles_y = g.tiles_y;
    d.tile_base = g.tile_base;
    d.pix_base = g.pix_base;
    d.item_base = g.item_base;
    d.out_rgb = g.rgb;
    d.out_depth = g.depth;
    d.out_alpha = g.alpha;
    d.out_feat = nullptr;
    views[v] = d;
    gate_ok[v] = ok ? 1u : 0u;
    sl->t_gather_ns = t0;  // the batch's GPU time starts before the wait
}

__global__ void k_serve_complete(Slot *ring, GatherArgs a, const uint32_t *counters, const uint32_t *gate_ok) {
    const int v = threadIdx.x;
    if (v >= a.n) return;
    const GatherView &g = a.v[v];
    Slot *sl = &ring[g.slot];
    const uint32_t K = counters[1];
    const bool over = counters[2] != 0 || K > a.pair_reservation;
    sl->status = !gate_ok[v] ? PVG_ERR_TIMEOUT : (over ? PVG_ERR_OVERFLOW : PVG_OK);
    sl->pairs = K;
    sl->t_done_ns = globaltimer_ns();
    __threadfence_system();
    st_release_sys(&sl->done_seq, g.seq);
}

struct Req {
    int32_t scene = 0;
    uint32_t slot = 0, seq = 0;
    ViewDesc view;  // host copy (bases 0)
    uint32_t tiles = 0, pix = 0;
    double t_submit = 0, t_start = -1, t_done = -1, gpu_ms = -1;
    int state = 0;  // 0 queued, 1 running, 2 done
    pvg_status_t status = PVG_OK;
    int32_t batch_views = 0;
    int32_t attempts = 0;
    double pairs_hint = 0;  // pairs per pixel measured when the request was requeued
};

struct Flight {
    std::vector<uint64_t> ids;
    std::vector<uint32_t> slots, seqs;
    uint64_t pix = 0;
    size_t bytes = 0;
};

struct Worker {
    std::thread th;
    cudaStream_t stream = nullptr;
    pvg_ctx_t *ctx = nullptr;
    pvg_frame_t *frame = nullptr;
    uint32_t *gate_ok = nullptr;  // device [kServeMaxBatch]
};

struct SceneInfo {
    pvg_scene_t scene;
    double pairs_per_pixel = kPairsPerPixelStart;
    bool measured = false;
};

}  // namespace

struct pvg_server {
    pvg_serve_config_t cfg;
    int device = 0;
    Clock::time_point t0;
    std::vector<SceneInfo> scenes;
    ViewDesc *scene_tab = nullptr;  // device [kMaxScenes]
    Slot *ring = nullptr;           // host pointer (mapped pinned)
    Slot *ring_dev = nullptr;       // its device address
    uint32_t ring_size = 0;
    std::vector<uint32_t> free_slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_id = 1;
    size_t in_flight = 0;
    bool stopping = false;
    std::vector<Worker> workers;
    int64_t batches = 0, views = 0, requeues = 0;
    int32_t withhold = 0;
    // arena of one worker
    uint64_t cap_items = 0, cap_pix = 0, cap_tiles = 0, cap_pairs = 0;
    size_t budget = 0, free_at_create = 0;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

// bytes of the workspace per Gaussian, pixel, tile and pair of a batch
constexpr size_t kBytesPerItem = 204, kBytesPerPixel = 16, kBytesPerTile = 12, kBytesPerPair = 16;

uint64_t est_pairs(const pvg_server *S, const Req &r) {
    const double ppp = std::max(S->scenes[r.scene].pairs_per_pixel, r.pairs_hint);
    return (uint64_t)std::ceil(ppp * 1.25 * (double)r.pix) + 256;
}

size_t req_bytes(const pvg_server *S, const Req &r) {
    return (size_t)r.view.n * kBytesPerItem + (size_t)r.pix * kBytesPerPixel + (size_t)r.tiles * kBytesPerTile +
           (size_t)est_pairs(S, r) * kBytesPerPair;
}

// Takes requests from the head of the queue into `fl` while they fit the
// worker's arena, the views limit and (unless nothing is in flight) the
// server's budget.  Called with S->mu held.
bool take_batch(pvg_server *S, Flight &fl, uint64_t *pairs) {
    uint64_t items = 0, tiles = 0, pix = 0, pr = 0;
    size_t bytes = 0;
    int deg = -1;
    while (!S->queue.empty() && (int)fl.ids.size() < S->cfg.max_batch_views) {
        Req &r = S->reqs[S->queue.front()];
        const int d = r.view.sh_degree;
        if (deg >= 0 && d != deg) break;  // one SH degree per launch sequence
        const uint64_t p = est_pairs(S, r);
        const size_t b = req_bytes(S, r);
        if (!fl.ids.empty()) {
            if (items + r.view.n > S->cap_items || pix + r.pix > S->cap_pix || tiles + r.tiles > S->cap_tiles ||
                pr + p > S->cap_pairs || S->in_flight + bytes + b > S->budget)
                break;
        } else if (S->in_flight > 0 && S->in_flight + b > S->budget) {
            break;  // wait for memory to free up
        }
        deg = d;
        items += r.view.n;
        tiles += r.tiles;
        pix += r.pix;
        pr += p;
        bytes += b;
        fl.ids.push_back(S->queue.front());
        S->queue.pop_front();
    }
    if (fl.ids.empty()) return false;
    fl.pix = pix;
    fl.bytes = bytes;
    *pairs = std::max<uint64_t>(pr, 1024);
    S->in_flight += bytes;
    return true;
}

bool slot_done(const pvg_server *S, uint32_t slot, uint32_t seq) {
    return __atomic_load_n(&S->ring[slot].done_seq, __ATOMIC_ACQUIRE) == seq;
}

// Enqueues the batch's launch sequence; returns the launch status (the
// requests are marked failed by the caller if it is not PVG_OK).
pvg_status_t launch_batch(pvg_server *S, Worker *W, Flight &fl, uint64_t pairs) {
    GatherArgs a;
    std::memset(&a, 0, sizeof(a));
    std::vector<ViewDesc> views;
    uint64_t items = 0, tiles = 0, pix = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        const double t = S->now_ms();
        a.n = (int32_t)fl.ids.size();
        for (int v = 0; v < a.n; v++) {
            Req &r = S->reqs[fl.ids[v]];
            r.state = 1;
            r.t_start = t;
            r.attempts += 1;
            ViewDesc d = r.view;
            d.tile_base = (uint32_t)tiles;
            d.pix_base = (uint32_t)pix;
            d.item_base = (uint32_t)items;
            views.push_back(d);
            GatherView &g = a.v[v];
            g.slot = r.slot;
            g.seq = r.seq;
            g.scene = (uint32_t)r.scene;
            g.tile_base = d.tile_base;
            g.pix_base = d.pix_base;
            g.item_base = d.item_base;
            g.W = d.W;
            g.H = d.H;
            g.tiles_x = d.tiles_x;
            g.tiles_y = d.tiles_y;
            g.rgb = d.out_rgb;
            g.depth = d.out_depth;
            g.alpha = d.out_alpha;
            fl.slots.push_back(r.slot);
            fl.seqs.push_back(r.seq);
            tiles += r.tiles;
            pix += r.pix;
            items += r.view.n;
        }
    }
    if (items >= (1ull << 31) || tiles >= (1ull << 31) || pix >= (1ull << 32)) return PVG_ERR_INVALID;
    const uint32_t cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(pairs, S->cap_pairs), 0xfffffff0ull);
    a.pair_reservation = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(pairs, S->cap_pairs), 0xfffffff0ull);
    a.timeout_ns = (unsigned long long)S->cfg.gate_timeout_us * 1000ull;
    // a requeued request keeps its sequence number: clear its done number
    // before the GPU can set it again
    for (int v = 0; v < a.n; v++) __atomic_store_n(&S->ring[fl.slots[v]].done_seq, 0u, __ATOMIC_RELEASE);
    // a batch beyond the reserved arena grows the workspace, which frees
    // buffers that earlier batches on this stream may still use
    if (items > S->cap_items || tiles > S->cap_tiles || pix > S->cap_pix || cap > S->cap_pairs)
        if (cudaStreamSynchronize(W->stream) != cudaSuccess) return PVG_ERR_CUDA;
    ViewDesc *dev_views = pvg::serve_view_buffer(W->frame);
    pvg::note_launch();
    k_serve_gather<<<1, kServeMaxBatch, 0, W->stream>>>(S->ring_dev, S->scene_tab, a, dev_views, W->gate_ok);
    if (cudaGetLastError() != cudaSuccess) return PVG_ERR_CUDA;
    // the descriptors copied into dev_views by the gather kernel are the ones
    // rendered; `views` gives the host the sizes and bases
    const pvg_status_t st =
        pvg::serve_forward(W->ctx, W->frame, views, (uint32_t)items, (uint32_t)tiles, (uint32_t)pix, cap, W->stream);
    if (st != PVG_OK) return st;
    pvg::note_launch();
    k_serve_complete<<<1, kServeMaxBatch, 0, W->stream>>>(S->ring_dev, a, pvg::serve_counters(W->frame), W->gate_ok);
    return cudaGetLastError() == cudaSuccess ? PVG_OK : PVG_ERR_CUDA;
}

// The batch finished on the GPU (every slot's done number is set): record
// results, requeue the requests of an overflowed batch.  S->mu held.
void finish_batch(pvg_server *S, Flight &fl) {
    const double t = S->now_ms();
    uint32_t K = 0;
    bool overflow = false;
    for (size_t v = 0; v < fl.ids.size(); v++) {
        const Slot &sl = S->ring[fl.slots[v]];
        K = std::max(K, sl.pairs);
        if (sl.status == PVG_ERR_OVERFLOW) overflow = true;
    }
    const double ppp = fl.pix ? (double)K / (double)fl.pix : 0.0;
    std::vector<uint64_t> requeue;
    for (size_t v = 0; v < fl.ids.size(); v++) {
        Req &r = S->reqs[fl.ids[v]];
        const Slot &sl = S->ring[fl.slots[v]];
        SceneInfo &si = S->scenes[r.scene];
        // the batch's pairs per pixel bounds every one of its scenes' density
        if (!si.measured || ppp > si.pairs_per_pixel) si.pairs_per_pixel = ppp;
        si.measured = true;
        pvg_status_t st = (pvg_status_t)sl.status;
        if (st == PVG_ERR_OVERFLOW && r.attempts < kMaxAttempts) {
            r.pairs_hint = std::max(r.pairs_hint, ppp * 1.1);
            r.state = 0;
            requeue.push_back(fl.ids[v]);
            continue;
        }
        r.state = 2;
        r.t_done = t;
        r.gpu_ms = (double)(sl.t_done_ns - sl.t_gather_ns) * 1e-6;
        r.status = st;
        r.batch_views = (int32_t)fl.ids.size();
    }
    if (overflow) S->requeues += 1;
    for (auto it = requeue.rbegin(); it != requeue.rend(); ++it) S->queue.push_front(*it);
    S->in_flight -= fl.bytes;
    S->batches += 1;
    S->views += (int64_t)fl.ids.size();
}

void fail_batch(pvg_server *S, Flight &fl, pvg_status_t st) {
    const double t = S->now_ms();
    for (uint64_t id : fl.ids) {
        Req &r = S->reqs[id];
        r.state = 2;
        r.t_done = t;
        r.status = st;
        r.batch_views = (int32_t)fl.ids.size();
    }
    S->in_flight -= fl.bytes;
    S->batches += 1;
    S->views += (int64_t)fl.ids.size();
}

void worker_loop(pvg_server *S, Worker *W) {
    cudaSetDevice(S->device);
    std::deque<Flight> flights;
    const int depth = S->cfg.pipeline_depth;
    for (;;) {
        bool progress = false;
        // completions, oldest first
        while (!flights.empty()) {
            Flight &fl = flights.front();
            bool done = true;
            for (size_t v = 0; v < fl.slots.size() && done; v++) done = slot_done(S, fl.slots[v], fl.seqs[v]);
            if (!done) {
                // a launch that failed on the device never sets its flags
                const cudaError_t e = cudaStreamQuery(W->stream);
                if (e != cudaSuccess && e != cudaErrorNotReady) {
                    cudaGetLastError();
                    std::lock_guard<std::mutex> lk(S->mu);
                    fail_batch(S, fl, PVG_ERR_CUDA);
                    flights.pop_front();
                    progress = true;
                    continue;
                }
                break;
            }
            {
                std::lock_guard<std::mutex> lk(S->mu);
                finish_batch(S, fl);
            }
            flights.pop_front();
            progress = true;
        }
        if (progress) {
            S->cv_done.notify_all();
            S->cv_work.notify_all();
        }
        // a new batch
        if ((int)flights.size() < depth) {
            Flight fl;
            uint64_t pairs = 0;
            bool got = false;
            {
                std::unique_lock<std::mutex> lk(S->mu);
                for (;;) {
                    got = take_batch(S, fl, &pairs);
                    if (got || !flights.empty()) break;
                    if (S->stopping && S->queue.empty()) return;
                    S->cv_work.wait(lk);
                }
            }
            if (got) {
                const pvg_status_t st = launch_batch(S, W, fl, pairs);
                if (st != PVG_OK) {
                    // nothing of a failed launch sequence is waited for:
                    // drain the stream, then fail the batch
                    cudaStreamSynchronize(W->stream);
                    cudaGetLastError();
                    {
                        std::lock_guard<std::mutex> lk(S->mu);
                        fail_batch(S, fl, st);
                    }
                    S->cv_done.notify_all();
                } else {
                    flights.push_back(std::move(fl));
                }
                progress = true;
            }
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

void stop_workers(pvg_server *S) {
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_work.notify_all();
    for (Worker &w : S->workers)
        if (w.th.joinable()) w.th.join();
    for (Worker &w : S->workers) {
        if (w.stream) cudaStreamSynchronize(w.stream);
        if (w.frame) pvg_frame_destroy(w.frame);
        if (w.ctx) pvg_destroy(w.ctx);
        if (w.gate_ok) cudaFree(w.gate_ok);
        if (w.stream) cudaStreamDestroy(w.stream);
    }
    S->workers.clear();
}

void free_server(pvg_server *S) {
    stop_workers(S);
    if (S->scene_tab) cudaFree(S->scene_tab);
    if (S->ring) cudaFreeHost(S->ring);
    delete S;
}

}  // namespace

extern "C" void pvg_serve_config_default(pvg_serve_config_t *c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->max_batch_views = 16;
    c->n_streams = 4;
    c->memory_budget = (int64_t)8 << 30;
    c->max_pending = 4096;
    c->tile_w = 16;
    c->tile_h = 16;
    c->pixels_per_thread = 1;
    c->gate_timeout_us = 1000000;
    c->pipeline_depth = 1;
    c->pair_capacity = 0;
}

extern "C" pvg_status_t pvg_serve_create(pvg_server_t **out, const pvg_serve_config_t *cfg) {
    if (!out) return PVG_ERR_INVALID;
    pvg_serve_config_t c;
    if (cfg) c = *cfg; else pvg_serve_config_default(&c);
    if (c.max_batch_views < 1 || c.max_batch_views > kServeMaxBatch || c.n_streams < 1 || c.n_streams > 16 ||
        c.memory_budget <= 0 || c.max_pending < 1 || c.max_pending > (1 << 20) || c.gate_timeout_us < 1 ||
        c.pipeline_depth < 1 || c.pipeline_depth > 4 || c.pair_capacity < 0)
        return PVG_ERR_INVALID;
    pvg_config_t rc;
    pvg_config_default(&rc);
    rc.tile_w = c.tile_w;
    rc.tile_h = c.tile_h;
    rc.pixels_per_thread = c.pixels_per_thread;
    rc.sync_sizes = 0;
    rc.pair_capacity = 1 << 20;
    pvg_server *S = new pvg_server();
    S->cfg = c;
    S->t0 = Clock::now();
    size_t free_b = 0, total_b = 0;
    if (cudaGetDevice(&S->device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return PVG_ERR_CUDA;
    }
    // admission by free memory: the arenas together take at most 90 % of it
    S->free_at_create = free_b;
    S->budget = std::min<size_t>((size_t)c.memory_budget, free_b / 10 * 9);
    const size_t arena = S->budget / (size_t)c.n_streams;
    S->cap_items = std::min<uint64_t>(arena * 45 / 100 / kBytesPerItem, (1ull << 31) - 1);
    S->cap_pix = std::min<uint64_t>(arena * 10 / 100 / kBytesPerPixel, (1ull << 32) - 1);
    S->cap_tiles = std::min<uint64_t>(arena * 5 / 100 / kBytesPerTile, (1ull << 31) - 1);
    S->cap_pairs = c.pair_capacity > 0 ? (uint64_t)c.pair_capacity
                                       : std::min<uint64_t>(arena * 40 / 100 / kBytesPerPair, 0xfffffff0ull);
    // the ring: every request holds a slot from submit to release
    S->ring_size = (uint32_t)c.max_pending * 2 + 64u * kServeMaxBatch;
    pvg_status_t st = PVG_OK;
    if (cudaHostAlloc((void **)&S->ring, sizeof(Slot) * S->ring_size, cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&S->ring_dev, S->ring, 0) != cudaSuccess) {
        cudaGetLastError();
        S->ring = nullptr;
        delete S;
        return PVG_ERR_OOM;
    }
    std::memset(S->ring, 0, sizeof(Slot) * S->ring_size);
    for (uint32_t k = S->ring_size; k-- > 0;) S->free_slots.push_back(k);
    if (cudaMalloc(&S->scene_tab, sizeof(ViewDesc) * kMaxScenes) != cudaSuccess) {
        cudaGetLastError();
        S->scene_tab = nullptr;
        free_server(S);
        return PVG_ERR_OOM;
    }
    S->workers.resize(c.n_streams);
    for (Worker &w : S->workers) {
        if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&w.gate_ok, sizeof(uint32_t) * kServeMaxBatch) != cudaSuccess) {
            cudaGetLastError();
            st = PVG_ERR_CUDA;
            break;
        }
        if ((st = pvg_create(&w.ctx, &rc)) != PVG_OK) break;
        if ((st = pvg_frame_create(&w.frame)) != PVG_OK) break;
        // the arena, reserved now so that serving allocates nothing
        if ((st = pvg::serve_reserve(w.ctx, w.frame, S->cap_items, S->cap_tiles, S->cap_pix, S->cap_pairs,
                                     kServeMaxBatch)) != PVG_OK)
            break;
    }
    if (st != PVG_OK) {
        free_server(S);
        return st;
    }
    for (Worker &w : S->workers) w.th = std::thread(worker_loop, S, &w);
    *out = S;
    return PVG_OK;
}

extern "C" pvg_status_t pvg_serve_add_scene(pvg_server_t *S, const pvg_scene_t *scene, int32_t *scene_id) {
    if (!S || !scene || !scene_id || scene->n < 0 || scene->sh_degree < 0 || scene->sh_degree > 3)
        return PVG_ERR_INVALID;
    // the scene's part of a view descriptor, for views whose slot never appears
    pvg_camera_t cam;
    std::memset(&cam, 0, sizeof(cam));
    cam.viewmat[0] = cam.viewmat[5] = cam.viewmat[10] = 1.f;
    cam.fx = cam.fy = 1.f;
    cam.width = cam.height = 1;
    float dummy = 0.f;
    pvg_image_t img;
    std::memset(&img, 0, sizeof(img));
    img.rgb = &dummy;
    ViewDesc d;
    uint32_t tiles = 0, pix = 0;
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->scenes.size() >= kMaxScenes) return PVG_ERR_INVALID;
    const pvg_status_t st = pvg::serve_view_desc(S->workers[0].ctx, scene, &cam, &img, &d, &tiles, &pix);
    if (st != PVG_OK) return st;
    if (cudaMemcpy(S->scene_tab + S->scenes.size(), &d, sizeof(d), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return PVG_ERR_CUDA;
    }
    SceneInfo si;
    si.scene = *scene;
    S->scenes.push_back(si);
    *scene_id = (int32_t)S->scenes.size() - 1;
    return PVG_OK;
}

extern "C" pvg_status_t pvg_serve_submit(pvg_server_t *S, int32_t scene_id, const pvg_camera_t *cam,
                                         const pvg_image_t *dst, uint64_t *req_id) {
    if (!S || !cam || !dst || !dst->rgb || !req_id) return PVG_ERR_INVALID;
    if (dst->feat_mask != 0) return PVG_ERR_INVALID;  // served requests render colour, depth, opacity
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (scene_id < 0 || scene_id >= (int32_t)S->scenes.size()) return PVG_ERR_NOT_FOUND;
        if ((int64_t)S->queue.size() >= S->cfg.max_pending || S->free_slots.empty()) return PVG_ERR_BUSY;
        Req r;
        r.scene = scene_id;
        const pvg_status_t st = pvg::serve_view_desc(S->workers[0].ctx, &S->scenes[scene_id].scene, cam, dst,
                                                     &r.view, &r.tiles, &r.pix);
        if (st != PVG_OK) return st;
        const uint64_t id = S->next_id++;
        r.slot = S->free_slots.back();
        S->free_slots.pop_back();
        r.seq = (uint32_t)(id & 0xffffffffu) | 1u;  // never 0, the value of an unset done number
        r.t_submit = S->now_ms();
        Slot &sl = S->ring[r.slot];
        sl.view = r.view;
        if (S->withhold > 0) {
            S->withhold -= 1;  // test hook: the slot is never published
        } else {
            __atomic_store_n(&sl.seq, r.seq, __ATOMIC_RELEASE);
        }
        S->reqs[id] = r;
        S->queue.push_back(id);
        *req_id = id;
    }
    S->cv_work.notify_one();
    return PVG_OK;
}

static void fill_stats(const Req &r, pvg_req_stats_t *st) {
    if (!st) return;
    std::memset(st, 0, sizeof(*st));
    st->submit_ms = r.t_submit;
    st->start_ms = r.t_start;
    st->done_ms = r.t_done;
    st->batch_views = r.batch_views;
    st->status = r.status;
    st->gpu_ms = r.gpu_ms;
    st->attempts = r.attempts;
}

extern "C" pvg_status_t pvg_serve_poll(pvg_server_t *S, uint64_t req_id, int32_t *done, pvg_req_stats_t *stats) {
    if (!S || !done) return PVG_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return PVG_ERR_NOT_FOUND;
    *done = it->second.state == 2;
    fill_stats(it->second, stats);
    return PVG_OK;
}

extern "C" pvg_status_t pvg_serve_wait(pvg_server_t *S, uint64_t req_id, double timeout_ms, pvg_req_stats_t *stats) {
    if (!S) return PVG_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return PVG_ERR_NOT_FOUND;
    const auto deadline = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
    while (it->second.state != 2) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state != 2)
            return PVG_ERR_TIMEOUT;
        it = S->reqs.find(req_id);
    }
    fill_stats(it->second, stats);
    return it->second.status;
}

extern "C" pvg_status_t pvg_serve_release(pvg_server_t *S, uint64_t req_id) {
    if (!S) return PVG_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return PVG_ERR_NOT_FOUND;
    if (it->second.state != 2) return PVG_ERR_BUSY;
    Slot &sl = S->ring[it->second.slot];
    __atomic_store_n(&sl.seq, 0u, __ATOMIC_RELEASE);
    S->free_slots.push_back(it->second.slot);
    S->reqs.erase(it);
    return PVG_OK;
}

extern "C" pvg_status_t pvg_serve_counters(pvg_server_t *S, int64_t *queued, int64_t *batches, int64_t *views,
                                           int64_t *in_flight_bytes) {
    if (!S) return PVG_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (int64_t)S->queue.size();
    if (batches) *batches = S->batches;
    if (views) *views = S->views;
    if (in_flight_bytes) *in_flight_bytes = (int64_t)S->in_flight;
    return PVG_OK;
}

extern "C" pvg_status_t pvg_serve_arena(pvg_server_t *S, int64_t *requeues, int64_t *items_per_batch,
                                        int64_t *pixels_per_batch, int64_t *pairs_per_batch,
                                        int64_t *free_bytes_at_create) {
    if (!S) return PVG_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (requeues) *requeues = S->requeues;
    if (items_per_batch) *items_per_batch = (int64_t)S->cap_items;
    if (pixels_per_batch) *pixels_per_batch = (int64_t)S->cap_pix;
    if (pairs_per_batch) *pairs_per_batch = (int64_t)S->cap_pairs;
    if (free_bytes_at_create) *free_bytes_at_create = (int64_t)S->free_at_create;
    return PVG_OK;
}

extern "C" pvg_status_t pvg_serve_debug_withhold(pvg_server_t *S, int32_t n) {
    if (!S) return PVG_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    S->withhold = n > 0 ? n : 0;
    return PVG_OK;
}

extern "C" pvg_status_t pvg_serve_destroy(pvg_server_t *S) {
    if (!S) return PVG_ERR_INVALID;
    free_server(S);
    return PVG_OK;
}

// serve.cu -- continuous-batching render server (pvg_serve_*).
//
// Several scenes stay resident in HBM (caller-owned device arrays).
// Requests (scene, camera at time t, destination images) are queued on the
// host.  Each of `n_streams` worker threads owns a CUDA stream, a context
// (workspace) and a frame; a free worker takes requests from the head of
// the queue into a batch -- as many as fit under `max_batch_views` and the
// device-memory budget still free -- renders the whole batch with one
// pvg_render_fwd_multi launch sequence (views of different scenes and
// sizes share the sorts), waits for its stream, and completes the
// requests.  Requests that arrive while batches are on the GPU join the
// next batch of whichever worker frees first, so work of different
// batches overlaps on the device (continuous batching).  A request whose
// estimated working memory does not fit waits in the queue until enough
// finishes; a full queue makes pvg_serve_submit return PVG_ERR_BUSY.
//
// Each image depends only on its own request: per-pixel lists hold only
// the view's own Gaussians, in (depth, index) order, so a request renders
// bit-identically alone and in any batch.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pvg.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    int32_t scene = 0;
    pvg_camera_t cam;
    pvg_image_t dst;
    double t_submit = 0, t_start = -1, t_done = -1;
    int state = 0;  // 0 queued, 1 running, 2 done
    pvg_status_t status = PVG_OK;
    int32_t batch_views = 0;
    size_t mem = 0;
};

struct Worker {
    std::thread th;
    cudaStream_t stream = nullptr;
    pvg_ctx_t *ctx = nullptr;
    pvg_frame_t *frame = nullptr;
};

}  // namespace

struct pvg_server {
    pvg_serve_config_t cfg;
    int device = 0;
    Clock::time_point t0;
    std::vector<pvg_scene_t> scenes;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_id = 1;
    size_t in_flight = 0;
    bool stopping = false;
    std::vector<Worker> workers;
    int64_t batches = 0, views = 0;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

// working-memory estimate of one request: per-Gaussian buffers of its
// scene (204 bytes: counts, depth bits, stored projection, sort buffers and
// offsets in the context; depth order, inverse map, record, footprint
// ellipse, row table, rectangle and count in the frame), per-pixel state
// and an allowance of pairs per pixel
size_t request_bytes(const pvg_scene_t &sc, const pvg_camera_t &cam) {
    const size_t pix = (size_t)cam.width * cam.height;
    return (size_t)sc.n * 204 + pix * 12 + pix * 6 * 16;
}

void worker_loop(pvg_server *S, Worker *W) {
    cudaSetDevice(S->device);
    std::vector<uint64_t> ids;
    std::vector<pvg_scene_t> scenes;
    std::vector<pvg_camera_t> cams;
    std::vector<pvg_image_t> outs;
    for (;;) {
        size_t mem = 0;
        ids.clear();
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                if (S->stopping && S->queue.empty()) return;
                if (!S->queue.empty()) {
                    // take requests from the head while they fit
                    int deg = -1;
                    while (!S->queue.empty() && (int)ids.size() < S->cfg.max_batch_views) {
                        Req &r = S->reqs[S->queue.front()];
                        const int d = S->scenes[r.scene].sh_degree;
                        if (deg >= 0 && d != deg) break;  // one SH degree per launch
                        const bool alone = ids.empty() && S->in_flight == 0;
                        if (!alone && S->in_flight + mem + r.mem > (size_t)S->cfg.memory_budget) break;
                        deg = d;
                        mem += r.mem;
                        ids.push_back(S->queue.front());
                        S->queue.pop_front();
                    }
                    if (!ids.empty()) break;
                }
                S->cv_work.wait(lk);
            }
            S->in_flight += mem;
            const double t = S->now_ms();
            scenes.clear();
            cams.clear();
            outs.clear();
            for (uint64_t id : ids) {
                Req &r = S->reqs[id];
                r.state = 1;
                r.t_start = t;
                scenes.push_back(S->scenes[r.scene]);
                cams.push_back(r.cam);
                outs.push_back(r.dst);
            }
        }
        pvg_status_t st = pvg_render_fwd_multi(W->ctx, scenes.data(), cams.data(), (int32_t)ids.size(), outs.data(),
                                               W->frame, W->stream);
        if (cudaStreamSynchronize(W->stream) != cudaSuccess) {
            cudaGetLastError();
            if (st == PVG_OK) st = PVG_ERR_CUDA;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            const double t = S->now_ms();
            for (uint64_t id : ids) {
                Req &r = S->reqs[id];
                r.state = 2;
                r.t_done = t;
                r.status = st;
                r.batch_views = (int32_t)ids.size();
            }
            S->in_flight -= mem;
            S->batches += 1;
            S->views += (int64_t)ids.size();
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
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
        if (w.frame) pvg_frame_destroy(w.frame);
        if (w.ctx) pvg_destroy(w.ctx);
        if (w.stream) cudaStreamDestroy(w.stream);
    }
    S->workers.clear();
}

}  // namespace

extern "C" void pvg_serve_config_default(pvg_serve_config_t *c) {
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->max_batch_views = 16;
    c->n_streams = 2;
    c->memory_budget = (int64_t)8 << 30;
    c->max_pending = 4096;
    c->tile_w = 16;
    c->tile_h = 16;
    c->pixels_per_thread = 1;
}

extern "C" pvg_status_t pvg_serve_create(pvg_server_t **out, const pvg_serve_config_t *cfg) {
    if (!out) return PVG_ERR_INVALID;
    pvg_serve_config_t c;
    if (cfg) c = *cfg; else pvg_serve_config_default(&c);
    if (c.max_batch_views < 1 || c.n_streams < 1 || c.n_streams > 16 || c.memory_budget <= 0 ||
        c.max_pending < 1)
        return PVG_ERR_INVALID;
    pvg_config_t rc;
    pvg_config_default(&rc);
    rc.tile_w = c.tile_w;
    rc.tile_h = c.tile_h;
    rc.pixels_per_thread = c.pixels_per_thread;
    pvg_server *S = new pvg_server();
    S->cfg = c;
    S->t0 = Clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return PVG_ERR_CUDA;
    }
    S->workers.resize(c.n_streams);
    pvg_status_t st = PVG_OK;
    for (Worker &w : S->workers) {
        if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            st = PVG_ERR_CUDA;
            break;
        }
        if ((st = pvg_create(&w.ctx, &rc)) != PVG_OK) break;
        if ((st = pvg_frame_create(&w.frame)) != PVG_OK) break;
    }
    if (st != PVG_OK) {
        stop_workers(S);
        delete S;
        return st;
    }
    for (Worker &w : S->workers) w.th = std::thread(worker_loop, S, &w);
    *out = S;
    return PVG_OK;
}

extern "C" pvg_status_t pvg_serve_add_scene(pvg_server_t *S, const pvg_scene_t *scene, int32_t *scene_id) {
    if (!S || !scene || !scene_id || scene->n < 0 || scene->sh_degree < 0 || scene->sh_degree > 3)
        return PVG_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    S->scenes.push_back(*scene);
    *scene_id = (int32_t)S->scenes.size() - 1;
    return PVG_OK;
}

extern "C" pvg_status_t pvg_serve_submit(pvg_server_t *S, int32_t scene_id, const pvg_camera_t *cam,
                                         const pvg_image_t *dst, uint64_t *req_id) {
    if (!S || !cam || !dst || !dst->rgb || !req_id) return PVG_ERR_INVALID;
    if (dst->feat_mask != 0) return PVG_ERR_INVALID;  // served requests render colour, depth, opacity
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384) return PVG_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (scene_id < 0 || scene_id >= (int32_t)S->scenes.size()) return PVG_ERR_NOT_FOUND;
        if ((int64_t)S->queue.size() >= S->cfg.max_pending) return PVG_ERR_BUSY;
        const uint64_t id = S->next_id++;
        Req &r = S->reqs[id];
        r.scene = scene_id;
        r.cam = *cam;
        r.dst = *dst;
        r.t_submit = S->now_ms();
        r.mem = request_bytes(S->scenes[scene_id], *cam);
        S->queue.push_back(id);
        *req_id = id;
    }
    S->cv_work.notify_one();
    return PVG_OK;
}

static void fill_stats(const Req &r, pvg_req_stats_t *st) {
    if (!st) return;
    st->submit_ms = r.t_submit;
    st->start_ms = r.t_start;
    st->done_ms = r.t_done;
    st->batch_views = r.batch_views;
    st->status = r.status;
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

extern "C" pvg_status_t pvg_serve_destroy(pvg_server_t *S) {
    if (!S) return PVG_ERR_INVALID;
    stop_workers(S);
    delete S;
    return PVG_OK;
}

/*
 * pvg.h -- C ABI of the GB300-native PVG rasterizer.
 *
 * The library renders a set of Periodic Vibration Gaussians (PVG, arXiv
 * 2311.18561) seen by one or more pinhole cameras at given times into RGB,
 * depth and opacity images, and computes the adjoint of that map.  Every
 * step runs in CUDA kernels written for sm_103a; this header is the only
 * way in.  All signatures use plain pointers and sizes.
 *
 * Method (the passage each part follows):
 *   - time evaluation of every point (Sec. 3.2, Eq. 6 and Eq. 7):
 *       mu~(t) = mu + l/(2 pi) sin(2 pi (t - tau)/l) v,
 *       o~(t)  = o exp(-(t - tau)^2 / (2 beta^2));
 *   - the state H(t) = {mu~(t), q, s, o~(t), c} is rendered like a static
 *     3D Gaussian scene (Sec. 3.2, Eq. 8): EWA projection
 *     Sigma' = J W Sigma W^T J^T (Sec. 3.1, Eq. 2) with
 *     Sigma = R(q) diag(s)^2 R(q)^T, sorting by camera depth and per-tile
 *     front-to-back alpha blending C = sum_i T_i alpha_i c_i (Sec. 3.1,
 *     Eq. 3), plus the depth and opacity channels that Sec. 3.1
 *     renders beside colour and O = sum T_i alpha_i (Sec. 3.4, sky refinement);
 *   - optional background from a sky cube map, temporal-smoothing shift
 *     (Sec. 3.4) and extra channels: velocity, staticness and semantic maps
 *     (Sec. 4);
 *   - the render function is differentiable (Sec. 3.1, Eq. 4): the backward
 *     entry point returns gradients for mu, v, tau, beta, l, s, q, o and
 *     the SH colour coefficients.
 *
 * Conventions the paper leaves open (3DGS conventions it inherits), fixed
 * here: alpha = min(0.99, o~ G_2D); a Gaussian with alpha < 1/255 at a
 * pixel is skipped; blending stops before a Gaussian that would leave the
 * transmittance below 1e-4; EWA dilation h = 0.3 px^2 (configurable);
 * x/z and y/z clamped to 1.3 x the half field of view inside J; pixel
 * (px, py) is sampled at (px + 0.5, py + 0.5); camera axes are OpenCV
 * (+x right, +y down, +z forward); depth ties are broken by Gaussian index;
 * colour = max(0, sum_k sh_k Y_k(d) + 0.5) with real spherical harmonics
 * (orthonormal, Condon-Shortley phase, index k = l^2 + l + m) at the unit
 * direction d from the camera centre to mu~(t).
 *
 * Memory: every pointer inside pvg_scene_t, pvg_image_t, pvg_image_grad_t
 * and pvg_scene_grad_t is a DEVICE pointer owned by the caller.  Camera
 * arrays are HOST memory.  The library owns its workspace (pvg_ctx_t) and
 * the saved state of a forward pass (pvg_frame_t).  All calls are
 * asynchronous on the given stream unless stated otherwise; a NULL stream
 * is the legacy default stream.
 *
 * Errors: every call returns a pvg_status_t; no exception crosses the ABI.
 * On an error nothing has been enqueued unless the status is PVG_ERR_CUDA
 * (a CUDA call failed; the message is in pvg_last_error()).
 */
#ifndef PVG_H
#define PVG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PVG_OK = 0,
    PVG_ERR_INVALID = 1,   /* bad argument (NULL pointer, size, degree...) */
    PVG_ERR_OOM = 2,       /* a device allocation failed */
    PVG_ERR_BUSY = 3,      /* serving: request not admitted now, retry later */
    PVG_ERR_TIMEOUT = 4,   /* a bounded wait gave up */
    PVG_ERR_CUDA = 5,      /* a CUDA runtime call failed */
    PVG_ERR_OVERFLOW = 6,  /* more tile/Gaussian pairs than the fixed capacity */
    PVG_ERR_NOT_FOUND = 7  /* unknown scene or request id */
} pvg_status_t;

/* Human-readable name of a status. */
const char *pvg_status_str(pvg_status_t s);
/* Last CUDA error message recorded on this thread ("" if none). */
const char *pvg_last_error(void);
/* Library version as major*10000 + minor*100 + patch. */
int pvg_version(void);
/* Test hook for failure handling: the next n device allocations the library
 * attempts (workspace and frame growth in any context) fail as if the
 * device were out of memory, so the calls that needed them return
 * PVG_ERR_OOM; n <= 0 clears the hook.  Allocations that are not needed
 * (buffers already large enough) are not counted. */
void pvg_debug_fail_allocations(int32_t n);

/* ------------------------------------------------------------------ */
/* data                                                                */
/* ------------------------------------------------------------------ */

/* A PVG scene: N points, structure of arrays, float32, device memory,
 * row-major.  The learnable per-point set of Sec. 3.2:
 *   mu      [N,3]  mean position
 *   vel     [N,3]  v, vibration direction / velocity at the life peak
 *   tau     [N]    life peak
 *   beta    [N]    lifespan (> 0)
 *   period  [N]    cycle length l (> 0); the paper fixes l = 0.2
 *   scale   [N,3]  s (> 0, linear, not log)
 *   quat    [N,4]  q = (w, x, y, z), need not be normalised (not all zero)
 *   opacity [N]    o in [0, 1] (physical, not a logit)
 *   sh      [N,(D+1)^2,3] colour coefficients, D = sh_degree in 0..3
 * Every array must be 4-byte aligned; mu, vel, scale, quat and sh may be
 * any alignment of float.  N = 0 is allowed (renders the background).
 *   sky     [6,R,R,3] optional learnable sky cube map (Sec. 3.4, sky
 *           refinement): when non-NULL the background of every view is
 *           (1 - O) f_sky(d) instead of T_final bg, d the pixel's world ray
 *           direction, faces +X -X +Y -Y +Z -Z with the OpenGL cube-map
 *           face coordinates, bilinear inside a face, edges clamped;
 *           R = sky_res (>= 1).
 *   sem     [N,n_sem] optional per-point semantic vector (semantic
 *           rendering, Sec. 4: 19 class probabilities in the paper),
 *           1 <= n_sem <= PVG_MAX_SEM; needed only for PVG_FEAT_SEM. */
typedef struct {
    int64_t n;
    int32_t sh_degree;
    int32_t sky_res;
    const float *mu, *vel, *tau, *beta, *period, *scale, *quat, *opacity, *sh;
    const float *sky;
    const float *sem;
    int32_t n_sem;
    int32_t reserved0;
} pvg_scene_t;

/* Extra composited channels (bit mask, pvg_image_t.feat_mask).  Each is a
 * per-point value x_i composited with the colour's weights and no
 * background, sum_i T_i alpha_i x_i:
 *   PVG_FEAT_VBAR  3 channels, the average velocity v_bar = v exp(-rho/2),
 *                  rho = beta / l (Eq. 10), world frame -- the velocity
 *                  map of Sec. 3.4 / Sec. 4;
 *   PVG_FEAT_RHO   1 channel, the staticness rho = beta / l clamped to
 *                  [0, 2] (the rho map of the dynamic-element analysis,
 *                  Sec. 4; small = dynamic, large = static);
 *   PVG_FEAT_SEM   n_sem channels, the scene's semantic vectors.
 * The feature image holds the selected channels in this order. */
#define PVG_FEAT_VBAR 1
#define PVG_FEAT_RHO 2
#define PVG_FEAT_SEM 4
#define PVG_MAX_SEM 32

/* A pinhole camera at time t (host memory). */
typedef struct {
    float viewmat[12];  /* world->camera, row-major 3x4 [R | t], OpenCV axes */
    float fx, fy, cx, cy;
    int32_t width, height; /* 1..16384 each */
    float t;            /* render time (Sec. 3.2: normalised timestamps) */
    float z_near;       /* points with camera depth <= z_near are culled */
    float bg[3];        /* constant background colour (C += T_final bg) */
    float dt;           /* temporal smoothing (Sec. 3.4): 0 renders H(t); otherwise
                         * the flow-translated state: every point queried at
                         * t - dt and moved by v_bar dt, v_bar = v exp(-beta/(2 l))
                         * (Eq. 10), with its opacity at t - dt */
    const float *sky_jitter; /* optional DEVICE array [2,H,W]: x and y offsets in
                         * pixels of each pixel's sky ray (the paper jitters the
                         * sky ray within its pixel during training); NULL = 0 */
} pvg_camera_t;

/* Output images of one view (device memory, caller-owned):
 *   rgb   [3,H,W] planar, required
 *   depth [H,W]  sum_i T_i alpha_i z_i (not normalised; divide by alpha
 *                for the normalised depth of Sec. 3.1), may be NULL
 *   alpha [H,W]  O = sum_i T_i alpha_i, may be NULL
 *   feat  [F,H,W] planar extra channels selected by feat_mask (PVG_FEAT_*;
 *                F = 3 [VBAR] + 1 [RHO] + n_sem [SEM]); required when
 *                feat_mask != 0.  Every view of one call must use the same
 *                feat_mask; the scene(s) must carry sem for PVG_FEAT_SEM
 *                (and, for several scenes, the same n_sem). */
typedef struct {
    float *rgb, *depth, *alpha;
    float *feat;
    int32_t feat_mask;
    int32_t reserved0;
} pvg_image_t;

/* dL/d(output) of one view, same layouts as pvg_image_t; NULL = zero.
 * feat uses the channels of the forward pass that filled the frame. */
typedef struct {
    const float *rgb, *depth, *alpha;
    const float *feat;
} pvg_image_grad_t;

/* Parameter gradients, same layouts as pvg_scene_t (device, caller-owned).
 * pvg_render_bwd zeroes them and then writes dL/dparam summed over all
 * views.  A NULL array is neither zeroed nor written.  sky: dL/d(sky
 * texels), used when the scene has a sky map.  sem: dL/d(semantic
 * vectors) [N,n_sem], used when the frame's forward rendered
 * PVG_FEAT_SEM.  The feature channels also reach vel, beta and period
 * (through v_bar and rho; rho's clamp passes no gradient at rho >= 2) and
 * the geometry (through the blending weights). */
typedef struct {
    float *mu, *vel, *tau, *beta, *period, *scale, *quat, *opacity, *sh;
    float *sky;
    float *sem;
} pvg_scene_grad_t;

/* ------------------------------------------------------------------ */
/* context and saved state                                             */
/* ------------------------------------------------------------------ */

typedef struct pvg_ctx pvg_ctx_t;
typedef struct pvg_frame pvg_frame_t;

typedef struct {
    int32_t tile_w, tile_h; /* tile shape, 16x16 by default */
    int32_t sync_sizes;     /* 1 (default): pvg_render_fwd reads the pair count
                             * back to the host once per call and grows the
                             * workspace; 0: never synchronises, uses the
                             * capacities below; pairs beyond the capacity are
                             * dropped and pvg_frame_stats reports the
                             * overflow (the images are then incomplete) */
    int32_t pixels_per_thread; /* compositing pixels per thread (1, 2 or 4; 0 = 1).
                             * Supported (tile_w, tile_h, pixels_per_thread):
                             * (16,16,1|2|4) (8,8,1|2) (16,8,1|2) (32,8,1)
                             * (32,16,1|2|4) (32,32,4) (16,32,4).  Images do not
                             * depend on the choice (bit-identical). */
    int64_t pair_capacity;  /* pairs per frame when sync_sizes = 0 */
    float dilation;         /* EWA low-pass h in px^2 (default 0.3) */
    float fov_clamp;        /* J clamp factor (default 1.3) */
    float reserved[6];
} pvg_config_t;

/* Fill *cfg with the defaults. */
void pvg_config_default(pvg_config_t *cfg);

/* Create a context on the CURRENT CUDA device.  cfg may be NULL
 * (defaults).  The context owns scratch memory that grows on demand; it is
 * used by one stream at a time (calls on one context must not overlap). */
pvg_status_t pvg_create(pvg_ctx_t **ctx, const pvg_config_t *cfg);
void pvg_destroy(pvg_ctx_t *ctx);
/* Change tile shape / dilation / clamp of an existing context. */
pvg_status_t pvg_set_config(pvg_ctx_t *ctx, const pvg_config_t *cfg);

/* Saved state of one forward pass (depth-sorted visible Gaussians, their
 * projected records, per-tile lists, per-pixel final transmittance and last
 * blended position), needed by pvg_render_bwd.  A frame belongs to the
 * device that was current at creation. */
pvg_status_t pvg_frame_create(pvg_frame_t **frame);
void pvg_frame_destroy(pvg_frame_t *frame);
/* Counters of the last forward into `frame` (synchronises `frame`'s last
 * stream): visible (view, Gaussian) pairs, tile/Gaussian pairs (one per
 * tile of a Gaussian's bounding rectangle that its footprint ellipse
 * o~ G >= 1/255, slightly widened, reaches) and the overflow status. */
pvg_status_t pvg_frame_stats(pvg_frame_t *frame, int64_t *n_visible, int64_t *n_pairs,
                             int32_t *overflowed);

/* ------------------------------------------------------------------ */
/* rendering                                                           */
/* ------------------------------------------------------------------ */

/* Render `scene` from `n_views` cameras (host array) into out[0..n_views)
 * (host array of device image pointers).  If `frame` is non-NULL the state
 * needed by pvg_render_bwd is kept in it (NULL: inference only).
 * Returns PVG_ERR_INVALID for NULL/size errors, PVG_ERR_OOM if the
 * workspace cannot grow. */
pvg_status_t pvg_render_fwd(pvg_ctx_t *ctx, const pvg_scene_t *scene, const pvg_camera_t *cams,
                            int32_t n_views, const pvg_image_t *out, pvg_frame_t *frame, void *stream);

/* Like pvg_render_fwd, but view v renders scenes[v] (host array of
 * n_views scene descriptors; several views may name the same arrays).  All
 * scenes must have the same SH degree.  Used to batch requests for
 * different scenes into one launch sequence; a frame rendered this way
 * with more than one distinct scene cannot be passed to pvg_render_bwd.
 *
 * CUDA-graph capture (both render entry points and pvg_render_bwd): a call
 * may be captured when the context was created with sync_sizes = 0 and the
 * same call (same sizes, same frame) has run once uncaptured, so that no
 * buffer has to grow; otherwise PVG_ERR_INVALID.  The view descriptors are
 * copied from pinned staging owned by the frame, a copy per capture that
 * nothing writes afterwards: a replayed graph renders the cameras and into
 * the images given at capture time, whatever later calls or captures on the
 * frame use (graphs of one frame share its device state, so they replay one
 * after another).  A graph is valid while its frame lives. */
pvg_status_t pvg_render_fwd_multi(pvg_ctx_t *ctx, const pvg_scene_t *scenes, const pvg_camera_t *cams,
                                  int32_t n_views, const pvg_image_t *out, pvg_frame_t *frame, void *stream);

/* Adjoint of the forward pass saved in `frame` (which must have been
 * rendered from the same scene values and cameras): zeroes `grads` and
 * writes dL/dparam for L = sum over views of <dL[v], image[v]>.
 * dL is a host array of n_views device-gradient descriptors.  `frame`
 * must be the frame the forward pass was given: with NULL, or a frame
 * whose last forward kept no state (a served frame), the call returns
 * PVG_ERR_INVALID and enqueues nothing. */
pvg_status_t pvg_render_bwd(pvg_ctx_t *ctx, const pvg_scene_t *scene, const pvg_camera_t *cams,
                            int32_t n_views, pvg_frame_t *frame, const pvg_image_grad_t *dL,
                            const pvg_scene_grad_t *grads, void *stream);

/* ------------------------------------------------------------------ */
/* serving                                                             */
/* ------------------------------------------------------------------ */

/* A render server: several scenes resident in HBM; render requests (scene,
 * camera at time t, destination images) of any size, time and pose are
 * batched into shared launch sequences while earlier batches are still on
 * the GPU (continuous batching).  There is no serving system in the paper
 * (it reports rendering speed only, Sec. 4 / Tab. 5); the design:
 *
 *   - Request ring.  pvg_serve_submit writes the request's view descriptor
 *     into a slot of a ring in mapped pinned memory, which the GPU reads
 *     directly, and then publishes the slot with a sequence number.
 *   - Launch sequences.  Each of `n_streams` workers (a thread, a CUDA
 *     stream, a workspace) takes queued requests into a batch and enqueues
 *     one launch sequence for it without waiting for its earlier batches
 *     (up to pipeline_depth in flight): a gather kernel waits for every
 *     slot of the batch to be published -- a bounded wait of at most
 *     gate_timeout_us, after which the slot's request completes with
 *     PVG_ERR_TIMEOUT and its view renders nothing -- and copies the
 *     descriptors into the workspace; the forward render of all the batch's
 *     views follows (one depth sort, one tile sort, one compositing launch
 *     over every view's tiles); a completion kernel writes each slot's
 *     status, the batch's pair count and GPU timestamps back into the ring.
 *     The host learns of completion from those flags; no stream is
 *     synchronised per batch.
 *   - Admission by memory.  At creation the server measures the free
 *     device memory (cudaMemGetInfo) and reserves for every worker an arena
 *     of min(memory_budget, 90 % of the free memory) / n_streams bytes:
 *     capacities for Gaussians, pixels, tiles and tile/Gaussian pairs per
 *     batch.  A batch takes requests from the head of the queue while their
 *     sum fits the arena; the pairs of a request are estimated from the
 *     pairs per pixel its scene produced before.  The GPU counts the pairs
 *     of the batch before emitting them; if the count exceeds the batch's
 *     reservation the batch's requests go back to the head of the queue
 *     with the measured count (count, reserve, then continue or requeue).
 *     The first request of a batch is always taken, so a request larger
 *     than an arena is rendered alone in a workspace grown for it.
 *
 * Every request renders bit-identically alone and in any batch, and equal
 * to pvg_render_fwd of the same scene and camera.  The server uses the
 * device that is current at creation. */
typedef struct pvg_server pvg_server_t;

typedef struct {
    int32_t max_batch_views;  /* views per launch sequence, 1..64 (default 16) */
    int32_t n_streams;        /* workers, each with its own stream and arena, 1..16 (default 4) */
    int64_t memory_budget;    /* bytes of the workers' arenas together (default 8 GiB), clamped to
                               * 90 % of the free device memory at creation */
    int32_t max_pending;      /* queued requests before submit returns PVG_ERR_BUSY (default 4096) */
    int32_t tile_w, tile_h, pixels_per_thread; /* compositing configuration (16, 16, 1) */
    int32_t gate_timeout_us;  /* bound of the gather kernel's wait for a slot (default 1,000,000) */
    int32_t pipeline_depth;   /* batches a worker keeps in flight, 1..4 (default 1) */
    int32_t pair_capacity;    /* pairs per batch; 0 (default) = the arena's share */
    int32_t reserved0;
} pvg_serve_config_t;

/* Per-request timing in milliseconds since the server was created (host
 * clock; start is the launch of the request's batch, done the moment the
 * host saw its completion flag), -1 until reached; gpu_ms = GPU time from
 * the gather kernel to the completion kernel of its batch. */
typedef struct {
    double submit_ms, start_ms, done_ms;
    int32_t batch_views;  /* views in the launch that rendered it */
    int32_t status;       /* pvg_status_t of the request */
    double gpu_ms;
    int32_t attempts;     /* launches it took (> 1 after a requeue) */
    int32_t reserved0;
} pvg_req_stats_t;

void pvg_serve_config_default(pvg_serve_config_t *cfg);
pvg_status_t pvg_serve_create(pvg_server_t **server, const pvg_serve_config_t *cfg);
/* Registers a resident scene (device arrays stay caller-owned and must
 * outlive the server); returns its id. */
pvg_status_t pvg_serve_add_scene(pvg_server_t *server, const pvg_scene_t *scene, int32_t *scene_id);
/* Queues a request; never blocks.  dst: device images ([3,H,W] rgb
 * required, depth / alpha may be NULL), written when the request is done.
 * PVG_ERR_BUSY if max_pending requests are already queued,
 * PVG_ERR_NOT_FOUND for an unknown scene id. */
pvg_status_t pvg_serve_submit(pvg_server_t *server, int32_t scene_id, const pvg_camera_t *cam,
                              const pvg_image_t *dst, uint64_t *req_id);
/* Non-blocking status: *done = 1 once the images are written. */
pvg_status_t pvg_serve_poll(pvg_server_t *server, uint64_t req_id, int32_t *done, pvg_req_stats_t *stats);
/* Blocks until the request is done or timeout_ms elapsed (PVG_ERR_TIMEOUT);
 * returns the status of the launch that rendered it. */
pvg_status_t pvg_serve_wait(pvg_server_t *server, uint64_t req_id, double timeout_ms, pvg_req_stats_t *stats);
/* Forgets a finished request (PVG_ERR_BUSY if it is not done yet). */
pvg_status_t pvg_serve_release(pvg_server_t *server, uint64_t req_id);
/* Queue length, launches and views so far, estimated in-flight bytes. */
pvg_status_t pvg_serve_counters(pvg_server_t *server, int64_t *queued, int64_t *batches, int64_t *views,
                                int64_t *in_flight_bytes);
/* Requeues after a pair count above the reservation, and the per-worker
 * arena capacities: Gaussians, pixels and pairs per batch, and the free
 * device memory measured at creation. */
pvg_status_t pvg_serve_arena(pvg_server_t *server, int64_t *requeues, int64_t *items_per_batch,
                             int64_t *pixels_per_batch, int64_t *pairs_per_batch, int64_t *free_bytes_at_create);
/* Test hook for the bounded device-side wait: the next n requests
 * submitted to `server` are queued but their ring slots are never
 * published, so the gather kernel's wait runs out after gate_timeout_us
 * and they complete with PVG_ERR_TIMEOUT (their images are not written);
 * the batches they were in, and the server, go on normally.  n <= 0
 * clears it. */
pvg_status_t pvg_serve_debug_withhold(pvg_server_t *server, int32_t n);
/* Finishes every queued request, stops the workers and frees the server. */
pvg_status_t pvg_serve_destroy(pvg_server_t *server);

/* ------------------------------------------------------------------ */
/* sorting                                                             */
/* ------------------------------------------------------------------ */

/* Stable LSD radix sort of n (key, value) pairs by bits [begin_bit,
 * end_bit) of the key, in place, on `stream` -- the sort the renderer uses
 * for the depth sort of Sec. 3.1 (camera-space depth order of the
 * Gaussians): float32 depth bits of the visible Gaussians, then tile ids
 * of the (tile, Gaussian) pairs.  keys / vals: caller-owned device arrays
 * of n uint32 each.  Pairs with equal sort bits keep their input order.
 * Scratch (ping-pong buffers of n pairs, digit histograms) belongs to
 * `ctx` and grows on demand.  PVG_ERR_INVALID if n < 0, n >= 2^32, a
 * pointer is NULL while n > 0, or not 0 <= begin_bit < end_bit <= 32. */
pvg_status_t pvg_sort_pairs(pvg_ctx_t *ctx, uint32_t *keys, uint32_t *vals, int64_t n, int32_t begin_bit,
                            int32_t end_bit, void *stream);

/* The sort of pvg_sort_pairs for callers that cannot allocate device
 * memory (code running during CUDA-graph capture, real-time or callback
 * threads where cudaMalloc may block on a device-wide synchronisation,
 * hosts that forbid allocations outside their own pool).  The paper has no
 * counterpart; this is an interface convenience.  It needs no context and
 * calls no cudaMalloc / cudaFree or allocating routine: its scratch is a
 * set of fixed device arrays inside this library (about 9.1 MiB, held on
 * every GPU that loads the library until the process exits).
 *   - n must be <= 1,048,576 (2^20); larger n returns PVG_ERR_INVALID and
 *     enqueues nothing.  Other arguments as for pvg_sort_pairs.
 *   - The first call on a device looks up that device's array addresses
 *     (cudaGetSymbolAddress); make that first call before any stream
 *     capture.
 *   - All calls share the arrays and leave the last call's contents in
 *     them: calls that overlap on the GPU (different streams or devices'
 *     threads racing on one device) race and corrupt each other's results;
 *     serialise them. */
pvg_status_t pvg_sort_pairs_noalloc(uint32_t *keys, uint32_t *vals, int64_t n, int32_t begin_bit,
                                    int32_t end_bit, void *stream);

/* ------------------------------------------------------------------ */
/* loss                                                                */
/* ------------------------------------------------------------------ */

/* L1 photometric term of the objective (Sec. 3.4, L = (1 - lambda_r) L1 +
 * ...): *loss = scale * sum_i |pred[i] - target[i]| and, if dl is
 * non-NULL, dl[i] = scale * sign(pred[i] - target[i]) (0 where equal).
 * All pointers are device memory of n floats (loss: one float, overwritten).
 * scale = 1/n gives the mean.  The sum is taken in a fixed order (per-block
 * partial sums added in block order), so the loss is bit-reproducible for
 * the same inputs on the same device.  Uses a small scratch array of ctx
 * (allocated by the first call; calls on one ctx must not overlap);
 * capturable in a CUDA graph after one uncaptured call.
 * n = 0 writes *loss = 0 (pred, target and dl may then be NULL).
 * PVG_ERR_INVALID for NULL pointers or n < 0. */
pvg_status_t pvg_l1_loss(pvg_ctx_t *ctx, const float *pred, const float *target, int64_t n, float scale,
                         float *dl, float *loss, void *stream);

/* Photometric loss of the objective (Sec. 3.4):
 *   L = (1 - lambda_r) L1 + lambda_r (1 - SSIM)   (the paper uses 0.2),
 * L1 = mean |pred - target|, SSIM the mean of the per-channel SSIM map of
 * 3D Gaussian Splatting (11x11 Gaussian window, sigma 1.5, zero padding,
 * C1 = 0.01^2, C2 = 0.03^2).  pred, target: device [channels, H, W]
 * planar float32; loss: device float[3] receiving (L, L1, SSIM); dl: device
 * [channels, H, W] receiving dL/dpred (sign(0) = 0), or NULL.  One fused
 * pass plus a fixed-order reduction (deterministic).  Uses ctx's workspace
 * (must not overlap other calls on ctx); capturable once the workspace has
 * grown to the image size.  PVG_ERR_INVALID for NULL pointers, sizes
 * outside 1..16384 (channels 1..65535) or lambda_r outside [0, 1]. */
pvg_status_t pvg_rgb_loss(pvg_ctx_t *ctx, const float *pred, const float *target, int32_t channels,
                          int32_t height, int32_t width, float lambda_r, float *dl, float *loss, void *stream);

/* ------------------------------------------------------------------ */
/* measurement and introspection                                       */
/* ------------------------------------------------------------------ */

/* Kernels this library has launched since it was loaded (all contexts). */
uint64_t pvg_kernel_launches(void);

/* Streaming multiprocessors of the current device, as the library sizes its
 * grids with them (cudaDevAttrMultiProcessorCount, read once per device). */
int32_t pvg_device_sm_count(void);

/* FP32 throughput probe, the measured peak of the compositing kernels'
 * roofline (not part of the rendering path): `blocks` blocks of 256
 * threads, every thread running `iters` rounds of 128 fused multiply-adds
 * in 8 independent chains x <- fma(x, a, b), then writing one float into
 * dst (device, blocks * 256 floats, so nothing is optimised away).  The
 * caller times the launch on `stream`: lane FMAs = blocks * 256 * iters *
 * 128.  Choose |a| < 1 so that the chains stay finite.
 * PVG_ERR_INVALID for dst NULL, blocks < 1 or iters < 1. */
pvg_status_t pvg_fma_probe(float *dst, int32_t blocks, int64_t iters, float a, float b, void *stream);

/* Stages timed by pvg_profile_* (CUDA events on the call's stream). */
enum {
    PVG_STAGE_PROJECT = 0,        /* time evaluation, projection, tile counts */
    PVG_STAGE_DEPTH_SORT = 1,     /* visible compaction + depth radix sort */
    PVG_STAGE_FINALIZE = 2,       /* records (incl. SH colour) in depth order */
    PVG_STAGE_PAIRS = 3,          /* pair count scan + emission */
    PVG_STAGE_TILE_SORT = 4,      /* tile-id radix sort + tile ranges */
    PVG_STAGE_COMPOSITE = 5,      /* per-tile alpha compositing */
    PVG_STAGE_COMPOSITE_BWD = 6,  /* compositing adjoint (image-space grads) */
    PVG_STAGE_PREPROCESS_BWD = 7, /* chain rule to the PVG parameters */
    PVG_NUM_STAGES = 8
};
/* Record CUDA events around every stage of later calls on `ctx` (on: 1). */
pvg_status_t pvg_profile_enable(pvg_ctx_t *ctx, int on);
/* Waits for the recorded events, writes the summed milliseconds and the
 * number of timed calls per stage into ms[8] / calls[8] (host arrays), and
 * forgets them. */
pvg_status_t pvg_profile_read(pvg_ctx_t *ctx, double *ms, int64_t *calls);

/* The compositing work of the last forward into `frame`, summed over all
 * pixels: *evals = entries of the pixel's tile list whose footprint box
 * contains the pixel, up to and including the entry that stopped it (E);
 * *blends (may be NULL) = those among them with alpha >= 1/255 (blended or
 * stopping the pixel).  Re-runs the compositor in a counting mode (writes
 * no image) with `ctx`'s scratch; synchronises the frame's stream. */
pvg_status_t pvg_frame_eval_count(pvg_ctx_t *ctx, pvg_frame_t *frame, int64_t *evals, int64_t *blends);

/* Copy device-side intermediate results of the last forward into
 * caller-owned DEVICE buffers (any may be NULL), for parity testing:
 *   sorted_gid [n_visible]   (view * N + index) in (view-major via tiles, depth, index) order
 *   depth_key  [n_visible]   float32 bits of the camera depth, same order
 *   rect       [n_visible*4] tile rectangle (tx0, ty0, tx1, ty1) of the footprint box,
 *                            half-open, int32 (a Gaussian's pairs are the tiles of it
 *                            that its footprint ellipse reaches)
 *   records    [n_visible*12] u, v, conic a, b, c, o~, z, hx, r, g, b, hy (float32;
 *                            hx, hy = footprint half extents in pixels)
 *   pair_vals  [n_pairs]     position in the depth order, sorted by (tile, depth, index);
 *                            each tile's list is that of the rectangles without the
 *                            Gaussians whose footprint ellipse misses the tile
 *   ranges     [total_tiles*2] [start, end) per tile, tiles of view 0 first
 * Synchronises the frame's stream. */
pvg_status_t pvg_frame_export(pvg_frame_t *frame, uint32_t *sorted_gid, uint32_t *depth_key,
                              int32_t *rect, float *records, uint32_t *pair_vals, uint32_t *ranges);

#ifdef __cplusplus
}
#endif
#endif /* PVG_H */

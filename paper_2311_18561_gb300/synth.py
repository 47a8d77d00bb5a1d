"""Seeded synthetic inputs: PVG scenes, cameras, view batches and request streams.

This module only draws numbers. It holds none of the renderer's arithmetic
(no time evaluation, projection, colour or compositing), so both the CUDA
path and the FP64 oracle can be fed the very same bytes from it.

The paper's workloads are posed Waymo / KITTI captures with trained PVG
scenes (Sec. 4, "Implementation details" and Tab. 1/5); neither the data nor
the trained scenes are available, so these generators stand in for them with
the shapes and value distributions of the paper's setting:

* time is normalised to [0, 1] over 50 frames (the paper rescales the frame
  spacing to 0.02, Sec. 4 "Implementation details");
* one normalised time unit is 5 s of a 10 Hz capture, so a speed in m/s is
  multiplied by 5 to become a velocity in metres per time unit;
* camera axes follow OpenCV: +x right, +y down, +z forward; a view matrix is
  the 3x4 row-major world->camera transform [R | t].

A scene is a dict of float32 numpy arrays::

    mu [N,3]  vel [N,3]  tau [N]  beta [N]  period [N]  scale [N,3]
    quat [N,4] (w,x,y,z; not normalised)  opacity [N]  sh [N,(D+1)^2,3]

and a camera is a dict with ``viewmat`` (3x4), ``fx fy cx cy``, ``width``,
``height``, ``t``, ``z_near``, ``bg`` (3,) and ``dt`` (temporal-smoothing
shift of the rendered state, 0 for a plain render).
"""
from __future__ import annotations

import math

import numpy as np

F32 = np.float32

# Degree-0 real spherical harmonic value, 1 / (2 sqrt(pi)): used only to draw
# DC coefficients whose degree-0 colour is uniform in [0, 1].
_Y00 = 0.5 / math.sqrt(math.pi)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _random_quats(rng, n):
    return rng.normal(size=(n, 4)).astype(np.float64)


def _pack(mu, vel, tau, beta, period, scale, quat, opacity, sh):
    scene = dict(mu=mu, vel=vel, tau=tau, beta=beta, period=period, scale=scale,
                 quat=quat, opacity=opacity, sh=sh)
    return {k: np.ascontiguousarray(v, dtype=F32) for k, v in scene.items()}


def sh_degree_of(scene) -> int:
    k = scene["sh"].shape[1]
    d = int(round(math.sqrt(k))) - 1
    assert (d + 1) ** 2 == k
    return d


def num_gaussians(scene) -> int:
    return int(scene["mu"].shape[0])


# ---------------------------------------------------------------------------
# scenes
# ---------------------------------------------------------------------------

def make_plain_scene(seed: int = 0, n: int = 2000, sh_degree: int = 0,
                     log_scale_mean: float = -3.0, log_scale_std: float = 0.5):
    """The 2,000-Gaussian plain scene: mu ~ U[-1,1]^3, v ~ N(0, 0.2^2),
    tau ~ U[0,1], l ~ LogNormal(0, 0.3), beta ~ U[0.1, 2],
    log-scale ~ N(-3, 0.5), random rotation, opacity = sigmoid(N(0,1)),
    degree-0 colour ~ U[0,1] (higher SH bands, if asked for, ~ N(0, 0.1^2))."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-1.0, 1.0, size=(n, 3))
    vel = rng.normal(0.0, 0.2, size=(n, 3))
    tau = rng.uniform(0.0, 1.0, size=n)
    period = rng.lognormal(0.0, 0.3, size=n)
    beta = rng.uniform(0.1, 2.0, size=n)
    scale = np.exp(rng.normal(log_scale_mean, log_scale_std, size=(n, 3)))
    quat = _random_quats(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.0, size=n))
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = (rgb - 0.5) / _Y00
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, size=(n, k - 1, 3))
    scene = _pack(mu, vel, tau, beta, period, scale, quat, opacity, sh)
    scene["_rgb0"] = rgb.astype(F32)  # the drawn degree-0 colour (test aid)
    return scene


def make_urban_scene(n: int, seed: int = 0, sh_degree: int = 3):
    """Urban-shaped scene in a 200 x 60 x 20 m slab (x along the street,
    z up).  70 % ground points (z in [0, 0.5]), 10 % facade points
    (y = +-15 m + N(0, 0.3), z in [0, 20]) and 20 % points in 300 object
    clusters (sigma 1 m, z in [0, 3]).  The cluster points are the dynamic
    20 %: each cluster moves with one speed U[0, 15] m/s in a random ground
    plane direction and its points get beta ~ U[0.05, 0.5].  The static 80 %
    get |v| < 0.05 m/s and beta ~ U[5, 10].  tau ~ U[0,1],
    l ~ LogNormal(0, 0.5), SH coefficients ~ N(0, 0.1^2),
    log-scale ~ N(-2, 0.5), opacity = sigmoid(N(0,1))."""
    rng = np.random.default_rng(seed)
    n_ground = int(round(0.7 * n))
    n_facade = int(round(0.1 * n))
    n_obj = n - n_ground - n_facade
    mu = np.empty((n, 3))
    # ground
    g = slice(0, n_ground)
    mu[g, 0] = rng.uniform(-100.0, 100.0, n_ground)
    mu[g, 1] = rng.uniform(-30.0, 30.0, n_ground)
    mu[g, 2] = rng.uniform(0.0, 0.5, n_ground)
    # facades
    f = slice(n_ground, n_ground + n_facade)
    side = np.where(rng.uniform(size=n_facade) < 0.5, -15.0, 15.0)
    mu[f, 0] = rng.uniform(-100.0, 100.0, n_facade)
    mu[f, 1] = side + rng.normal(0.0, 0.3, n_facade)
    mu[f, 2] = rng.uniform(0.0, 20.0, n_facade)
    # object clusters (dynamic)
    o = slice(n_ground + n_facade, n)
    n_clusters = 300
    centers = np.stack([rng.uniform(-100.0, 100.0, n_clusters),
                        rng.uniform(-12.0, 12.0, n_clusters)], axis=1)
    cid = rng.integers(0, n_clusters, n_obj)
    mu[o, 0:2] = centers[cid] + rng.normal(0.0, 1.0, (n_obj, 2))
    mu[o, 2] = rng.uniform(0.0, 3.0, n_obj)

    vel = np.zeros((n, 3))
    beta = np.empty(n)
    # static: |v| < 0.05 m/s, random ground-plane direction
    n_static = n_ground + n_facade
    ang = rng.uniform(0.0, 2.0 * math.pi, n_static)
    spd = rng.uniform(0.0, 0.05, n_static) * 5.0
    vel[:n_static, 0] = spd * np.cos(ang)
    vel[:n_static, 1] = spd * np.sin(ang)
    beta[:n_static] = rng.uniform(5.0, 10.0, n_static)
    # dynamic: one velocity per cluster
    c_ang = rng.uniform(0.0, 2.0 * math.pi, n_clusters)
    c_spd = rng.uniform(0.0, 15.0, n_clusters) * 5.0
    vel[o, 0] = (c_spd * np.cos(c_ang))[cid]
    vel[o, 1] = (c_spd * np.sin(c_ang))[cid]
    beta[o] = rng.uniform(0.05, 0.5, n_obj)

    tau = rng.uniform(0.0, 1.0, n)
    period = rng.lognormal(0.0, 0.5, n)
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.1, (n, k, 3))
    scale = np.exp(rng.normal(-2.0, 0.5, (n, 3)))
    quat = _random_quats(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.0, n))
    return _pack(mu, vel, tau, beta, period, scale, quat, opacity, sh)


def make_fd_scene(seed: int = 0, n: int = 500, sh_degree: int = 3):
    """Small dynamic scene for finite-difference checks (500 Gaussians,
    viewed at 64x48 by :func:`fd_camera`): mu ~ U[-1,1]^3 with larger splats
    (log-scale ~ N(-2.3, 0.3)) so that each covers a few pixels, dynamic
    parameters as in the plain scene and SH bands ~ N(0, 0.2^2)."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-1.0, 1.0, size=(n, 3))
    vel = rng.normal(0.0, 0.3, size=(n, 3))
    tau = rng.uniform(0.0, 1.0, size=n)
    period = rng.lognormal(0.0, 0.3, size=n)
    beta = rng.uniform(0.2, 2.0, size=n)
    scale = np.exp(rng.normal(-2.3, 0.3, size=(n, 3)))
    quat = _random_quats(rng, n)
    opacity = _sigmoid(rng.normal(-0.5, 1.0, size=n))
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.2, size=(n, k, 3))
    sh[:, 0, :] = (rng.uniform(0.2, 0.8, size=(n, 3)) - 0.5) / _Y00
    return _pack(mu, vel, tau, beta, period, scale, quat, opacity, sh)


def subset(scene, idx):
    return {k: np.ascontiguousarray(v[idx]) for k, v in scene.items()}


# ---------------------------------------------------------------------------
# cameras
# ---------------------------------------------------------------------------

def look_at(eye, target, up):
    """World->camera 3x4 matrix with OpenCV axes (x right, y down, z fwd)."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    down = -np.asarray(up, np.float64)
    down = down - fwd * np.dot(down, fwd)
    down /= np.linalg.norm(down)
    right = np.cross(down, fwd)
    rot = np.stack([right, down, fwd], axis=0)
    trans = -rot @ eye
    return np.concatenate([rot, trans[:, None]], axis=1)


def make_camera(viewmat, width, height, fx, fy=None, cx=None, cy=None, t=0.5,
                z_near=0.2, bg=(0.0, 0.0, 0.0), dt=0.0):
    fy = fx if fy is None else fy
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    return dict(viewmat=np.asarray(viewmat, np.float32).reshape(3, 4),
                fx=float(fx), fy=float(fy), cx=float(cx), cy=float(cy),
                width=int(width), height=int(height), t=float(t),
                z_near=float(z_near), bg=np.asarray(bg, np.float32).reshape(3), dt=float(dt))


def focal_from_hfov(width, hfov_deg):
    return (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)


def plain_camera(width=160, height=120, hfov_deg=60.0, t=0.5, bg=(0.0, 0.0, 0.0)):
    """Camera at (0,0,-4) looking at the origin, world +y up."""
    vm = look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    return make_camera(vm, width, height, focal_from_hfov(width, hfov_deg), t=t, bg=bg)


def fd_camera(width=64, height=48, t=0.4):
    vm = look_at((0.0, 0.0, -3.5), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    return make_camera(vm, width, height, focal_from_hfov(width, 55.0), t=t)


def street_camera(t, width=1920, height=1280, hfov_deg=50.0, fx=None, lateral=0.0,
                  height_m=1.6, yaw_deg=0.0):
    """A camera 1.6 m above the ground moving down the street:
    x = -90 + 180 t, looking along +x (optionally yawed)."""
    x = -90.0 + 180.0 * t
    eye = (x, lateral, height_m)
    yaw = math.radians(yaw_deg)
    target = (x + math.cos(yaw), lateral + math.sin(yaw), height_m)
    vm = look_at(eye, target, (0.0, 0.0, 1.0))
    f = focal_from_hfov(width, hfov_deg) if fx is None else fx
    return make_camera(vm, width, height, f, t=t)


def urban_frame_camera(frame=25, width=1920, height=1280, hfov_deg=50.0):
    """Frame f of the 50-frame street path, t = f / 49."""
    return street_camera(frame / 49.0, width, height, hfov_deg)


def kitti_camera(t=0.5, width=1242, height=375, focal=720.0):
    return street_camera(t, width, height, fx=focal)


def batched_views(seed=0, n_views=64):
    """64 views: 22 at 1920x1280 (hfov 50), 21 at 1242x375 (f = 720) and
    21 at 960x640 (hfov 50), each with its own t ~ U[0,1] on the street path."""
    rng = np.random.default_rng(seed)
    shapes = ([(1920, 1280, None)] * 22 + [(1242, 375, 720.0)] * 21
              + [(960, 640, None)] * 21)
    shapes = (shapes * ((n_views + len(shapes) - 1) // len(shapes)))[:n_views]
    cams = []
    for (w, h, f) in shapes:
        t = float(rng.uniform(0.0, 1.0))
        cams.append(street_camera(t, w, h, fx=f))
    return cams


SERVE_RESOLUTIONS = ((640, 480), (1242, 375), (1920, 1280))
SERVE_SCENE_SIZES = (500_000, 1_000_000, 2_000_000, 4_000_000)


def serve_requests(rate_hz, duration_s, n_scenes=4, seed=0):
    """Poisson arrivals at ``rate_hz`` for ``duration_s`` seconds.  Each
    request draws a scene, t ~ U[0,1], a pose on the street path at t with a
    lateral offset U[-2, 2] m, and a resolution from SERVE_RESOLUTIONS.
    Returns a list of (arrival_s, scene_id, camera)."""
    rng = np.random.default_rng(seed)
    out = []
    now = 0.0
    while True:
        now += float(rng.exponential(1.0 / rate_hz))
        if now >= duration_s:
            break
        sid = int(rng.integers(0, n_scenes))
        t = float(rng.uniform(0.0, 1.0))
        w, h = SERVE_RESOLUTIONS[int(rng.integers(0, len(SERVE_RESOLUTIONS)))]
        cam = street_camera(t, w, h, lateral=float(rng.uniform(-2.0, 2.0)))
        out.append((now, sid, cam))
    return out


def random_image(height, width, seed=1):
    """Target image ~ U[0,1]^3, planar [3, H, W]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(3, height, width)).astype(F32)


def make_semantics(n, n_classes=19, seed=3, one_hot=False):
    """Per-Gaussian class-probability vectors [n, n_classes] (19 classes in
    the paper's semantic rendering): a softmax of N(0, 1.5^2) logits, or
    one-hot rows of a uniformly drawn class."""
    rng = np.random.default_rng(seed)
    if one_hot:
        out = np.zeros((n, n_classes))
        out[np.arange(n), rng.integers(0, n_classes, size=n)] = 1.0
        return out.astype(F32)
    z = rng.normal(0.0, 1.5, size=(n, n_classes))
    z = np.exp(z - z.max(axis=1, keepdims=True))
    return (z / z.sum(axis=1, keepdims=True)).astype(F32)

"""Pins of the oracle's sky cube map (the sky step of Sec. 3.4:
C_f = C + (1 - O) f_sky(d), the sky colour depending only on the ray
direction d).  No GPU.

* a constant map renders as that constant behind an empty scene, and as
  alpha c_g + (1 - alpha) c behind one Gaussian (closed form);
* each axis direction lands on its own face;
* a map whose texels hold their own direction returns, for every pixel,
  that pixel's ray direction from the pinhole model (up to bilinear
  filtering), so faces, orientations and edges are consistent;
* the reverse mode matches FP64 finite differences for sky texels and for
  Gaussian parameters (whose opacity now also scales the sky).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_18561_gb300 import synth

Y00 = 0.5 / math.sqrt(math.pi)
# OpenGL cube-map faces (+X -X +Y -Y +Z -Z): (major axis, sign, s axis, s sign, t axis, t sign)
FACES = [(0, 1, 2, -1, 1, -1), (0, -1, 2, 1, 1, -1), (1, 1, 0, 1, 2, 1),
         (1, -1, 0, 1, 2, -1), (2, 1, 0, 1, 1, -1), (2, -1, 0, -1, 1, -1)]


def texel_directions(R):
    """[6, R, R, 3] unit direction through each texel centre."""
    out = np.zeros((6, R, R, 3))
    c = (np.arange(R) + 0.5) / R * 2 - 1
    tt, ss = np.meshgrid(c, c, indexing="ij")
    for f, (ma, msign, sa, ssign, ta, tsign) in enumerate(FACES):
        d = np.zeros((R, R, 3))
        d[..., ma] = msign
        d[..., sa] = ssign * ss
        d[..., ta] = tsign * tt
        out[f] = d / np.linalg.norm(d, axis=-1, keepdims=True)
    return out


def empty_scene():
    return {k: v[:0] for k, v in synth.make_plain_scene(seed=0, n=4).items()}


def ray_dirs(cam):
    W, H = cam["width"], cam["height"]
    ys, xs = np.mgrid[0:H, 0:W]
    dc = np.stack([(xs + 0.5 - cam["cx"]) / cam["fx"], (ys + 0.5 - cam["cy"]) / cam["fy"], np.ones((H, W))], -1)
    R = np.asarray(cam["viewmat"], np.float64)[:, :3]
    d = dc @ R  # R^T dc
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def test_constant_sky_closed_form():
    cam = synth.plain_camera(33, 25)
    sky = np.ones((6, 8, 8, 3)) * np.array([0.2, 0.4, 0.9])
    out = oracle.render(empty_scene(), cam, sky=sky)
    np.testing.assert_allclose(out["rgb"], np.broadcast_to([0.2, 0.4, 0.9], out["rgb"].shape), atol=1e-15)
    # one Gaussian on the axis: alpha c_g + (1 - alpha) c
    sc = dict(mu=np.zeros((1, 3)), vel=np.zeros((1, 3)), tau=np.full(1, 0.5), beta=np.ones(1), period=np.ones(1),
              scale=np.full((1, 3), 0.08), quat=np.array([[1.0, 0, 0, 0]]), opacity=np.array([0.7]),
              sh=((np.array([0.9, 0.1, 0.3]) - 0.5) / Y00).reshape(1, 1, 3))
    out = oracle.render(sc, cam, opts=dict(h=0.0), sky=sky)
    s_px = cam["fx"] * 0.08 / 4.0
    ys, xs = np.mgrid[0:25, 0:33]
    a = 0.7 * np.exp(-0.5 * ((xs + 0.5 - cam["cx"]) ** 2 + (ys + 0.5 - cam["cy"]) ** 2) / s_px ** 2)
    a = np.where(a < 1 / 255, 0.0, a)
    expect = a[..., None] * np.array([0.9, 0.1, 0.3]) + (1 - a[..., None]) * np.array([0.2, 0.4, 0.9])
    np.testing.assert_allclose(out["rgb"], expect, atol=1e-12)


@pytest.mark.parametrize("face", range(6))
def test_axis_directions_hit_their_face(face):
    sky = np.zeros((6, 4, 4, 3))
    for f in range(6):
        sky[f] = f
    ma, msign = FACES[face][0], FACES[face][1]
    target = np.zeros(3)
    target[ma] = msign
    up = np.array([0.0, 0.0, 1.0]) if ma != 2 else np.array([0.0, 1.0, 0.0])
    cam = synth.make_camera(synth.look_at((0, 0, 0), target, up), 9, 9, 9.0)
    out = oracle.render(empty_scene(), cam, sky=sky)
    assert out["rgb"][4, 4, 0] == pytest.approx(face, abs=1e-12)


def _face_coords(d):
    """max |face coordinate| of each direction (1 at a face edge)."""
    a = np.abs(d)
    ma = a.max(axis=-1, keepdims=True)
    return np.sort(a / ma, axis=-1)[..., 1]


def test_direction_map_returns_the_ray_direction():
    # bilinear filtering of a smooth map is second-order accurate inside a
    # face (a half-texel misplacement would show as a first-order error);
    # the last half texel at a face edge is clamped
    R = 64
    sky = texel_directions(R)
    rng = np.random.default_rng(0)
    for _ in range(6):
        target = rng.normal(size=3)
        cam = synth.make_camera(synth.look_at((0, 0, 0), target, (0.3, 0.2, 1.0)), 40, 30, 14.0)
        out = oracle.render(empty_scene(), cam, sky=sky)
        d = ray_dirs(cam)
        err = np.abs(out["rgb"] - d).max(axis=-1)
        inner = _face_coords(d) < 1.0 - 3.0 / R
        assert inner.sum() > 100
        assert err[inner].max() < 2e-3
        assert err.max() < 4.0 / R


def test_jitter_moves_the_sample():
    R = 32
    sky = texel_directions(R)
    cam = synth.make_camera(synth.look_at((0, 0, 0), (1, 0.2, 0.1), (0, 0, 1)), 20, 16, 10.0)
    jit = np.zeros((2, 16, 20))
    jit[0] = 0.5  # half a pixel to the right = the ray through the next half pixel
    a = oracle.render(empty_scene(), cam, sky=sky, sky_jitter=jit)
    cam2 = dict(cam)
    cam2["cx"] = cam["cx"] - 0.5
    b = oracle.render(empty_scene(), cam2, sky=sky)
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-12)


def _loss(sc, cam, sky, w):
    return float((oracle.render(sc, cam, sky=sky)["rgb"] * w).sum())


def test_sky_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    sc = {k: v.astype(np.float64) for k, v in synth.make_fd_scene(seed=2, n=40, sh_degree=1).items()}
    cam = synth.fd_camera(24, 18, t=0.5)
    sky = rng.uniform(0, 1, size=(6, 6, 6, 3))
    w = rng.normal(size=(18, 24, 3))
    g = oracle.render_bwd(sc, cam, w, np.zeros((18, 24)), np.zeros((18, 24)), sky=sky)
    used = np.argsort(-np.abs(g["sky"].reshape(-1)))[:12]
    for idx in used:
        flat = sky.reshape(-1)
        x0 = flat[idx]
        flat[idx] = x0 + 1e-6
        lp = _loss(sc, cam, sky, w)
        flat[idx] = x0 - 1e-6
        lm = _loss(sc, cam, sky, w)
        flat[idx] = x0
        assert g["sky"].reshape(-1)[idx] == pytest.approx((lp - lm) / 2e-6, rel=1e-6, abs=1e-9)
    # Gaussian parameters: their opacity also scales the sky term
    checked = 0
    for name in ("opacity", "mu", "scale"):
        flat = sc[name].reshape(-1)
        for idx in np.argsort(-np.abs(g[name].reshape(-1)))[:4]:
            x0 = flat[idx]
            h = 1e-6 * max(1.0, abs(x0))
            fd = []
            for step in (h, 0.5 * h):
                flat[idx] = x0 + step
                lp = _loss(sc, cam, sky, w)
                flat[idx] = x0 - step
                lm = _loss(sc, cam, sky, w)
                flat[idx] = x0
                fd.append((lp - lm) / (2 * step))
            if abs(fd[0] - fd[1]) > 1e-4 * max(1.0, abs(fd[0])):
                continue
            assert g[name].reshape(-1)[idx] == pytest.approx(fd[1], rel=2e-4, abs=2e-6), (name, idx)
            checked += 1
    assert checked >= 8

"""Pins of the oracle's compositing (Sec. 3.1, Eq. 3 and the depth and
opacity channels rendered beside colour) and of its reverse mode (Sec. 3.1 Eq. 4 / Sec. 3.2 Eq. 8:
the render function is differentiable).  No GPU.

* one isotropic Gaussian on the optical axis with h = 0: every pixel equals
  o~ exp(-r^2 / (2 sigma_px^2)) c + (1 - alpha) bg in closed form;
* two and three Gaussians composited by hand, including the depth order
  (not the index order) deciding who is in front, the index tie-break at
  equal depth, the alpha gate and the transmittance stop;
* O = 1 - T_final (telescoping of Eq. 3 with c = 1);
* the 3DGS special case (v = 0, beta -> inf, Sec. 3.2) renders the same at
  every t;
* brute force equals the culled mode;
* the analytic gradient equals FP64 central differences of the forward.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_18561_gb300 import synth

Y00 = 0.5 / math.sqrt(math.pi)


def _scene_of(mus, sigmas, opacities, rgbs, tau=0.5):
    n = len(mus)
    return dict(mu=np.asarray(mus, np.float64).reshape(n, 3), vel=np.zeros((n, 3)), tau=np.full(n, tau),
                beta=np.ones(n), period=np.ones(n),
                scale=np.repeat(np.asarray(sigmas, np.float64).reshape(n, 1), 3, axis=1),
                quat=np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), opacity=np.asarray(opacities, np.float64),
                sh=((np.asarray(rgbs, np.float64).reshape(n, 3) - 0.5) / Y00).reshape(n, 1, 3))


def _axis_cam(W=33, H=25, bg=(0.1, 0.2, 0.3)):
    cam = synth.plain_camera(width=W, height=H, bg=bg)
    return cam


def test_single_isotropic_gaussian_closed_form():
    W, H = 33, 25
    cam = _axis_cam(W, H)
    zc, sigma, o, rgb = 4.0, 0.08, 0.7, (0.9, 0.4, 0.2)
    sc = _scene_of([[0, 0, zc - 4.0]], [sigma], [o], [rgb])
    out = oracle.render(sc, cam, opts=dict(h=0.0))
    s_px = cam["fx"] * sigma / zc
    ys, xs = np.mgrid[0:H, 0:W]
    r2 = (xs + 0.5 - cam["cx"]) ** 2 + (ys + 0.5 - cam["cy"]) ** 2
    a = o * np.exp(-0.5 * r2 / s_px ** 2)
    a = np.where(a < 1 / 255, 0.0, np.minimum(a, 0.99))
    for c in range(3):
        np.testing.assert_allclose(out["rgb"][..., c], a * rgb[c] + (1 - a) * cam["bg"][c], atol=1e-12)
    np.testing.assert_allclose(out["depth"], a * zc, atol=1e-12)
    np.testing.assert_allclose(out["alpha"], a, atol=1e-12)
    np.testing.assert_allclose(out["T"], 1 - a, atol=1e-12)
    assert out["nblend"].max() == 1 and out["nblend"].sum() == np.count_nonzero(a)


def test_two_gaussians_depth_order_not_index_order():
    cam = _axis_cam(9, 9, bg=(0.0, 0.0, 0.0))
    # index 0 is behind index 1: the front one (index 1) is blended first
    back = ([0, 0, 1.0], 0.3, 0.6, (1.0, 0.0, 0.0))
    front = ([0, 0, -1.0], 0.3, 0.5, (0.0, 1.0, 0.0))
    sc = _scene_of([back[0], front[0]], [back[1], front[1]], [back[2], front[2]], [back[3], front[3]])
    out = oracle.render(sc, cam, opts=dict(h=0.0))
    cy, cx = 4, 4  # centre pixel (4.5, 4.5) is the principal point
    a_front, a_back = 0.5, 0.6
    expect = np.array([0.0, 1.0, 0.0]) * a_front + np.array([1.0, 0.0, 0.0]) * a_back * (1 - a_front)
    np.testing.assert_allclose(out["rgb"][cy, cx], expect, atol=1e-12)
    np.testing.assert_allclose(out["depth"][cy, cx], 3.0 * a_front + 5.0 * a_back * (1 - a_front), atol=1e-12)
    np.testing.assert_allclose(out["T"][cy, cx], (1 - a_front) * (1 - a_back), atol=1e-12)


def test_equal_depth_breaks_ties_by_index():
    cam = _axis_cam(9, 9, bg=(0.0, 0.0, 0.0))
    g0 = ([0, 0, 0.0], 0.3, 0.5, (1.0, 0.0, 0.0))
    g1 = ([0, 0, 0.0], 0.3, 0.8, (0.0, 0.0, 1.0))
    sc = _scene_of([g0[0], g1[0]], [g0[1], g1[1]], [g0[2], g1[2]], [g0[3], g1[3]])
    out = oracle.render(sc, cam, opts=dict(h=0.0))
    expect = np.array([1.0, 0.0, 0.0]) * 0.5 + np.array([0.0, 0.0, 1.0]) * 0.8 * 0.5
    np.testing.assert_allclose(out["rgb"][4, 4], expect, atol=1e-12)
    sc_sw = _scene_of([g1[0], g0[0]], [g1[1], g0[1]], [g1[2], g0[2]], [g1[3], g0[3]])
    out = oracle.render(sc_sw, cam, opts=dict(h=0.0))
    expect = np.array([0.0, 0.0, 1.0]) * 0.8 + np.array([1.0, 0.0, 0.0]) * 0.5 * 0.2
    np.testing.assert_allclose(out["rgb"][4, 4], expect, atol=1e-12)


def test_transmittance_stop_and_alpha_gate():
    cam = _axis_cam(9, 9, bg=(1.0, 1.0, 1.0))
    # five Gaussians at increasing depth with alpha 0.95 at the centre:
    # T = 1, 0.05, 0.0025, 1.25e-4, then 6.25e-6 < 1e-4 stops the 4th.  A
    # faint sixth one (alpha 0.1: T (1 - alpha) would stay above 1e-4) must
    # not be blended either: the stop ends the pixel, it is not a skip.
    zs = [-1.0, -0.5, 0.0, 0.5, 1.0, 1.2]
    cols = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1)]
    sc = _scene_of([[0, 0, z] for z in zs], [0.3] * 6, [0.95] * 5 + [0.1], cols)
    out = oracle.render(sc, cam, opts=dict(h=0.0))
    assert out["nblend"][4, 4] == 3
    T = [1.0, 0.05, 0.0025]
    expect = sum(np.array(cols[k], float) * 0.95 * T[k] for k in range(3)) + 0.0025 * 0.05 * np.ones(3)
    np.testing.assert_allclose(out["rgb"][4, 4], expect, atol=1e-12)
    np.testing.assert_allclose(out["T"][4, 4], 1.25e-4, rtol=1e-12)
    # a Gaussian whose alpha at the pixel is below 1/255 is skipped
    faint = _scene_of([[0, 0, -1.0], [0, 0, 0.0]], [0.3, 0.3], [0.9 / 255, 0.5], [(1, 0, 0), (0, 1, 0)])
    out = oracle.render(faint, cam, opts=dict(h=0.0))
    np.testing.assert_allclose(out["rgb"][4, 4], [0.5, 1.0, 0.5], atol=1e-12)
    assert out["nblend"][4, 4] == 1


def test_alpha_cap():
    cam = _axis_cam(9, 9, bg=(0.0, 0.0, 0.0))
    sc = _scene_of([[0, 0, 0.0]], [0.3], [1.0], [(1, 1, 1)])
    out = oracle.render(sc, cam, opts=dict(h=0.0))
    np.testing.assert_allclose(out["alpha"][4, 4], 0.99, atol=1e-15)


def test_opacity_channel_telescopes():
    sc = synth.make_plain_scene(seed=1, n=300)
    cam = synth.plain_camera(64, 48)
    out = oracle.render(sc, cam)
    np.testing.assert_allclose(out["alpha"], 1.0 - out["T"], atol=1e-12)


def test_static_special_case_renders_same_at_every_t():
    sc = synth.make_plain_scene(seed=2, n=300)
    sc = {k: v.astype(np.float64) for k, v in sc.items()}
    sc["vel"][:] = 0.0
    sc["beta"][:] = 1e9
    ref = oracle.render(sc, synth.plain_camera(48, 36, t=0.0))
    for t in (0.13, 0.5, 0.99, 7.0):
        out = oracle.render(sc, synth.plain_camera(48, 36, t=t))
        for k in ("rgb", "depth", "alpha"):
            np.testing.assert_allclose(out[k], ref[k], atol=1e-12)


def test_brute_equals_culled():
    sc = synth.make_plain_scene(seed=0, n=2000)
    cam = synth.plain_camera(80, 60)
    a = oracle.render(sc, cam, mode="brute")
    b = oracle.render(sc, cam, mode="culled")
    for k in ("rgb", "depth", "alpha", "T"):
        np.testing.assert_allclose(a[k], b[k], atol=1e-12)
    np.testing.assert_array_equal(a["nblend"], b["nblend"])


def test_pixel_list_matches_full_image():
    sc = synth.make_plain_scene(seed=0, n=500)
    cam = synth.plain_camera(40, 30)
    full = oracle.render(sc, cam)
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(0, 40, 50), rng.integers(0, 30, 50)], axis=1)
    part = oracle.render(sc, cam, mode="culled", pixels=pix)
    np.testing.assert_allclose(part["rgb"], full["rgb"][pix[:, 1], pix[:, 0]], atol=1e-12)


# --------------------------------------------------------------------------
# reverse mode vs finite differences
# --------------------------------------------------------------------------

def _loss(sc, cam, w_rgb, w_d, w_a, opts=None):
    out = oracle.render(sc, cam, opts=opts)
    return float((out["rgb"] * w_rgb).sum() + (out["depth"] * w_d).sum() + (out["alpha"] * w_a).sum())


@pytest.mark.parametrize("degree,dt", [(0, 0.0), (3, 0.0), (3, 0.04)])
def test_backward_matches_finite_differences(degree, dt):
    rng = np.random.default_rng(7 + degree)
    sc = synth.make_fd_scene(seed=degree, n=60, sh_degree=degree)
    sc = {k: v.astype(np.float64) for k, v in sc.items()}
    cam = synth.fd_camera(32, 24, t=0.45)
    cam["dt"] = dt  # dt != 0: the flow-translated state of Sec. 3.4
    cam["bg"] = np.array([0.2, 0.5, 0.8], np.float32)
    W, H = cam["width"], cam["height"]
    w_rgb = rng.normal(size=(H, W, 3))
    w_d = rng.normal(size=(H, W)) * 0.1
    w_a = rng.normal(size=(H, W))
    g = oracle.render_bwd(sc, cam, w_rgb, w_d, w_a)
    checked = 0
    for name in oracle.oracle.GRAD_NAMES:
        flat = sc[name].reshape(-1)
        gflat = g[name].reshape(-1)
        # sample entries with non-negligible gradient plus a few random ones
        cand = np.argsort(-np.abs(gflat))[:6].tolist() + rng.integers(0, flat.size, 3).tolist()
        for idx in cand:
            x0 = flat[idx]
            h = 1e-6 * max(1.0, abs(x0))
            fd = []
            for step in (h, 0.5 * h):
                flat[idx] = x0 + step
                lp = _loss(sc, cam, w_rgb, w_d, w_a)
                flat[idx] = x0 - step
                lm = _loss(sc, cam, w_rgb, w_d, w_a)
                flat[idx] = x0
                fd.append((lp - lm) / (2 * step))
            # a gate flip inside the stencil makes the two estimates disagree
            if abs(fd[0] - fd[1]) > 1e-4 * max(1.0, abs(fd[0])):
                continue
            assert gflat[idx] == pytest.approx(fd[1], rel=2e-4, abs=2e-5), (name, idx)
            checked += 1
    assert checked >= 60


def test_backward_on_a_pixel_list_equals_masked_full_image():
    """The pixel-list (culled) backward is the full-image backward with the
    upstream gradient zero outside the list."""
    rng = np.random.default_rng(11)
    sc = synth.make_fd_scene(seed=5, n=80, sh_degree=2)
    cam = synth.fd_camera(24, 20, t=0.3)
    H, W = cam["height"], cam["width"]
    pix = np.stack([rng.integers(0, W, 60), rng.integers(0, H, 60)], axis=1)
    pix = np.unique(pix, axis=0)
    w_rgb = rng.normal(size=(len(pix), 3))
    w_d = rng.normal(size=len(pix))
    w_a = rng.normal(size=len(pix))
    part = oracle.render_bwd(sc, cam, w_rgb, w_d, w_a, mode="culled", pixels=pix)
    full_rgb = np.zeros((H, W, 3))
    full_d = np.zeros((H, W))
    full_a = np.zeros((H, W))
    full_rgb[pix[:, 1], pix[:, 0]] = w_rgb
    full_d[pix[:, 1], pix[:, 0]] = w_d
    full_a[pix[:, 1], pix[:, 0]] = w_a
    full = oracle.render_bwd(sc, cam, full_rgb, full_d, full_a)
    for k in full:
        np.testing.assert_allclose(part[k], full[k], rtol=1e-10, atol=1e-12)

"""Pins of the oracle's frustum clamp inside the EWA Jacobian (no GPU).

The projected covariance of Sec. 3.1, Eq. 2 uses J, the Jacobian of the
perspective map at the Gaussian's camera-space mean.  Like the 3DGS
rasterizer the paper inherits, the oracle evaluates J not at the mean
itself when the mean lies far outside the view, but at the point of the
same depth whose x/z and y/z are clamped to +-1.3 x the half field of view
(1.3 W / (2 fx) horizontally, 1.3 H / (2 fy) vertically).  The projected
mean (u, v) is not clamped.

These tests fix that reading without restating the oracle's formula:

* J is taken here as the numerical Jacobian of the plain pinhole map
  (x, y, z) -> (fx x / z + cx, fy y / z + cy) evaluated at the clamped
  point, and Sigma comes from scipy's quaternion rotation, so a swapped
  limit (W with H, fx with fy), a wrong sign of the clamped ratio or a clamp
  applied to the projected mean fails;
* points just inside the limits are not clamped;
* the reverse mode through the clamped branch matches FP64 central
  differences on a scene where most Gaussians sit beyond the limits, on both
  axes and both sides, with footprints still reaching into the image.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2311_18561_gb300 import synth

CLAMP = 1.3


def _camera(W=160, H=120, fx=120.0, fy=150.0):
    # fx != fy and W != H, so that every mix-up of the four quantities in
    # the two limits changes a limit
    vm = synth.look_at((0.3, -0.2, -4.0), (0.0, 0.1, 0.0), (0.0, 1.0, 0.0))
    return synth.make_camera(vm, W, H, fx, fy=fy, cx=0.47 * W, cy=0.53 * H)


def _limits(cam):
    return CLAMP * 0.5 * cam["width"] / cam["fx"], CLAMP * 0.5 * cam["height"] / cam["fy"]


def _to_world(cam, P):
    # exact inverse of the (float32, so not exactly orthonormal) view matrix
    V = np.asarray(cam["viewmat"], np.float64)
    return np.linalg.solve(V[:, :3], (np.asarray(P, np.float64) - V[:, 3]).T).T


def _pinhole_cam(cam, P):
    P = np.asarray(P, np.float64)
    return np.array([cam["fx"] * P[0] / P[2] + cam["cx"], cam["fy"] * P[1] / P[2] + cam["cy"]])


def _numerical_J(cam, P, h=1e-6):
    J = np.zeros((2, 3))
    for c in range(3):
        e = np.zeros(3)
        e[c] = h * max(1.0, abs(P[c]))
        J[:, c] = (_pinhole_cam(cam, P + e) - _pinhole_cam(cam, P - e)) / (2 * e[c])
    return J


def _single(mu, scale, quat, opacity=0.8):
    return dict(mu=np.asarray([mu], np.float64), vel=np.zeros((1, 3)), tau=np.full(1, 0.5),
                beta=np.ones(1), period=np.ones(1), scale=np.asarray([scale], np.float64),
                quat=np.asarray([quat], np.float64), opacity=np.asarray([opacity], np.float64),
                sh=np.zeros((1, 1, 3)))


def _expected_cov2(cam, P_eval, q, s, h):
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    R = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: scalar last
    Sigma_world = R @ np.diag(np.asarray(s) ** 2) @ R.T
    Wr = np.asarray(cam["viewmat"], np.float64)[:, :3]
    Sigma_cam = Wr @ Sigma_world @ Wr.T
    J = _numerical_J(cam, P_eval)
    ref = J @ Sigma_cam @ J.T
    return np.array([ref[0, 0] + h, ref[0, 1], ref[1, 1] + h])


# ratios (x/z, y/z) in units of the two limits: both sides of each axis,
# both axes at once, and one axis clamped while the other is not
_RATIOS = [(1.6, 0.3), (-1.45, -0.2), (0.25, 1.7), (-0.4, -1.35), (1.5, -1.9), (-2.2, 1.25), (3.0, 0.0)]


@pytest.mark.parametrize("rx,ry", _RATIOS)
@pytest.mark.parametrize("h", [0.0, 0.3])
def test_clamped_covariance_is_the_jacobian_at_the_clamped_point(rx, ry, h):
    cam = _camera()
    limx, limy = _limits(cam)
    rng = np.random.default_rng(int(1000 * (rx + 3) + 10 * (ry + 3)))
    for _ in range(4):
        z = float(rng.uniform(2.0, 6.0))
        P = np.array([rx * limx * z, ry * limy * z, z])
        q = rng.normal(size=4)
        s = np.exp(rng.normal(-1.5, 0.5, 3))
        sc = _single(_to_world(cam, P), s, q)
        pp = oracle.preprocess(sc, cam, opts=dict(h=h))
        assert pp["valid"][0] == 1
        np.testing.assert_allclose(pp["pcam"][0], P, rtol=1e-12, atol=1e-12 * z)
        # the clamped point: same depth, ratios clamped to the limits
        Pc = np.array([np.clip(rx, -1, 1) * limx * z, np.clip(ry, -1, 1) * limy * z, z])
        want = _expected_cov2(cam, Pc, q, s, h)
        np.testing.assert_allclose(pp["cov2"][0], want, rtol=1e-6, atol=1e-9 * np.abs(want).max())
        # the unclamped Jacobian gives a different answer (the pin has teeth)
        if abs(rx) > 1 or abs(ry) > 1:
            other = _expected_cov2(cam, P, q, s, h)
            assert np.abs(other - want).max() > 1e-3 * np.abs(want).max()
        # the projected mean is the true projection, not the clamped one
        np.testing.assert_allclose(pp["uv"][0], _pinhole_cam(cam, P), rtol=1e-12)


def test_inside_the_limits_nothing_is_clamped():
    cam = _camera()
    limx, limy = _limits(cam)
    rng = np.random.default_rng(5)
    for rx, ry in [(0.999, 0.0), (-0.999, 0.5), (0.2, 0.999), (-0.7, -0.999), (0.99, -0.99)]:
        z = float(rng.uniform(2.0, 6.0))
        P = np.array([rx * limx * z, ry * limy * z, z])
        q = rng.normal(size=4)
        s = np.exp(rng.normal(-1.5, 0.5, 3))
        pp = oracle.preprocess(_single(_to_world(cam, P), s, q), cam, opts=dict(h=0.3))
        want = _expected_cov2(cam, P, q, s, 0.3)
        np.testing.assert_allclose(pp["cov2"][0], want, rtol=1e-6, atol=1e-9 * np.abs(want).max())


def test_clamp_factor_option_moves_the_limit():
    # with fov_clamp = 2 a point at 1.4 x the default limit (1.82 x the half
    # field of view) is no longer clamped
    cam = _camera()
    limx, limy = _limits(cam)
    z = 3.0
    P = np.array([1.4 * limx * z, -0.3 * limy * z, z])
    q, s = np.array([0.9, 0.1, -0.3, 0.2]), np.array([0.3, 0.1, 0.2])
    pp = oracle.preprocess(_single(_to_world(cam, P), s, q), cam, opts=dict(h=0.0, fov_clamp=2.0))
    want = _expected_cov2(cam, P, q, s, 0.0)
    np.testing.assert_allclose(pp["cov2"][0], want, rtol=1e-6, atol=1e-9 * np.abs(want).max())


# --------------------------------------------------------------------------
# reverse mode through the clamped branch
# --------------------------------------------------------------------------

def clamped_scene(cam, n=30, seed=0):
    """n Gaussians, about two thirds of them centred beyond the clamp limits
    (both axes, both sides) but large enough that their footprints reach
    into the image; the rest on screen.  Dynamic parameters are small, so
    the evaluated means stay on their side of the limits."""
    limx, limy = _limits(cam)
    rng = np.random.default_rng(seed)
    P = np.zeros((n, 3))
    n_off = (2 * n) // 3
    for i in range(n):
        z = rng.uniform(2.5, 4.0)
        if i < n_off:
            kind = i % 6
            a = rng.uniform(1.05, 1.3)
            b = rng.uniform(-0.6, 0.6)
            rx, ry = [(a, b), (-a, b), (b, a), (b, -a), (a, a), (-a, -a)][kind]
        else:
            rx, ry = rng.uniform(-0.6, 0.6, 2)
        P[i] = [rx * limx * z, ry * limy * z, z]
    mu = _to_world(cam, P)
    vel = rng.normal(0.0, 0.02, (n, 3))
    tau = rng.uniform(0.3, 0.7, n)
    period = rng.lognormal(0.0, 0.3, n)
    beta = rng.uniform(0.5, 2.0, n)
    scale = np.exp(rng.normal(-0.6, 0.2, (n, 3)))
    scale[n_off:] *= 0.3
    quat = rng.normal(size=(n, 4))
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(0.5, 0.7, n)))
    sh = rng.normal(0.0, 0.2, (n, 4, 3))
    sh[:, 0, :] = (rng.uniform(0.2, 0.8, (n, 3)) - 0.5) / (0.5 / math.sqrt(math.pi))
    return dict(mu=mu, vel=vel, tau=tau, beta=beta, period=period, scale=scale, quat=quat,
                opacity=opacity, sh=sh), n_off


def _fd_camera():
    vm = synth.look_at((0.0, 0.0, -3.5), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    return synth.make_camera(vm, 40, 30, 28.0, fy=32.0, t=0.45, bg=(0.2, 0.5, 0.8))


def _loss(sc, cam, w_rgb, w_d, w_a):
    out = oracle.render(sc, cam)
    return float((out["rgb"] * w_rgb).sum() + (out["depth"] * w_d).sum() + (out["alpha"] * w_a).sum())


def test_clamped_scene_is_mostly_clamped_and_visible():
    cam = _fd_camera()
    sc, n_off = clamped_scene(cam)
    limx, limy = _limits(cam)
    pp = oracle.preprocess(sc, cam)
    r = pp["pcam"][:, :2] / pp["pcam"][:, 2:3]
    clamped = (np.abs(r[:, 0]) > limx) | (np.abs(r[:, 1]) > limy)
    assert clamped.sum() == n_off and clamped[:n_off].all()
    for sx in (1, -1):
        assert np.any(sx * r[:n_off, 0] > limx) and np.any(sx * r[:n_off, 1] > limy)
    # every clamped Gaussian blends into at least one pixel
    w = np.ones((cam["height"], cam["width"]))
    g = oracle.render_bwd(sc, cam, np.zeros(w.shape + (3,)), np.zeros_like(w), w)
    assert np.all(np.abs(g["opacity"][:n_off]) > 0)


def test_backward_through_the_clamp_matches_finite_differences():
    cam = _fd_camera()
    sc, n_off = clamped_scene(cam)
    W, H = cam["width"], cam["height"]
    rng = np.random.default_rng(17)
    w_rgb = rng.normal(size=(H, W, 3))
    w_d = rng.normal(size=(H, W)) * 0.1
    w_a = rng.normal(size=(H, W))
    g = oracle.render_bwd(sc, cam, w_rgb, w_d, w_a)
    checked = 0
    per_group = {}
    for name in ("mu", "vel", "tau", "beta", "period", "scale", "quat", "opacity", "sh"):
        arr, garr = sc[name], g[name]
        rows = arr.reshape(arr.shape[0], -1)
        grows = garr.reshape(garr.shape[0], -1)
        # the clamped Gaussians' entries with the largest gradients
        cand = []
        for i in range(n_off):
            j = int(np.argmax(np.abs(grows[i])))
            cand.append((abs(grows[i, j]), i, j))
        cand.sort(reverse=True)
        for _, i, j in cand[:8]:
            x0 = rows[i, j]
            h = 1e-6 * max(1.0, abs(x0))
            fd = []
            for step in (h, 0.5 * h):
                rows[i, j] = x0 + step
                lp = _loss(sc, cam, w_rgb, w_d, w_a)
                rows[i, j] = x0 - step
                lm = _loss(sc, cam, w_rgb, w_d, w_a)
                rows[i, j] = x0
                fd.append((lp - lm) / (2 * step))
            if abs(fd[0] - fd[1]) > 1e-4 * max(1.0, abs(fd[0])):
                continue  # a gate flips inside the stencil
            assert grows[i, j] == pytest.approx(fd[1], rel=2e-4, abs=2e-5), (name, i, j)
            checked += 1
            per_group[name] = per_group.get(name, 0) + 1
    assert checked >= 50, per_group
    assert all(per_group.get(k, 0) >= 3 for k in ("mu", "scale", "quat", "opacity")), per_group


def test_mean_depth_gradient_through_the_clamp():
    """In the clamped branch J depends on the mean only through its depth:
    moving the mean along x (in camera space) changes the covariance only
    through the unclamped axis.  The camera-space gradient of the loss wrt
    the mean's x from the oracle must match central differences taken in
    camera space (a check of the branch's partial derivatives on their own,
    with the colour direction held by a degree-0 colour)."""
    cam = _fd_camera()
    sc, n_off = clamped_scene(cam, n=12, seed=3)
    sc["sh"] = sc["sh"][:, :1, :].copy()
    sc["vel"][:] = 0.0
    W, H = cam["width"], cam["height"]
    rng = np.random.default_rng(4)
    w_rgb = rng.normal(size=(H, W, 3))
    w_d = np.zeros((H, W))
    w_a = rng.normal(size=(H, W))
    g = oracle.render_bwd(sc, cam, w_rgb, w_d, w_a)
    Wr = np.asarray(cam["viewmat"], np.float64)[:, :3]
    checked = 0
    for i in range(n_off):
        gcam = Wr @ g["mu"][i]  # d loss / d (camera-space mean)
        for c in range(3):
            e = Wr[c] * 1e-6  # a camera-axis step expressed in world coordinates
            x0 = sc["mu"][i].copy()
            sc["mu"][i] = x0 + e
            lp = _loss(sc, cam, w_rgb, w_d, w_a)
            sc["mu"][i] = x0 - e
            lm = _loss(sc, cam, w_rgb, w_d, w_a)
            sc["mu"][i] = x0
            fd = (lp - lm) / 2e-6
            if abs(gcam[c]) < 1e-6 and abs(fd) < 1e-6:
                continue
            assert gcam[c] == pytest.approx(fd, rel=5e-4, abs=5e-5), (i, c)
            checked += 1
    assert checked >= 15

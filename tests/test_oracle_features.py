"""Pins of the oracle's extra composited channels: the average-velocity map
(v_bar = v exp(-rho/2), Eq. 10), the staticness map (rho = beta / l clamped
to [0, 2], dynamic-element analysis of Sec. 4) and semantic rendering (a
per-Gaussian class vector composited like colour).  No GPU.

* constant rho (or v and rho) across the scene: the map is that constant
  times the opacity map O (closed form: sum T a x = x sum T a);
* semantics equal to each Gaussian's (view-independent) colour reproduce
  the colour image minus its background T bg, so the feature weights are
  the colour weights; one-hot semantics sum to O;
* brute force and culled compositing agree; turning features on leaves the
  other channels untouched;
* the reverse mode matches FP64 finite differences for the semantic
  vectors, v, beta, l and the geometry.
"""
import numpy as np
import pytest

import oracle
from paper_2311_18561_gb300 import synth

Y00 = 0.5 / np.sqrt(np.pi)
VBAR, RHO, SEM = oracle.FEAT_VBAR, oracle.FEAT_RHO, oracle.FEAT_SEM


def f64(scene):
    return {k: np.asarray(v, np.float64).copy() for k, v in scene.items()}


@pytest.mark.parametrize("rho0", [0.7, 3.1])
def test_rho_map_is_clamped_rho_times_opacity(rho0):
    sc = f64(synth.make_fd_scene(seed=4, n=300, sh_degree=1))
    sc["beta"] = rho0 * sc["period"]
    cam = synth.fd_camera(40, 30, t=0.3)
    out = oracle.render(sc, cam, features=RHO)
    assert out["alpha"].max() > 0.5
    np.testing.assert_allclose(out["feat"][..., 0], min(rho0, 2.0) * out["alpha"], rtol=0, atol=1e-13)


@pytest.mark.parametrize("rho0", [0.5, 1e-9])
def test_vbar_map_of_a_shared_velocity(rho0):
    sc = f64(synth.make_fd_scene(seed=5, n=300, sh_degree=0))
    v0 = np.array([0.3, -0.2, 0.5])
    sc["vel"][:] = v0
    sc["beta"] = rho0 * sc["period"]
    cam = synth.fd_camera(40, 30, t=0.6)
    out = oracle.render(sc, cam, features=VBAR | RHO)
    expect = np.exp(-0.5 * rho0) * v0[None, None, :] * out["alpha"][..., None]
    np.testing.assert_allclose(out["feat"][..., :3], expect, rtol=0, atol=1e-13)
    if rho0 < 1e-6:  # rho -> 0: v_bar -> v
        np.testing.assert_allclose(out["feat"][..., :3], v0 * out["alpha"][..., None], atol=1e-8)
    np.testing.assert_allclose(out["feat"][..., 3], rho0 * out["alpha"], atol=1e-13)


def test_semantics_equal_to_colour_reproduce_the_colour_weights():
    sc = f64(synth.make_fd_scene(seed=6, n=300, sh_degree=0))
    colour = Y00 * sc["sh"][:, 0, :] + 0.5  # degree 0: view-independent, in (0.2, 0.8)
    assert colour.min() > 0
    cam = synth.fd_camera(40, 30, t=0.45)
    cam["bg"] = np.array([0.3, 0.1, 0.6])
    out = oracle.render(sc, cam, features=SEM, sem=colour)
    expect = out["rgb"] - out["T"][..., None] * cam["bg"]
    np.testing.assert_allclose(out["feat"], expect, rtol=0, atol=1e-13)


def test_one_hot_semantics_sum_to_opacity():
    sc = f64(synth.make_fd_scene(seed=7, n=300, sh_degree=0))
    sem = synth.make_semantics(300, 19, one_hot=True)
    cam = synth.fd_camera(40, 30, t=0.5)
    out = oracle.render(sc, cam, features=VBAR | RHO | SEM, sem=sem)
    assert out["feat"].shape == (30, 40, 3 + 1 + 19)
    np.testing.assert_allclose(out["feat"][..., 4:].sum(-1), out["alpha"], atol=1e-13)
    assert (out["feat"][..., 4:] >= 0).all()


def test_features_leave_other_channels_and_culling_agrees():
    sc = f64(synth.make_fd_scene(seed=8, n=400, sh_degree=2))
    sem = synth.make_semantics(400, 5)
    cam = synth.fd_camera(48, 36, t=0.7)
    plain = oracle.render(sc, cam)
    a = oracle.render(sc, cam, features=VBAR | RHO | SEM, sem=sem)
    b = oracle.render(sc, cam, features=VBAR | RHO | SEM, sem=sem, mode="culled")
    for k in ("rgb", "depth", "alpha", "T"):
        np.testing.assert_array_equal(plain[k], a[k])
    np.testing.assert_allclose(a["feat"], b["feat"], atol=1e-13)


def _loss(sc, cam, sem, w_rgb, w_f, mask):
    out = oracle.render(sc, cam, features=mask, sem=sem)
    return float((out["rgb"] * w_rgb).sum() + (out["feat"] * w_f).sum())


def test_feature_backward_matches_finite_differences():
    rng = np.random.default_rng(11)
    n, S = 60, 4
    sc = f64(synth.make_fd_scene(seed=9, n=n, sh_degree=1))
    sem = np.asarray(synth.make_semantics(n, S), np.float64)
    cam = synth.fd_camera(24, 18, t=0.5)
    mask = VBAR | RHO | SEM
    F = oracle.feat_count(mask, S)
    w_rgb = rng.normal(size=(18, 24, 3))
    w_f = rng.normal(size=(18, 24, F))
    g = oracle.render_bwd(sc, cam, w_rgb, np.zeros((18, 24)), np.zeros((18, 24)), features=mask, sem=sem,
                          dL_feat=w_f)
    # semantic vectors enter linearly: central differences are exact up to rounding
    for idx in np.argsort(-np.abs(g["sem"].reshape(-1)))[:8]:
        flat = sem.reshape(-1)
        x0 = flat[idx]
        flat[idx] = x0 + 1e-6
        lp = _loss(sc, cam, sem, w_rgb, w_f, mask)
        flat[idx] = x0 - 1e-6
        lm = _loss(sc, cam, sem, w_rgb, w_f, mask)
        flat[idx] = x0
        assert g["sem"].reshape(-1)[idx] == pytest.approx((lp - lm) / 2e-6, rel=1e-6, abs=1e-9)
    checked = {}
    for name in ("vel", "beta", "period", "opacity", "mu", "scale"):
        flat = sc[name].reshape(-1)
        for idx in np.argsort(-np.abs(g[name].reshape(-1)))[:4]:
            x0 = flat[idx]
            h = 1e-6 * max(1.0, abs(x0))
            fd = []
            for step in (h, 0.5 * h):
                flat[idx] = x0 + step
                lp = _loss(sc, cam, sem, w_rgb, w_f, mask)
                flat[idx] = x0 - step
                lm = _loss(sc, cam, sem, w_rgb, w_f, mask)
                flat[idx] = x0
                fd.append((lp - lm) / (2 * step))
            if abs(fd[0] - fd[1]) > 1e-4 * max(1.0, abs(fd[0])):
                continue  # a gate or the rho clamp lies within the step
            assert g[name].reshape(-1)[idx] == pytest.approx(fd[1], rel=2e-4, abs=2e-6), (name, idx)
            checked[name] = checked.get(name, 0) + 1
    assert sum(checked.values()) >= 16 and len(checked) >= 5, checked


def test_feature_gradient_alone_is_the_feature_adjoint():
    # with dL_rgb = 0 the gradient of v, beta, l comes only through the
    # feature channels; with the features off it is exactly zero
    n = 50
    sc = f64(synth.make_fd_scene(seed=12, n=n, sh_degree=0))
    cam = synth.fd_camera(24, 18, t=0.5)
    z = np.zeros((18, 24))
    w_f = np.random.default_rng(1).normal(size=(18, 24, 4))
    g = oracle.render_bwd(sc, cam, np.zeros((18, 24, 3)), z, z, features=VBAR | RHO, dL_feat=w_f)
    g0 = oracle.render_bwd(sc, cam, np.zeros((18, 24, 3)), z, z)
    assert np.abs(g["vel"]).max() > 0 and np.abs(g["beta"]).max() > 0
    for k in g0:
        assert np.abs(g0[k]).max() == 0.0

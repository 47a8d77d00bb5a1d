"""Tile binning by the footprint ellipse on footprints that take its less
common paths: Gaussians taller than 8 tile rows (their tiles found by the
warp-cooperative row search from the stored ellipse, not a row table) and
needles whose conic is too ill-conditioned for the ellipse test (whole
rectangle rows kept).  Lists checked against the oracle's rectangle lists
and blended tiles, images against the FP64 oracle, bit-identical across
tile shapes, and the backward pass against the oracle.  GPU only.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18561_gb300 import render as R
from paper_2311_18561_gb300 import synth

from .gpu_util import check_tile_lists, compare_to_oracle, gpu_render, to_numpy_images

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

W, H = 320, 240


def tall_and_needle_scene(seed=21):
    """The plain scene with 30 large elongated Gaussians (tens of pixels
    along one axis) and 12 needles (one axis 1000x the others)."""
    scene = synth.make_plain_scene(seed=seed, n=600)
    rng = np.random.default_rng(seed + 1)
    big = rng.choice(600, 42, replace=False)
    tall, needle = big[:30], big[30:]
    scene["scale"][tall] = np.stack([rng.uniform(0.02, 0.05, 30), rng.uniform(0.3, 0.6, 30),
                                     rng.uniform(0.02, 0.05, 30)], axis=1).astype(np.float32)
    scene["scale"][needle] = np.stack([np.full(12, 1.0), np.full(12, 1e-3), np.full(12, 1e-3)],
                                      axis=1).astype(np.float32)
    scene["opacity"][big] = rng.uniform(0.5, 0.95, 42).astype(np.float32)
    scene["mu"][big, 2] = rng.uniform(-0.5, 0.5, 42).astype(np.float32)
    return scene


def camera():
    return synth.plain_camera(width=W, height=H, t=0.5, bg=(0.1, 0.2, 0.3))


def test_scene_takes_the_rare_paths():
    """Not a GPU check: the scene has visible Gaussians spanning more than
    8 rows of 8-pixel tiles and visible needles ((a + c)^2 > 1e4 (ac - b^2))."""
    pp = oracle.preprocess(tall_and_needle_scene(), camera())
    ok = pp["valid"] != 0
    a, b, c = pp["conic"][ok].T
    assert np.sum((a + c) ** 2 > 1e4 * (a * c - b * b)) >= 3
    ry = pp["box"][ok][:, 1]
    assert np.sum(2 * ry > 9 * 8) >= 10


@pytest.mark.parametrize("cfg", [(8, 8, 1), (16, 8, 2), (32, 32, 4)])
def test_lists_and_images(cfg):
    scene = tall_and_needle_scene()
    cam = camera()
    r = R.Renderer(tile=cfg[:2], pixels_per_thread=cfg[2])
    fr = R.Frame()
    out = gpu_render(r, R.scene_to_device(scene), [cam], frame=fr)[0]
    tx, ty = R.tiles_of(cam, cfg[:2])
    ex = fr.export(tx * ty)
    rect = ex["rect"]
    if cfg[1] == 8:
        assert np.sum(rect[:, 3] - rect[:, 1] > 8) >= 10  # the warp-cooperative rows
    kept, full = check_tile_lists(ex, scene, cam, cfg[:2], tx, ty)
    assert kept < full
    compare_to_oracle(to_numpy_images(out), oracle.render(scene, cam))
    r.close()
    fr.close()


def test_images_identical_across_tile_shapes():
    scene = tall_and_needle_scene()
    st = R.scene_to_device(scene)
    ref = None
    for (tw, th, px) in [(8, 8, 1), (16, 16, 1), (16, 8, 2), (32, 16, 4), (16, 32, 4)]:
        r = R.Renderer(tile=(tw, th), pixels_per_thread=px)
        out = gpu_render(r, st, [camera()])[0]
        cur = [out[k].cpu().numpy() for k in ("rgb", "depth", "alpha")]
        if ref is None:
            ref = cur
        else:
            for x, y in zip(ref, cur):
                np.testing.assert_array_equal(x, y, err_msg=str((tw, th, px)))
        r.close()


def test_backward_matches_oracle():
    scene = tall_and_needle_scene()
    cam = camera()
    rng = np.random.default_rng(3)
    w_rgb = rng.normal(size=(3, H, W))
    r = R.Renderer(tile=(8, 8), pixels_per_thread=1)
    fr = R.Frame()
    st = R.scene_to_device(scene)
    r.forward(st, [cam], frame=fr)
    grads = r.backward(st, [cam], fr, [dict(rgb=torch.tensor(w_rgb, dtype=torch.float32, device="cuda"))])
    torch.cuda.synchronize()
    ref = oracle.render_bwd(scene, cam, np.transpose(w_rgb, (1, 2, 0)), np.zeros((H, W)), np.zeros((H, W)))
    for k in R.PARAM_NAMES:
        g = grads[k].detach().cpu().numpy().astype(np.float64).reshape(-1)
        rr = ref[k].reshape(-1)
        nr = np.linalg.norm(rr)
        assert nr > 0, k
        assert np.linalg.norm(g - rr) / nr <= 1e-2, k


def _strip_scene(axis, seed=31):
    """2,000 Gaussians in a thin slab around the image's long axis (world
    axis `axis` spans it), a few of them huge (footprints wider than 255
    tiles of 8 pixels: no row table)."""
    scene = synth.make_plain_scene(seed=seed, n=2000)
    rng = np.random.default_rng(seed)
    other = 1 - axis
    scene["mu"][:, other] = rng.uniform(-0.002, 0.002, 2000).astype(np.float32)
    scene["vel"][:, other] = 0.0
    scene["scale"][:8] = rng.uniform(1.5, 3.0, size=(8, 3)).astype(np.float32)
    scene["opacity"][:8] = 0.2
    return scene


@pytest.mark.parametrize("shape", [(16384, 24), (24, 16384)])
def test_maximum_image_size(shape):
    """The largest accepted image side (16384 pixels) renders like the
    oracle at sampled pixels, with 8x8 tiles (2048 tiles along the long
    side); one pixel more is rejected."""
    W, H = shape
    scene = _strip_scene(0 if W > H else 1)
    vm = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0))
    cam = synth.make_camera(vm, W, H, 4000.0, t=0.5, bg=(0.05, 0.1, 0.15))
    r = R.Renderer(tile=(8, 8), pixels_per_thread=1)
    fr = R.Frame()
    out = gpu_render(r, R.scene_to_device(scene), [cam], frame=fr)[0]
    tx, ty = R.tiles_of(cam, (8, 8))
    rect = fr.export(tx * ty)["rect"]
    assert np.any(rect[:, 2] - rect[:, 0] > 255) or np.any(rect[:, 3] - rect[:, 1] > 255)
    rng = np.random.default_rng(1)
    long_ = max(W, H)
    a = np.concatenate([rng.integers(0, long_, 600), rng.integers(long_ // 2 - 1500, long_ // 2 + 1500, 600)])
    b = rng.integers(0, min(W, H), a.size)
    pix = np.stack([a, b], 1) if W > H else np.stack([b, a], 1)
    ref = oracle.render(scene, cam, mode="culled", pixels=pix)
    img = to_numpy_images(out)
    got = {k: img[k][pix[:, 1], pix[:, 0]] for k in ("rgb", "depth", "alpha")}
    compare_to_oracle(got, ref, pixels=pix)
    assert float(img["alpha"].max()) > 0.5  # the strip is not empty
    r.close()
    fr.close()
    too_big = synth.make_camera(vm, W + (W > H), H + (H > W), 4000.0)
    r2 = R.Renderer()
    with pytest.raises(Exception):
        r2.forward(R.scene_to_device(scene), [too_big])
    r2.close()

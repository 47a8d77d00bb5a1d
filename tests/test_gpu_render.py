"""Parity of the CUDA forward path (stages a-c) with the FP64 oracle,
through the C ABI.  GPU only."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import binning
from paper_2311_18561_gb300 import render as R
from paper_2311_18561_gb300 import synth

from .gpu_util import DENSE_TIE_FLAG_FRAC, check_tile_lists, compare_to_oracle, gpu_render, to_numpy_images
from .test_oracle_clamp import _camera as clamp_camera
from .test_oracle_clamp import _limits as clamp_limits
from .test_oracle_clamp import clamped_scene

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

# every supported (tile width, tile height, pixels per thread)
CONFIGS = [(16, 16, 1), (16, 16, 2), (16, 16, 4), (8, 8, 1), (8, 8, 2), (16, 8, 1), (16, 8, 2), (32, 8, 1),
           (32, 16, 1), (32, 16, 2), (32, 16, 4), (32, 32, 4), (16, 32, 4)]


@pytest.fixture(scope="module")
def renderer():
    return R.Renderer()


def test_plain_config_image_parity(renderer):
    """2,000 Gaussians, 160x120, t = 0.5, 16x16 tiles (the plain config)."""
    scene = synth.make_plain_scene(seed=0, n=2000)
    cam = synth.plain_camera()
    out = gpu_render(renderer, R.scene_to_device(scene), [cam])[0]
    ref = oracle.render(scene, cam, mode="brute")
    rep = compare_to_oracle(to_numpy_images(out), ref)
    assert rep["max_rgb"] < 1e-3


@pytest.mark.parametrize("t", [0.0, 0.31, 0.77])
@pytest.mark.parametrize("size", [(37, 23), (161, 121), (1, 1), (16, 16)])
def test_ragged_sizes_and_times(renderer, t, size):
    scene = synth.make_plain_scene(seed=3, n=1500)
    W, H = size
    cam = synth.plain_camera(width=W, height=H, t=t, bg=(0.2, 0.4, 0.6))
    out = gpu_render(renderer, R.scene_to_device(scene), [cam])[0]
    ref = oracle.render(scene, cam)
    compare_to_oracle(to_numpy_images(out), ref, max_flag_frac=1.0 if W * H < 100 else DENSE_TIE_FLAG_FRAC)


def test_sh3_dynamic_scene_parity(renderer):
    scene = synth.make_fd_scene(seed=1, n=800, sh_degree=3)
    cam = synth.fd_camera(96, 72, t=0.37)
    out = gpu_render(renderer, R.scene_to_device(scene), [cam])[0]
    compare_to_oracle(to_numpy_images(out), oracle.render(scene, cam))


@pytest.mark.parametrize("deg", [1, 2])
def test_sh_degrees_1_2(renderer, deg):
    scene = synth.make_fd_scene(seed=2, n=600, sh_degree=deg)
    cam = synth.fd_camera(64, 48, t=0.6)
    out = gpu_render(renderer, R.scene_to_device(scene), [cam])[0]
    compare_to_oracle(to_numpy_images(out), oracle.render(scene, cam))


def test_tile_shape_invariance_bit_exact():
    """The per-pixel work does not depend on the tile shape or on how many
    pixels a thread handles: images are bit-identical for every supported
    configuration."""
    scene = synth.make_plain_scene(seed=4, n=3000)
    cam = synth.plain_camera(width=203, height=141, t=0.42)
    st = R.scene_to_device(scene)
    ref = None
    for (tw, th, px) in CONFIGS:
        r = R.Renderer(tile=(tw, th), pixels_per_thread=px)
        out = gpu_render(r, st, [cam])[0]
        cur = [out[k].cpu().numpy() for k in ("rgb", "depth", "alpha")]
        if ref is None:
            ref = cur
        else:
            for a, b in zip(ref, cur):
                np.testing.assert_array_equal(a, b, err_msg=str((tw, th, px)))
        r.close()


@pytest.mark.parametrize("cfg", [(16, 16, 4), (32, 32, 4), (8, 8, 2)])
def test_multi_pixel_configs_match_oracle(cfg):
    scene = synth.make_fd_scene(seed=12, n=900, sh_degree=3)
    cam = synth.fd_camera(77, 53, t=0.55)
    r = R.Renderer(tile=cfg[:2], pixels_per_thread=cfg[2])
    out = gpu_render(r, R.scene_to_device(scene), [cam])[0]
    compare_to_oracle(to_numpy_images(out), oracle.render(scene, cam), max_flag_frac=DENSE_TIE_FLAG_FRAC)
    r.close()


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16), (32, 32)])
def test_depth_order_tile_lists_and_ranges_bit_exact(tile):
    scene = synth.make_plain_scene(seed=5, n=2000)
    # duplicate some positions so that exact depth ties occur
    scene["mu"][1000:1100] = scene["mu"][:100]
    scene["vel"][1000:1100] = scene["vel"][:100]
    scene["tau"][1000:1100] = scene["tau"][:100]
    scene["period"][1000:1100] = scene["period"][:100]
    cam = synth.plain_camera(width=150, height=110, t=0.5)
    r = R.Renderer(tile=tile, pixels_per_thread=4 if tile == (32, 32) else 1)
    fr = R.Frame()
    gpu_render(r, R.scene_to_device(scene), [cam], frame=fr)
    tx, ty = R.tiles_of(cam, tile)
    ex = fr.export(tx * ty)
    gid, zk, rect = ex["sorted_gid"], ex["depth_key"], ex["rect"]
    z = zk.view(np.float32)
    assert np.all(z > 0)
    # depth order: the GPU's order equals (z bits, gid) order of its own keys
    np.testing.assert_array_equal(binning.depth_order(np.sort(gid), z[np.argsort(gid)]), gid)
    kept, full = check_tile_lists(ex, scene, cam, tile, tx, ty)
    assert kept < full  # the ellipse test leaves tiles out
    r.close()
    fr.close()


def test_records_match_oracle_preprocess():
    scene = synth.make_fd_scene(seed=6, n=500, sh_degree=3)
    cam = synth.fd_camera(64, 48, t=0.3)
    r = R.Renderer()
    fr = R.Frame()
    gpu_render(r, R.scene_to_device(scene), [cam], frame=fr)
    tx, ty = R.tiles_of(cam)
    ex = fr.export(tx * ty)
    pp = oracle.preprocess(scene, cam)
    gid = ex["sorted_gid"].astype(np.int64)
    assert np.all(pp["valid"][gid] == 1)
    rec = ex["records"]
    np.testing.assert_allclose(rec[:, 0:2], pp["uv"][gid], rtol=1e-5, atol=1e-3)
    conic = pp["conic"][gid]
    scale = np.abs(conic).max(axis=1, keepdims=True)
    np.testing.assert_allclose(rec[:, 2:4] / scale, conic[:, 0:2] / scale, atol=1e-4)
    np.testing.assert_allclose(rec[:, 4] / scale[:, 0], conic[:, 2] / scale[:, 0], atol=1e-4)
    np.testing.assert_allclose(rec[:, 5], pp["ot"][gid], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(rec[:, 6], pp["pcam"][gid, 2], rtol=1e-6)
    np.testing.assert_allclose(rec[:, 8:11], pp["rgb"][gid], atol=1e-5)
    r.close()
    fr.close()


def test_multi_view_call_equals_single_views(renderer):
    scene = synth.make_plain_scene(seed=7, n=2500)
    st = R.scene_to_device(scene)
    cams = [synth.plain_camera(width=90, height=70, t=0.2), synth.plain_camera(width=160, height=120, t=0.9),
            synth.plain_camera(width=33, height=17, t=0.5, bg=(1, 0, 0))]
    many = gpu_render(renderer, st, cams)
    for k, cam in enumerate(cams):
        one = gpu_render(renderer, st, [cam])[0]
        for key in ("rgb", "depth", "alpha"):
            assert torch.equal(many[k][key], one[key]), (k, key)


def test_empty_scene_and_all_culled(renderer):
    cam = synth.plain_camera(width=40, height=30, bg=(0.25, 0.5, 0.75))
    empty = {k: v[:0] for k, v in synth.make_plain_scene(seed=0, n=4).items()}
    out = gpu_render(renderer, R.scene_to_device(empty), [cam])[0]
    for c, b in enumerate((0.25, 0.5, 0.75)):
        assert torch.all(out["rgb"][c] == b)
    assert torch.all(out["alpha"] == 0) and torch.all(out["depth"] == 0)
    scene = synth.make_plain_scene(seed=0, n=500)
    away = synth.make_camera(synth.look_at((0, 0, -4), (0, 0, -8), (0, 1, 0)), 40, 30,
                             synth.focal_from_hfov(40, 60), bg=(0.25, 0.5, 0.75))
    out = gpu_render(renderer, R.scene_to_device(scene), [away])[0]
    assert torch.all(out["alpha"] == 0)


def test_nan_parameters_are_culled(renderer):
    scene = synth.make_plain_scene(seed=8, n=1000)
    scene["mu"][10] = np.nan
    scene["scale"][20] = np.nan
    scene["quat"][30] = 0.0
    cam = synth.plain_camera(width=64, height=48)
    out = gpu_render(renderer, R.scene_to_device(scene), [cam])[0]
    assert all(torch.isfinite(out[k]).all() for k in ("rgb", "depth", "alpha"))
    keep = np.setdiff1d(np.arange(1000), [10, 20, 30])
    ref = oracle.render(synth.subset(scene, keep), cam)
    compare_to_oracle(to_numpy_images(out), ref, max_flag_frac=DENSE_TIE_FLAG_FRAC)


def test_huge_gaussian_covering_everything(renderer):
    scene = synth.make_plain_scene(seed=9, n=300)
    scene["scale"][0] = [3.0, 3.0, 3.0]
    scene["opacity"][0] = 0.3
    cam = synth.plain_camera(width=96, height=80)
    out = gpu_render(renderer, R.scene_to_device(scene), [cam])[0]
    compare_to_oracle(to_numpy_images(out), oracle.render(scene, cam))


def test_static_special_case_matches_every_t(renderer):
    scene = synth.make_plain_scene(seed=10, n=1500)
    scene["vel"][:] = 0.0
    scene["beta"][:] = 1e9
    st = R.scene_to_device(scene)
    ref = gpu_render(renderer, st, [synth.plain_camera(t=0.0)])[0]
    for t in (0.25, 0.5, 0.99):
        out = gpu_render(renderer, st, [synth.plain_camera(t=t)])[0]
        for k in ("rgb", "depth", "alpha"):
            torch.testing.assert_close(out[k], ref[k], rtol=0, atol=1e-6)


def test_no_sync_mode_matches_and_reports_overflow():
    scene = synth.make_plain_scene(seed=11, n=2000)
    cam = synth.plain_camera()
    st = R.scene_to_device(scene)
    a = gpu_render(R.Renderer(), st, [cam])[0]
    r = R.Renderer(sync_sizes=False, pair_capacity=1 << 20)
    fr = R.Frame()
    b = gpu_render(r, st, [cam], frame=fr)[0]
    assert fr.stats()[2] == 0
    for k in ("rgb", "depth", "alpha"):
        assert torch.equal(a[k], b[k])
    small = R.Renderer(sync_sizes=False, pair_capacity=64)
    fr2 = R.Frame()
    gpu_render(small, st, [cam], frame=fr2)
    m, k, ov = fr2.stats()
    assert ov == 1 and k > 64


@pytest.mark.parametrize("dt", [0.03, -0.05])
def test_flow_translated_state_matches_oracle(renderer, dt):
    """Temporal smoothing (Sec. 3.4): rendering the flow-translated state."""
    scene = synth.make_fd_scene(seed=13, n=900, sh_degree=3)
    cam = synth.fd_camera(80, 60, t=0.4)
    cam["dt"] = dt
    out = gpu_render(renderer, R.scene_to_device(scene), [cam])[0]
    compare_to_oracle(to_numpy_images(out), oracle.render(scene, cam), max_flag_frac=DENSE_TIE_FLAG_FRAC)
    plain = dict(cam)
    plain["dt"] = 0.0
    ref_plain = gpu_render(renderer, R.scene_to_device(scene), [plain])[0]
    assert not torch.equal(out["rgb"], ref_plain["rgb"])


@pytest.mark.parametrize("jitter", [False, True])
def test_sky_cube_map_matches_oracle(renderer, jitter):
    """Sky refinement (Sec. 3.4): C + (1 - O) f_sky(d)."""
    rng = np.random.default_rng(14)
    scene = synth.make_fd_scene(seed=14, n=600, sh_degree=2)
    cam = synth.fd_camera(72, 56, t=0.5)
    sky = rng.uniform(0, 1, size=(6, 16, 16, 3)).astype(np.float32)
    jit = rng.uniform(-0.5, 0.5, size=(2, 56, 72)).astype(np.float32) if jitter else None
    st = R.scene_to_device(scene)
    st["sky"] = torch.tensor(sky, device="cuda")
    gcam = dict(cam)
    if jitter:
        gcam["sky_jitter"] = torch.tensor(jit, device="cuda")
    out = gpu_render(renderer, st, [gcam])[0]
    ref = oracle.render(scene, cam, sky=sky, sky_jitter=jit)
    compare_to_oracle(to_numpy_images(out), ref)


def test_sky_behind_an_empty_scene_is_the_sky(renderer):
    rng = np.random.default_rng(15)
    empty = {k: v[:0] for k, v in synth.make_plain_scene(seed=0, n=4).items()}
    sky = rng.uniform(0, 1, size=(6, 8, 8, 3)).astype(np.float32)
    cam = synth.street_camera(0.3, 64, 40)
    st = R.scene_to_device(empty)
    st["sky"] = torch.tensor(sky, device="cuda")
    out = gpu_render(renderer, st, [cam])[0]
    ref = oracle.render(empty, cam, sky=sky)
    np.testing.assert_allclose(to_numpy_images(out)["rgb"], ref["rgb"], atol=1e-5)


@pytest.mark.parametrize("cfg", [(16, 16, 1), (32, 32, 4), (8, 8, 2)])
def test_gaussians_beyond_the_jacobian_clamp_match_oracle(cfg):
    """Large Gaussians centred outside the view, beyond the clamp limits of
    the EWA Jacobian on both axes and both sides (x/z or y/z past 1.3 x
    the half field of view), whose footprints still cover the image; the
    camera has fx != fy, W != H and an off-centre principal point."""
    cam = clamp_camera()
    cam["t"] = 0.45
    scene, n_off = clamped_scene(cam, n=150, seed=1)
    scene = {k: v.astype(np.float32) for k, v in scene.items()}  # the same bytes for both sides
    limx, limy = clamp_limits(cam)
    pp = oracle.preprocess(scene, cam)
    r_xy = pp["pcam"][:, :2] / pp["pcam"][:, 2:3]
    assert np.all((np.abs(r_xy[:n_off, 0]) > limx) | (np.abs(r_xy[:n_off, 1]) > limy))
    r = R.Renderer(tile=cfg[:2], pixels_per_thread=cfg[2])
    fr = R.Frame()
    out = gpu_render(r, R.scene_to_device(scene), [cam], frame=fr)[0]
    compare_to_oracle(to_numpy_images(out), oracle.render(scene, cam))
    # the clamped Gaussians reach the image and their records carry the
    # clamped covariance
    tx, ty = R.tiles_of(cam, cfg[:2])
    ex = fr.export(tx * ty)
    gid = ex["sorted_gid"].astype(np.int64)
    assert np.sum(gid < n_off) >= n_off - 2
    conic = pp["conic"][gid]
    scale = np.abs(conic).max(axis=1, keepdims=True)
    np.testing.assert_allclose(ex["records"][:, 2:4] / scale, conic[:, 0:2] / scale, atol=1e-4)
    np.testing.assert_allclose(ex["records"][:, 4] / scale[:, 0], conic[:, 2] / scale[:, 0], atol=1e-4)
    r.close()
    fr.close()

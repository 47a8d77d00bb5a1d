"""Parity at the benchmarked sizes, through the C ABI.  GPU only.

* The urban frame the benchmark times (1.5M Gaussians, SH-3, 1920x1280,
  street-path frame 25) rendered in the compositing configurations the
  autotuner picks for it (32x32 tiles with 4 pixels per thread) and the
  default (16x16, 1): RGB, depth and opacity of 4,000 uniformly drawn
  pixels plus 1,000 in the dense band around the horizon, against the
  FP64 oracle's culled per-pixel compositing (Sec. 3.1, Eq. 3) at the
  image tolerance.  These frames exercise what the small parity scenes
  hardly reach: tile lists of thousands of entries, the heaviest-first tile
  order, the 16-keys-per-thread path of the tile sort and float atomics
  over thousands of tiles per Gaussian in the adjoint.
* The training frame (1M Gaussians, SH-3, 1242x375, f = 720) and the urban
  frame (in the benchmarked 32x32, 4-pixel configuration) backward with
  dL/dimage non-zero on 2,000 sampled pixels only (pixels the oracle does
  not flag), against the oracle's reverse mode restricted to those pixels:
  all nine parameter groups at the gradient tolerance (Sec. 3.2, Eq. 8: the
  render function is differentiable), for a colour loss (the training
  step's L1 path) and with depth and opacity weights.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18561_gb300 import render as R
from paper_2311_18561_gb300 import synth

from .gpu_util import compare_to_oracle, to_numpy_images
from .test_gpu_backward import _compare_grads

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def urban():
    scene = synth.make_urban_scene(1_500_000, seed=0)
    cam = synth.urban_frame_camera(25)
    W, H = cam["width"], cam["height"]
    rng = np.random.default_rng(25)
    uni = np.stack([rng.integers(0, W, 4000), rng.integers(0, H, 4000)], axis=1)
    band = np.stack([rng.integers(0, W, 1000), rng.integers(H // 2 - 96, H // 2 + 96, 1000)], axis=1)
    pix = np.concatenate([uni, band]).astype(np.int32)
    ref = oracle.render(scene, cam, mode="culled", pixels=pix)
    return scene, cam, pix, ref


@pytest.mark.parametrize("cfg", [(32, 32, 4), (16, 16, 1), (16, 32, 4)])
def test_urban_frame_sampled_pixels_match_oracle(urban, cfg):
    scene, cam, pix, ref = urban
    r = R.Renderer(tile=cfg[:2], pixels_per_thread=cfg[2])
    fr = R.Frame()
    out = r.forward(R.scene_to_device(scene), [cam], frame=fr)[0]
    torch.cuda.synchronize()
    m, k, ov = fr.stats()
    assert ov == 0 and m > 400_000 and k > 3_000_000  # the benchmark's visible and pair counts
    img = to_numpy_images(out)
    got = {key: img[key][pix[:, 1], pix[:, 0]] for key in ("rgb", "depth", "alpha")}
    compare_to_oracle(got, ref, pixels=pix)
    assert float(ref["alpha"].mean()) > 0.5  # the sample sees the scene, not the background
    assert int(ref["nblend"].max()) > 100  # deep per-pixel lists are among the sample
    r.close()
    fr.close()


def test_urban_frame_wide_sort_paths_render_identically(urban):
    """The sorts take 16 keys per thread above 4M keys, with their first
    digit histogram counted by the kernel that writes the keys (the
    compaction, the pair expansion).  The urban frame rendered with an 8M
    pair capacity (the tile sort's wide path) and as three identical views
    in one call (4.5M items: the depth sort's wide path) must give the
    single-view images bit for bit (the per-tile lists are the same)."""
    scene, cam, _, _ = urban
    st = R.scene_to_device(scene)
    r = R.Renderer(tile=(32, 32), pixels_per_thread=4)
    fr = R.Frame()
    ref = r.forward(st, [cam], frame=fr)[0]
    m, k, ov = fr.stats()
    assert ov == 0 and k < (4 << 20) < 8_000_000
    wide = R.Renderer(tile=(32, 32), pixels_per_thread=4, sync_sizes=False, pair_capacity=8_000_000)
    fr2 = R.Frame()
    out = wide.forward(st, [cam], frame=fr2)[0]
    m2, k2, ov2 = fr2.stats()
    assert (m2, k2, ov2) == (m, k, 0)
    fr3 = R.Frame()
    outs = r.forward(st, [cam, cam, cam], frame=fr3)
    m3, k3, ov3 = fr3.stats()
    assert (m3, k3, ov3) == (3 * m, 3 * k, 0) and 3 * 1_500_000 > (4 << 20)
    torch.cuda.synchronize()
    for got in [out] + list(outs):
        for key in ("rgb", "depth", "alpha"):
            assert torch.equal(got[key], ref[key]), key
    for x in (r, wide, fr, fr2, fr3):
        x.close()


@pytest.fixture(scope="module")
def training():
    scene = synth.make_urban_scene(1_000_000, seed=0)
    cam = synth.street_camera(25 / 49.0, 1242, 375, fx=720.0)
    cam["bg"] = np.array([0.1, 0.2, 0.3], np.float32)
    W, H = cam["width"], cam["height"]
    rng = np.random.default_rng(3)
    idx = rng.choice(W * H, 2300, replace=False)
    pix = np.stack([idx % W, idx // W], axis=1).astype(np.int32)
    flags = oracle.render(scene, cam, mode="culled", pixels=pix)["flag"]
    pix = pix[flags == 0][:2000]  # pixels where FP32 and FP64 take the same gate decisions
    assert pix.shape[0] == 2000
    return scene, cam, pix


def _sampled_backward(scene, cam, pix, cfg, colour_only):
    """dL/dimage non-zero on the sampled pixels only; the nine gradient
    groups against the oracle's reverse mode restricted to those pixels."""
    W, H = cam["width"], cam["height"]
    P = pix.shape[0]
    rng = np.random.default_rng(4)
    w_rgb = rng.normal(size=(P, 3)) / P
    w_d = np.zeros(P) if colour_only else rng.normal(size=P) * 0.01 / P
    w_a = np.zeros(P) if colour_only else rng.normal(size=P) / P
    dl_rgb = np.zeros((3, H, W), np.float32)
    dl_rgb[:, pix[:, 1], pix[:, 0]] = w_rgb.T
    dl = dict(rgb=torch.tensor(dl_rgb, device="cuda"))
    if not colour_only:
        dl_d = np.zeros((H, W), np.float32)
        dl_a = np.zeros((H, W), np.float32)
        dl_d[pix[:, 1], pix[:, 0]] = w_d
        dl_a[pix[:, 1], pix[:, 0]] = w_a
        dl["depth"] = torch.tensor(dl_d, device="cuda")
        dl["alpha"] = torch.tensor(dl_a, device="cuda")
    # the oracle sees the FP32 weights the GPU sees
    w_rgb = dl_rgb[:, pix[:, 1], pix[:, 0]].T.astype(np.float64)
    if not colour_only:
        w_d = dl["depth"].cpu().numpy()[pix[:, 1], pix[:, 0]].astype(np.float64)
        w_a = dl["alpha"].cpu().numpy()[pix[:, 1], pix[:, 0]].astype(np.float64)
    r = R.Renderer(tile=cfg[:2], pixels_per_thread=cfg[2])
    fr = R.Frame()
    st = R.scene_to_device(scene)
    r.forward(st, [cam], frame=fr)
    grads = r.backward(st, [cam], fr, [dl])
    torch.cuda.synchronize()
    ref = oracle.render_bwd(scene, cam, w_rgb, w_d, w_a, mode="culled", pixels=pix)
    touched = np.count_nonzero(np.abs(ref["opacity"]))
    assert touched > 5000  # many Gaussians receive gradient from the sampled pixels
    _compare_grads(grads, ref)
    r.close()
    fr.close()


@pytest.mark.parametrize("cfg", [(16, 8, 1), (32, 32, 4)])
@pytest.mark.parametrize("colour_only", [True, False])
def test_training_frame_backward_on_sampled_pixels(training, cfg, colour_only):
    scene, cam, pix = training
    _sampled_backward(scene, cam, pix, cfg, colour_only)


@pytest.mark.parametrize("colour_only", [True, False])
def test_urban_frame_backward_on_sampled_pixels(urban, colour_only):
    """The benchmarked step's backward: the urban frame in the autotuner's
    configuration (32x32 tiles, 4 pixels per thread), colour-only (the L1
    path the benchmark times) and with depth and opacity weights, on 2,000
    of the sampled pixels where the oracle flags no gate decision."""
    scene, cam, pix, ref = urban
    pix = pix[ref["flag"] == 0]
    # distinct pixels: the oracle sums over the list, the image holds one
    # weight per pixel, so a repeated pixel would count twice on one side
    _, first = np.unique(pix[:, 1] * cam["width"] + pix[:, 0], return_index=True)
    pix = pix[np.sort(first)][:2000]
    assert pix.shape[0] == 2000
    _sampled_backward(scene, cam, pix, (32, 32, 4), colour_only)

"""Parity of the extra composited channels (velocity map, staticness map,
semantic map; Sec. 4) of the CUDA path with the FP64 oracle, forward and
backward, through the C ABI.  GPU only.

Tolerances, per channel: a channel value x composited with weights summing
to O <= 1 is held to 1e-3 max(1, max|x|) on pixels the oracle does not flag
and to (1/255 + 1e-3) max(1, max|x|) on flagged ones (the colour channels'
rule, scaled by that channel's range over the points: max |v_c| for the
velocity channel c, since v_bar = v exp(-rho/2) never exceeds v; 2 for the
clamped staticness; max |sem_j| for class j); gradients as in the colour
backward tests (relative norm and max-element error <= 1e-2 per parameter
group).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18561_gb300 import abi
from paper_2311_18561_gb300 import render as R
from paper_2311_18561_gb300 import synth

from . import parity_log
from .gpu_util import FLAG_TOL, MAX_FLAG_FRAC, DENSE_TIE_FLAG_FRAC, TOL, compare_to_oracle, to_numpy_images

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

VBAR, RHO, SEM = abi.FEAT_VBAR, abi.FEAT_RHO, abi.FEAT_SEM
NAMES = R.PARAM_NAMES


def _device_scene(scene, sem=None):
    st = R.scene_to_device(scene)
    if sem is not None:
        st["sem"] = torch.tensor(np.asarray(sem, np.float32), device="cuda")
    return st


def _feat_np(out):
    return out["feat"].permute(1, 2, 0).cpu().numpy().astype(np.float64)


def channel_scales(mask, scene, sem=None):
    """max(1, range of the per-point values) of every channel of `mask`, in
    the feature image's channel order."""
    out = []
    if mask & VBAR:
        out += [max(1.0, float(np.abs(scene["vel"][:, c]).max(initial=0))) for c in range(3)]
    if mask & RHO:
        out.append(2.0)
    if mask & SEM:
        out += [max(1.0, float(np.abs(sem[:, j]).max(initial=0))) for j in range(sem.shape[1])]
    return np.asarray(out)


def _compare_feat(got, ref, scales, max_flag_frac=MAX_FLAG_FRAC):
    """Per-channel comparison: got and ref["feat"] are [..., F], scales [F]."""
    flag = ref["flag"] != 0
    err = np.abs(got - ref["feat"]) / scales  # [..., F] in units of each channel's scale
    ok = ~flag
    per_ch = err[ok].max(axis=0, initial=0) if err[ok].size else np.zeros(err.shape[-1])
    rep = dict(max_err=float(per_ch.max(initial=0)), worst_channel=int(np.argmax(per_ch)) if per_ch.size else -1,
               flagged=int(flag.sum()), flagged_max=float(err[flag].max(initial=0)),
               scales=[round(float(v), 3) for v in scales])
    parity_log.record("feat", flag.size, flag.sum(), scaled=rep["max_err"], flagged_max=rep["flagged_max"])
    assert rep["max_err"] <= TOL, rep
    assert rep["flagged_max"] <= FLAG_TOL, rep
    assert flag.mean() <= max_flag_frac, rep
    return rep


@pytest.mark.parametrize("mask,n_sem", [(VBAR, 0), (RHO, 0), (SEM, 19), (VBAR | RHO | SEM, 19),
                                        (VBAR | RHO | SEM, 32), (RHO | SEM, 1)])
def test_feature_maps_match_oracle(mask, n_sem):
    # 70 x 50: 5 x 4 tiles of 16 x 16 with a ragged right and bottom edge
    scene = synth.make_fd_scene(seed=3, n=500, sh_degree=1)
    sem = synth.make_semantics(500, n_sem) if n_sem else None
    cam = synth.fd_camera(70, 50, t=0.55)
    st = _device_scene(scene, sem)
    r = R.Renderer()
    plain = R.Renderer().forward(st, [cam])[0]
    out = r.forward(st, [cam], features=mask)[0]
    torch.cuda.synchronize()
    F = R.feat_count(mask, n_sem)
    assert tuple(out["feat"].shape) == (F, 50, 70)
    # the colour, depth and opacity images do not change
    for k in ("rgb", "depth", "alpha"):
        assert torch.equal(plain[k], out[k]), k
    ref = oracle.render(scene, cam, mode="culled", features=mask, sem=sem)
    _compare_feat(_feat_np(out), ref, channel_scales(mask, scene, sem), max_flag_frac=DENSE_TIE_FLAG_FRAC)


@pytest.mark.parametrize("tile,px", [((16, 16), 1), ((8, 8), 2), ((32, 16), 4), ((32, 32), 4), ((16, 8), 1)])
def test_feature_maps_do_not_depend_on_the_tile_shape(tile, px):
    scene = synth.make_fd_scene(seed=4, n=600, sh_degree=0)
    sem = synth.make_semantics(600, 7)
    cam = synth.fd_camera(83, 61, t=0.35)
    st = _device_scene(scene, sem)
    base = R.Renderer().forward(st, [cam], features=VBAR | RHO | SEM)[0]
    out = R.Renderer(tile=tile, pixels_per_thread=px).forward(st, [cam], features=VBAR | RHO | SEM)[0]
    torch.cuda.synchronize()
    assert torch.equal(base["feat"], out["feat"])


def test_semantic_weights_are_the_colour_weights():
    # degree-0 colours used as 3-channel semantics: with a zero background
    # the semantic map equals the colour image up to the colours' rounding
    scene = synth.make_fd_scene(seed=5, n=500, sh_degree=0)
    colour = (np.float32(0.5 / np.sqrt(np.pi)) * scene["sh"][:, 0, :] + np.float32(0.5)).astype(np.float32)
    assert colour.min() > 0
    cam = synth.fd_camera(64, 48, t=0.5)
    st = _device_scene(scene, colour)
    out = R.Renderer().forward(st, [cam], features=SEM)[0]
    torch.cuda.synchronize()
    diff = (out["feat"] - out["rgb"]).abs().max().item()
    assert diff <= 2e-6, diff


def test_feature_maps_of_an_empty_scene_are_zero():
    scene = {k: v[:0] for k, v in synth.make_fd_scene(seed=0, n=4, sh_degree=0).items()}
    st = _device_scene(scene, np.zeros((0, 3), np.float32))
    cam = synth.fd_camera(40, 30)
    out = R.Renderer().forward(st, [cam], features=VBAR | RHO | SEM)[0]
    torch.cuda.synchronize()
    assert out["feat"].shape[0] == 7 and out["feat"].abs().max().item() == 0.0


def test_feature_requests_are_validated():
    scene = synth.make_fd_scene(seed=0, n=50, sh_degree=0)
    st = _device_scene(scene)
    cam = synth.fd_camera(32, 32)
    r = R.Renderer()
    with pytest.raises(abi.PVGError):  # semantics without semantic vectors
        outs = r.alloc_images([cam], features=SEM, n_sem=3)
        r.forward(st, [cam], outs=outs, features=SEM)
    with pytest.raises(abi.PVGError):  # unknown channel bit
        outs = r.alloc_images([cam], features=VBAR)
        r.forward(st, [cam], outs=outs, features=8)
    fr = R.Frame()
    r.forward(st, [cam], frame=fr)
    with pytest.raises(abi.PVGError):  # channel gradient for a forward without channels
        r.backward(st, [cam], fr, [dict(feat=torch.zeros(4, 32, 32, device="cuda"))])
    torch.cuda.synchronize()


def _compare_grads(got, ref, names, rel=1e-2):
    report = {}
    for k in names:
        g = got[k].detach().cpu().numpy().astype(np.float64).reshape(-1)
        r = ref[k].reshape(-1)
        nr = np.linalg.norm(r)
        if nr == 0:
            assert np.abs(g).max(initial=0) == 0, k
            continue
        report[k] = (float(np.linalg.norm(g - r) / nr), float(np.abs(g - r).max() / np.abs(r).max()))
    for k, (nrm, mx) in report.items():
        assert nrm <= rel and mx <= rel, (k, report)
    return report


@pytest.mark.parametrize("with_rgb", [True, False])
def test_feature_backward_matches_oracle(with_rgb):
    n, S = 500, 5
    scene = synth.make_fd_scene(seed=6, n=n, sh_degree=1)
    sem = synth.make_semantics(n, S, seed=7)
    cam = synth.fd_camera(64, 48, t=0.45)
    H, W = cam["height"], cam["width"]
    mask = VBAR | RHO | SEM
    F = R.feat_count(mask, S)
    rng = np.random.default_rng(8)
    w_rgb = rng.normal(size=(3, H, W)) if with_rgb else np.zeros((3, H, W))
    w_f = rng.normal(size=(F, H, W))
    st = _device_scene(scene, sem)
    r = R.Renderer()
    fr = R.Frame()
    r.forward(st, [cam], frame=fr, features=mask)
    dl = dict(feat=torch.tensor(w_f, dtype=torch.float32, device="cuda"))
    if with_rgb:
        dl["rgb"] = torch.tensor(w_rgb, dtype=torch.float32, device="cuda")
    grads = r.backward(st, [cam], fr, [dl])
    torch.cuda.synchronize()
    ref = oracle.render_bwd(scene, cam, np.transpose(w_rgb, (1, 2, 0)), np.zeros((H, W)), np.zeros((H, W)),
                            features=mask, sem=sem, dL_feat=np.transpose(w_f, (1, 2, 0)))
    _compare_grads(grads, ref, NAMES + ("sem",))


def test_feature_backward_two_views_accumulates():
    n, S = 400, 3
    scene = synth.make_fd_scene(seed=9, n=n, sh_degree=0)
    sem = synth.make_semantics(n, S, seed=2)
    cams = [synth.fd_camera(48, 40, t=0.3), synth.fd_camera(56, 32, t=0.6)]
    mask = RHO | SEM | VBAR
    F = R.feat_count(mask, S)
    rng = np.random.default_rng(10)
    wf = [rng.normal(size=(F, c["height"], c["width"])) for c in cams]
    st = _device_scene(scene, sem)
    r = R.Renderer()
    fr = R.Frame()
    r.forward(st, cams, frame=fr, features=mask)
    grads = r.backward(st, cams, fr, [dict(feat=torch.tensor(w, dtype=torch.float32, device="cuda")) for w in wf])
    torch.cuda.synchronize()
    ref = None
    for c, w in zip(cams, wf):
        H, W = c["height"], c["width"]
        g = oracle.render_bwd(scene, c, np.zeros((H, W, 3)), np.zeros((H, W)), np.zeros((H, W)), features=mask,
                              sem=sem, dL_feat=np.transpose(w, (1, 2, 0)))
        ref = g if ref is None else {k: ref[k] + g[k] for k in ref}
    _compare_grads(grads, ref, NAMES + ("sem",))


def test_feature_maps_at_street_scale_sampled_pixels():
    """A 200k-Gaussian urban scene at 1242 x 375 in the 32 x 16 x 4
    compositor configuration, 19-class semantics: 1500 sampled pixels of
    every channel (colour, depth, opacity and the extra channels) against
    the oracle's culled per-pixel compositing."""
    n, S = 200_000, 19
    scene = synth.make_urban_scene(n, seed=1)
    sem = synth.make_semantics(n, S, seed=4)
    cam = synth.kitti_camera(t=0.5)
    st = _device_scene(scene, sem)
    r = R.Renderer(tile=(32, 16), pixels_per_thread=4)
    mask = VBAR | RHO | SEM
    out = r.forward(st, [cam], features=mask)[0]
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(0, cam["width"], 1500), rng.integers(0, cam["height"], 1500)], -1)
    ref = oracle.render(scene, cam, mode="culled", pixels=pix, features=mask, sem=sem)
    feat = _feat_np(out)[pix[:, 1], pix[:, 0]]
    _compare_feat(feat, ref, channel_scales(mask, scene, sem), max_flag_frac=DENSE_TIE_FLAG_FRAC)
    got = to_numpy_images(out)
    compare_to_oracle({k: got[k][pix[:, 1], pix[:, 0]] for k in ("rgb", "depth", "alpha")}, ref, pixels=pix,
                      max_flag_frac=DENSE_TIE_FLAG_FRAC)

"""Parity of the CUDA backward path (stage d) with the oracle's FP64
reverse mode, through the C ABI and through torch.autograd.  GPU only.

Tolerance: per parameter group, ||g - g_ref|| / ||g_ref|| <= 1e-2, and
per element |g - g_ref| <= 1e-2 max|g_ref| (FP32 accumulation order and
rare gate decisions that FP32 takes differently from FP64 stay inside it).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_18561_gb300 import render as R
from paper_2311_18561_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

NAMES = R.PARAM_NAMES

from .test_oracle_clamp import _camera as clamp_camera  # noqa: E402
from .test_oracle_clamp import clamped_scene  # noqa: E402


def _compare_grads(got, ref, rel=1e-2):
    report = {}
    for k in NAMES:
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


def _weights(H, W, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(3, H, W)), rng.normal(size=(H, W)) * 0.1, rng.normal(size=(H, W))


@pytest.mark.parametrize("deg,dt", [(0, 0.0), (3, 0.0), (3, 0.04)])
def test_backward_matches_oracle_fd_subcase(deg, dt):
    """The 500-Gaussian, 64x48 sub-case of the training config (dt != 0:
    the flow-translated state of Sec. 3.4)."""
    scene = synth.make_fd_scene(seed=0, n=500, sh_degree=deg)
    cam = synth.fd_camera(64, 48, t=0.45)
    cam["dt"] = dt
    cam["bg"] = np.array([0.2, 0.5, 0.8], np.float32)
    H, W = cam["height"], cam["width"]
    w_rgb, w_d, w_a = _weights(H, W, 1)
    r = R.Renderer()
    fr = R.Frame()
    st = R.scene_to_device(scene)
    r.forward(st, [cam], frame=fr)
    dl = dict(rgb=torch.tensor(w_rgb, dtype=torch.float32, device="cuda"),
              depth=torch.tensor(w_d, dtype=torch.float32, device="cuda"),
              alpha=torch.tensor(w_a, dtype=torch.float32, device="cuda"))
    grads = r.backward(st, [cam], fr, [dl])
    torch.cuda.synchronize()
    ref = oracle.render_bwd(scene, cam, np.transpose(w_rgb, (1, 2, 0)), w_d, w_a)
    _compare_grads(grads, ref)


def test_autograd_l1_training_step():
    """L1 loss against a random target (the training config's loss) through
    torch.autograd; gradients against the oracle's with dL/dimage = sign/n."""
    scene = synth.make_fd_scene(seed=3, n=500, sh_degree=3)
    cam = synth.fd_camera(64, 48, t=0.6)
    target = synth.random_image(48, 64, seed=1)
    st = R.scene_to_device(scene)
    params = {k: v.clone().requires_grad_(True) for k, v in st.items()}
    rgb, depth, alpha = R.render_differentiable(params, cam)
    tgt = torch.tensor(target, device="cuda")
    loss = (rgb - tgt).abs().mean()
    loss.backward()
    torch.cuda.synchronize()
    dl = torch.sign(rgb.detach() - tgt).cpu().numpy() / rgb.numel()
    ref = oracle.render_bwd(scene, cam, np.transpose(dl, (1, 2, 0)), np.zeros((48, 64)), np.zeros((48, 64)))
    _compare_grads({k: params[k].grad for k in NAMES}, ref)


@pytest.mark.parametrize("cfg", [(16, 16, 2), (16, 16, 4), (32, 32, 4)])
def test_backward_multi_pixel_configs(cfg):
    scene = synth.make_fd_scene(seed=7, n=500, sh_degree=3)
    cam = synth.fd_camera(64, 48, t=0.35)
    H, W = cam["height"], cam["width"]
    w_rgb, w_d, w_a = _weights(H, W, 5)
    r = R.Renderer(tile=cfg[:2], pixels_per_thread=cfg[2])
    fr = R.Frame()
    st = R.scene_to_device(scene)
    r.forward(st, [cam], frame=fr)
    dl = dict(rgb=torch.tensor(w_rgb, dtype=torch.float32, device="cuda"),
              depth=torch.tensor(w_d, dtype=torch.float32, device="cuda"),
              alpha=torch.tensor(w_a, dtype=torch.float32, device="cuda"))
    grads = r.backward(st, [cam], fr, [dl])
    torch.cuda.synchronize()
    ref = oracle.render_bwd(scene, cam, np.transpose(w_rgb, (1, 2, 0)), w_d, w_a)
    _compare_grads(grads, ref)


def test_multi_view_backward_sums_views():
    scene = synth.make_fd_scene(seed=4, n=400, sh_degree=1)
    cams = [synth.fd_camera(48, 40, t=0.2), synth.fd_camera(64, 48, t=0.7)]
    st = R.scene_to_device(scene)
    r = R.Renderer()
    fr = R.Frame()
    r.forward(st, cams, frame=fr)
    dls, ref = [], None
    for k, cam in enumerate(cams):
        w_rgb, w_d, w_a = _weights(cam["height"], cam["width"], 10 + k)
        dls.append(dict(rgb=torch.tensor(w_rgb, dtype=torch.float32, device="cuda"),
                        depth=torch.tensor(w_d, dtype=torch.float32, device="cuda"),
                        alpha=torch.tensor(w_a, dtype=torch.float32, device="cuda")))
        g = oracle.render_bwd(scene, cam, np.transpose(w_rgb, (1, 2, 0)), w_d, w_a)
        ref = g if ref is None else {n: ref[n] + g[n] for n in NAMES}
    grads = r.backward(st, cams, fr, dls)
    torch.cuda.synchronize()
    _compare_grads(grads, ref)


def test_backward_of_empty_scene_is_empty():
    empty = {k: v[:0] for k, v in synth.make_plain_scene(seed=0, n=4).items()}
    st = R.scene_to_device(empty)
    cam = synth.plain_camera(width=32, height=24)
    r = R.Renderer()
    fr = R.Frame()
    r.forward(st, [cam], frame=fr)
    grads = r.backward(st, [cam], fr, [dict(rgb=torch.ones(3, 24, 32, device="cuda"))])
    assert all(g.numel() == 0 for g in grads.values())


def test_backward_with_sky_cube_map():
    rng = np.random.default_rng(16)
    scene = synth.make_fd_scene(seed=8, n=400, sh_degree=1)
    cam = synth.fd_camera(64, 48, t=0.5)
    sky = rng.uniform(0, 1, size=(6, 8, 8, 3)).astype(np.float32)
    H, W = cam["height"], cam["width"]
    w_rgb, w_d, w_a = _weights(H, W, 17)
    st = R.scene_to_device(scene)
    st["sky"] = torch.tensor(sky, device="cuda")
    r = R.Renderer()
    fr = R.Frame()
    r.forward(st, [cam], frame=fr)
    dl = dict(rgb=torch.tensor(w_rgb, dtype=torch.float32, device="cuda"),
              depth=torch.tensor(w_d, dtype=torch.float32, device="cuda"),
              alpha=torch.tensor(w_a, dtype=torch.float32, device="cuda"))
    grads = r.backward(st, [cam], fr, [dl])
    torch.cuda.synchronize()
    ref = oracle.render_bwd(scene, cam, np.transpose(w_rgb, (1, 2, 0)), w_d, w_a, sky=sky)
    _compare_grads(grads, ref)
    g = grads["sky"].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref["sky"]) <= 1e-3 * np.linalg.norm(ref["sky"])


@pytest.mark.parametrize("cfg", [(16, 16, 1), (16, 32, 4), (32, 16, 2)])
def test_backward_colour_only(cfg):
    """Only dL/drgb given (no depth or opacity-map gradient, no sky): the
    compositor adjoint's reduced form, against the oracle with zero depth
    and opacity weights."""
    scene = synth.make_fd_scene(seed=11, n=500, sh_degree=3)
    cam = synth.fd_camera(64, 48, t=0.55)
    cam["bg"] = np.array([0.3, 0.1, 0.6], np.float32)
    H, W = cam["height"], cam["width"]
    w_rgb, _, _ = _weights(H, W, 9)
    r = R.Renderer(tile=cfg[:2], pixels_per_thread=cfg[2])
    fr = R.Frame()
    st = R.scene_to_device(scene)
    r.forward(st, [cam], frame=fr)
    grads = r.backward(st, [cam], fr, [dict(rgb=torch.tensor(w_rgb, dtype=torch.float32, device="cuda"))])
    torch.cuda.synchronize()
    ref = oracle.render_bwd(scene, cam, np.transpose(w_rgb, (1, 2, 0)), np.zeros((H, W)), np.zeros((H, W)))
    _compare_grads(grads, ref)


@pytest.mark.parametrize("colour_only", [False, True])
def test_backward_through_the_jacobian_clamp(colour_only):
    """Gradients of a scene whose large Gaussians sit beyond the EWA
    Jacobian's clamp limits (both axes, both sides), against the oracle's
    reverse mode through its clamped branch."""
    cam = clamp_camera()
    cam["t"] = 0.45
    cam["bg"] = np.array([0.2, 0.5, 0.8], np.float32)
    scene, n_off = clamped_scene(cam, n=150, seed=2)
    scene = {k: v.astype(np.float32) for k, v in scene.items()}  # the same bytes for both sides
    H, W = cam["height"], cam["width"]
    w_rgb, w_d, w_a = _weights(H, W, 21)
    if colour_only:
        w_d, w_a = np.zeros((H, W)), np.zeros((H, W))
    r = R.Renderer()
    fr = R.Frame()
    st = R.scene_to_device(scene)
    r.forward(st, [cam], frame=fr)
    dl = dict(rgb=torch.tensor(w_rgb, dtype=torch.float32, device="cuda"))
    if not colour_only:
        dl["depth"] = torch.tensor(w_d, dtype=torch.float32, device="cuda")
        dl["alpha"] = torch.tensor(w_a, dtype=torch.float32, device="cuda")
    grads = r.backward(st, [cam], fr, [dl])
    torch.cuda.synchronize()
    ref = oracle.render_bwd(scene, cam, np.transpose(w_rgb, (1, 2, 0)), w_d, w_a)
    _compare_grads(grads, ref)
    # the clamped Gaussians carry gradient
    assert np.count_nonzero(np.abs(ref["mu"][:n_off]).sum(axis=1)) >= n_off - 2


def test_backward_of_70_views_sums_the_views():
    """70 views of one scene (more than the 64 views one pass of the
    multi-view adjoint groups together), some seeing a Gaussian and some
    not: the gradients are the sum of the oracle's per-view gradients."""
    scene = synth.make_fd_scene(seed=9, n=300, sh_degree=2)
    rng = np.random.default_rng(19)
    cams = []
    for k in range(70):
        eye = (rng.uniform(-1.5, 1.5), rng.uniform(-1.0, 1.0), -3.5)
        vm = synth.look_at(eye, (rng.uniform(-0.3, 0.3), 0.0, 0.0), (0.0, 1.0, 0.0))
        w, h = int(rng.integers(20, 40)), int(rng.integers(16, 32))
        cams.append(synth.make_camera(vm, w, h, synth.focal_from_hfov(w, 55.0), t=float(rng.uniform(0, 1))))
    st = R.scene_to_device(scene)
    r = R.Renderer()
    fr = R.Frame()
    r.forward(st, cams, frame=fr)
    dls, ref = [], None
    for k, cam in enumerate(cams):
        w_rgb, w_d, w_a = _weights(cam["height"], cam["width"], 100 + k)
        dls.append(dict(rgb=torch.tensor(w_rgb, dtype=torch.float32, device="cuda"),
                        depth=torch.tensor(w_d, dtype=torch.float32, device="cuda"),
                        alpha=torch.tensor(w_a, dtype=torch.float32, device="cuda")))
        g = oracle.render_bwd(scene, cam, np.transpose(w_rgb, (1, 2, 0)), w_d, w_a)
        ref = g if ref is None else {n: ref[n] + g[n] for n in NAMES}
    # stale values in the gradient buffers must not survive: every entry is written
    grads = {k: torch.full_like(st[k], 7.0) for k in NAMES}
    r.backward(st, cams, fr, dls, grads=grads)
    torch.cuda.synchronize()
    _compare_grads(grads, ref)


@pytest.mark.parametrize("deg", [3, 2])
def test_backward_into_unaligned_and_partial_gradient_buffers(deg):
    """The per-item adjoint writes every gradient entry, float4-wide where
    the arrays allow it.  Gradient arrays that start 4 bytes past a 16-byte
    boundary, a Gaussian count that leaves a partial last chunk (1,037 =
    16 x 64 + 13), SH rows that are not whole float4 (degree 2: 27 floats)
    and arrays left out (NULL) must give the values of aligned arrays
    (equal up to the order of the compositor adjoint's float atomics, which
    differs between calls; exact zeros for the culled Gaussians) and must
    write nothing else."""
    scene = synth.make_fd_scene(seed=21, n=1037, sh_degree=deg)
    scene["mu"][::3, 0] += 1000.0  # every third Gaussian far off to the side: culled
    cam = synth.fd_camera(64, 48, t=0.4)
    H, W = cam["height"], cam["width"]
    w_rgb, w_d, w_a = _weights(H, W, 23)
    dl = dict(rgb=torch.tensor(w_rgb, dtype=torch.float32, device="cuda"),
              depth=torch.tensor(w_d, dtype=torch.float32, device="cuda"),
              alpha=torch.tensor(w_a, dtype=torch.float32, device="cuda"))
    r = R.Renderer()
    fr = R.Frame()
    st = R.scene_to_device(scene)
    r.forward(st, [cam], frame=fr)
    ref = r.backward(st, [cam], fr, [dl])
    assert int((ref["opacity"] != 0).sum()) > 300 and int((ref["opacity"] == 0).sum()) >= 346
    # each array one float past its buffer's (aligned) start, guarded on both sides
    bufs, grads = {}, {}
    for k in NAMES:
        n = st[k].numel()
        bufs[k] = torch.full((n + 2,), 7.0, device="cuda")
        grads[k] = bufs[k][1:1 + n].view(st[k].shape)
        assert grads[k].data_ptr() % 16 == 4
    culled = torch.zeros(st["mu"].shape[0], dtype=torch.bool, device="cuda")
    culled[::3] = True

    def same(a, b, k):
        assert torch.all(a[culled] == 0) and torch.all(b[culled] == 0), k
        assert float((a - b).abs().max()) <= 1e-5 * float(b.abs().max()), k

    got = r.backward(st, [cam], fr, [dl], grads=grads)
    torch.cuda.synchronize()
    for k in NAMES:
        same(got[k], ref[k], k)
        assert float(bufs[k][0]) == 7.0 and float(bufs[k][-1]) == 7.0, k
    # only some arrays asked for: those match, nothing else is touched
    some = {k: (torch.full_like(st[k], 7.0) if k in ("mu", "opacity", "sh") else None) for k in NAMES}
    got = r.backward(st, [cam], fr, [dl], grads=some)
    torch.cuda.synchronize()
    for k in ("mu", "opacity", "sh"):
        same(got[k], ref[k], k)
    r.close()
    fr.close()


@pytest.mark.parametrize("n_views", [1, 3])
def test_repeated_backward_writes_every_entry(n_views):
    """The per-item adjoints hand out their chunks from a ticket that the
    backward's first kernel resets: a second backward on the same frame,
    into gradient buffers filled with NaN, writes every entry again (zeros
    for the Gaussians no view sees) and gives the first call's gradients up
    to the order of the float atomics."""
    scene = synth.make_urban_scene(20_000, seed=3)
    cams = [synth.street_camera(0.3 + 0.2 * v, 160, 120) for v in range(n_views)]
    st = R.scene_to_device(scene)
    r = R.Renderer(tile=(16, 16), pixels_per_thread=2)
    fr = R.Frame()
    r.forward(st, cams, frame=fr)
    rng = np.random.default_rng(7)
    dls = [dict(rgb=torch.tensor(rng.normal(size=(3, 120, 160)), dtype=torch.float32, device="cuda"))
           for _ in cams]
    runs = []
    for _ in range(2):
        grads = {k: torch.full_like(st[k], float("nan")) for k in NAMES}
        r.backward(st, cams, fr, dls, grads=grads)
        torch.cuda.synchronize()
        runs.append(grads)
    m, _, _ = fr.stats()
    assert 0 < m < n_views * 20_000  # some Gaussians are seen, some are not
    for k in NAMES:
        a, b = runs[0][k], runs[1][k]
        assert torch.isfinite(a).all() and torch.isfinite(b).all(), k
        scale = max(a.abs().max().item(), 1e-30)
        assert (a - b).abs().max().item() <= 1e-4 * scale, k

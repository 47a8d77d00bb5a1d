"""PyTorch-facing API of the rasterizer.

PyTorch supplies device memory and the stream; every step of the render and
of its adjoint runs in the CUDA library through :mod:`.abi`.

``render(scene, cams)`` renders N-view images; ``PVGRender`` is the
``torch.autograd.Function`` whose backward calls ``pvg_render_bwd``
(Sec. 3.1, Eq. 4: the render function is differentiable; gradients for
every learnable parameter of Sec. 3.2).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import abi

PARAM_NAMES = ("mu", "vel", "tau", "beta", "period", "scale", "quat", "opacity", "sh")


def scene_to_device(scene, device="cuda"):
    """numpy scene dict -> dict of contiguous float32 CUDA tensors."""
    return {k: torch.as_tensor(np.ascontiguousarray(scene[k], dtype=np.float32)).to(device)
            for k in PARAM_NAMES}


def sh_degree(scene_t) -> int:
    k = scene_t["sh"].shape[1]
    d = int(round(k ** 0.5)) - 1
    if (d + 1) ** 2 != k or not 0 <= d <= 3:
        raise ValueError("sh must be [N, (D+1)^2, 3] with D in 0..3")
    return d


def _check_scene(scene_t):
    n = scene_t["mu"].shape[0]
    shapes = dict(mu=(n, 3), vel=(n, 3), tau=(n,), beta=(n,), period=(n,), scale=(n, 3), quat=(n, 4),
                  opacity=(n,))
    for k, s in shapes.items():
        t = scene_t[k]
        if tuple(t.shape) != s or t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError("scene[%r] must be a contiguous float32 CUDA tensor of shape %s" % (k, s))
    sh = scene_t["sh"]
    if sh.dim() != 3 or sh.shape[0] != n or sh.shape[2] != 3 or sh.dtype != torch.float32 or not sh.is_contiguous():
        raise ValueError("scene['sh'] must be a contiguous float32 CUDA tensor [N, K, 3]")
    return n


def abi_scene(scene_t) -> abi.Scene:
    n = _check_scene(scene_t)
    s = abi.Scene()
    s.n = n
    s.sh_degree = sh_degree(scene_t)
    for k in PARAM_NAMES:
        setattr(s, k, scene_t[k].data_ptr() if n > 0 else None)
    sky = scene_t.get("sky")
    if sky is not None:
        if (sky.dim() != 4 or sky.shape[0] != 6 or sky.shape[1] != sky.shape[2] or sky.shape[3] != 3
                or sky.dtype != torch.float32 or not sky.is_contiguous() or not sky.is_cuda):
            raise ValueError("scene['sky'] must be a contiguous float32 CUDA tensor [6, R, R, 3]")
        s.sky = sky.data_ptr()
        s.sky_res = int(sky.shape[1])
    sem = scene_t.get("sem")
    if sem is not None:
        if (sem.dim() != 2 or sem.shape[0] != n or not 1 <= sem.shape[1] <= abi.MAX_SEM
                or sem.dtype != torch.float32 or not sem.is_contiguous() or not sem.is_cuda):
            raise ValueError("scene['sem'] must be a contiguous float32 CUDA tensor [N, S], 1 <= S <= %d"
                             % abi.MAX_SEM)
        s.sem = sem.data_ptr() if n > 0 else None
        s.n_sem = int(sem.shape[1])
    return s


def feat_count(features, n_sem=0):
    """Channels of the extra-channel image for a FEAT_* mask."""
    return ((3 if features & abi.FEAT_VBAR else 0) + (1 if features & abi.FEAT_RHO else 0)
            + (n_sem if features & abi.FEAT_SEM else 0))


def _fill_images(imgs, outs, features):
    for k, o in enumerate(outs):
        imgs[k].rgb = o["rgb"].data_ptr()
        imgs[k].depth = o["depth"].data_ptr() if o.get("depth") is not None else None
        imgs[k].alpha = o["alpha"].data_ptr() if o.get("alpha") is not None else None
        if features:
            if o.get("feat") is None:
                raise ValueError("features requested: every output needs a 'feat' tensor [F, H, W]")
            imgs[k].feat = o["feat"].data_ptr()
            imgs[k].feat_mask = int(features)


def _stream_ptr(stream=None):
    st = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(st.cuda_stream)


class Renderer:
    """Owns one ``pvg_ctx_t`` (workspace) on the current CUDA device."""

    def __init__(self, tile=(16, 16), sync_sizes=True, pair_capacity=1 << 24, dilation=0.3, fov_clamp=1.3,
                 pixels_per_thread=1):
        self._lib = abi.lib()
        self.cfg = abi.config(tile, sync_sizes, pair_capacity, dilation, fov_clamp, pixels_per_thread)
        h = C.c_void_p()
        abi.check(self._lib.pvg_create(C.byref(h), C.byref(self.cfg)), "pvg_create")
        self.handle = h
        self.device = torch.cuda.current_device()

    def close(self):
        if self.handle:
            self._lib.pvg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tile(self, tile, pixels_per_thread=None):
        self.cfg.tile_w, self.cfg.tile_h = int(tile[0]), int(tile[1])
        if pixels_per_thread is not None:
            self.cfg.pixels_per_thread = int(pixels_per_thread)
        abi.check(self._lib.pvg_set_config(self.handle, C.byref(self.cfg)), "pvg_set_config")

    def alloc_images(self, cams, device="cuda", features=0, n_sem=0):
        outs = []
        F = feat_count(features, n_sem)
        for cam in cams:
            H, W = int(cam["height"]), int(cam["width"])
            o = dict(rgb=torch.empty(3, H, W, device=device), depth=torch.empty(H, W, device=device),
                     alpha=torch.empty(H, W, device=device))
            if F:
                o["feat"] = torch.empty(F, H, W, device=device)
            outs.append(o)
        return outs

    def forward(self, scene_t, cams, outs=None, frame=None, stream=None, features=0):
        """Render into ``outs`` (list of dicts rgb [3,H,W], depth, alpha and,
        with ``features`` (a mask of abi.FEAT_*), feat [F,H,W]); returns
        ``outs``.  ``frame`` (a :class:`Frame`) keeps the state the backward
        pass needs."""
        if outs is None:
            sem = scene_t.get("sem")
            outs = self.alloc_images(cams, features=features, n_sem=0 if sem is None else int(sem.shape[1]))
        sc = abi_scene(scene_t)
        ca = abi.cameras(cams)
        imgs = (abi.Image * len(cams))()
        _fill_images(imgs, outs, features)
        st = self._lib.pvg_render_fwd(self.handle, C.byref(sc), ca, len(cams), imgs,
                                      frame.handle if frame is not None else None, _stream_ptr(stream))
        abi.check(st, "pvg_render_fwd")
        return outs

    def backward(self, scene_t, cams, frame, grads_out, stream=None, grads=None):
        """dL/d(images) ``grads_out`` (list of dicts, entries may be None) ->
        dict of parameter gradients (allocated if ``grads`` is None).
        ``frame`` is the :class:`Frame` the forward pass filled."""
        if frame is None:
            raise ValueError("backward needs the Frame that its forward pass filled")
        sc = abi_scene(scene_t)
        ca = abi.cameras(cams)
        if grads is None:
            grads = {k: torch.empty_like(scene_t[k]) for k in PARAM_NAMES}
            if scene_t.get("sky") is not None:
                grads["sky"] = torch.empty_like(scene_t["sky"])
            if scene_t.get("sem") is not None:
                grads["sem"] = torch.zeros_like(scene_t["sem"])
        g = abi.SceneGrad()
        for k in PARAM_NAMES + ("sky", "sem"):
            setattr(g, k, grads[k].data_ptr() if (grads.get(k) is not None and grads[k].numel()) else None)
        dl = (abi.ImageGrad * len(cams))()
        for k, d in enumerate(grads_out):
            for name in ("rgb", "depth", "alpha", "feat"):
                t = d.get(name)
                setattr(dl[k], name, t.contiguous().data_ptr() if t is not None else None)
        st = self._lib.pvg_render_bwd(self.handle, C.byref(sc), ca, len(cams), frame.handle, dl, C.byref(g),
                                      _stream_ptr(stream))
        abi.check(st, "pvg_render_bwd")
        return grads


class Frame:
    """Saved state of one forward pass (``pvg_frame_t``)."""

    def __init__(self):
        self._lib = abi.lib()
        h = C.c_void_p()
        abi.check(self._lib.pvg_frame_create(C.byref(h)), "pvg_frame_create")
        self.handle = h

    def close(self):
        if self.handle:
            self._lib.pvg_frame_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self):
        m, k, ov = C.c_int64(), C.c_int64(), C.c_int32()
        abi.check(self._lib.pvg_frame_stats(self.handle, C.byref(m), C.byref(k), C.byref(ov)), "pvg_frame_stats")
        return int(m.value), int(k.value), int(ov.value)

    def export(self, total_tiles):
        """Device intermediates of the last forward as CPU numpy arrays."""
        m, k, _ = self.stats()
        dev = torch.device("cuda", torch.cuda.current_device())
        sg = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        zk = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
        rect = torch.empty(max(m, 1), 4, dtype=torch.int32, device=dev)
        rec = torch.empty(max(m, 1), 12, dtype=torch.float32, device=dev)
        pv = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
        rg = torch.empty(max(total_tiles, 1), 2, dtype=torch.int32, device=dev)
        abi.check(self._lib.pvg_frame_export(self.handle, sg.data_ptr(), zk.data_ptr(), rect.data_ptr(),
                                             rec.data_ptr(), pv.data_ptr(), rg.data_ptr()), "pvg_frame_export")
        u32 = lambda t, n: t.cpu().numpy().view(np.uint32)[:n].copy()
        return dict(sorted_gid=u32(sg, m), depth_key=u32(zk, m), rect=rect.cpu().numpy()[:m],
                    records=rec.cpu().numpy()[:m], pair_vals=u32(pv, k),
                    ranges=rg.cpu().numpy().view(np.uint32)[:total_tiles].copy())


def tiles_of(cam, tile=(16, 16)):
    tw, th = tile
    return (int(cam["width"]) + tw - 1) // tw, (int(cam["height"]) + th - 1) // th


_DEFAULT = {}


def default_renderer():
    dev = torch.cuda.current_device()
    if dev not in _DEFAULT:
        _DEFAULT[dev] = Renderer()
    return _DEFAULT[dev]


def render(scene_t, cams, renderer=None, frame=None, features=0):
    """Render a list of cameras; returns a list of dicts (rgb, depth, alpha
    and, for a FEAT_* mask ``features``, feat)."""
    r = renderer or default_renderer()
    return r.forward(scene_t, cams, frame=frame, features=features)


class PVGRender(torch.autograd.Function):
    """images = Render({H_i(t)}; E, I) (Sec. 3.2, Eq. 8) for one camera,
    differentiable w.r.t. all nine parameter arrays and the optional sky
    cube map (Sec. 3.4)."""

    @staticmethod
    def forward(ctx, cam, renderer, mu, vel, tau, beta, period, scale, quat, opacity, sh, sky=None):
        scene_t = dict(mu=mu.contiguous(), vel=vel.contiguous(), tau=tau.contiguous(), beta=beta.contiguous(),
                       period=period.contiguous(), scale=scale.contiguous(), quat=quat.contiguous(),
                       opacity=opacity.contiguous(), sh=sh.contiguous())
        if sky is not None:
            scene_t["sky"] = sky.contiguous()
        frame = Frame()
        out = renderer.forward(scene_t, [cam], frame=frame)[0]
        ctx.cam, ctx.renderer, ctx.frame = cam, renderer, frame
        ctx.has_sky = sky is not None
        ctx.save_for_backward(*[scene_t[k] for k in PARAM_NAMES], *([scene_t["sky"]] if sky is not None else []))
        return out["rgb"], out["depth"], out["alpha"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha):
        saved = ctx.saved_tensors
        scene_t = dict(zip(PARAM_NAMES, saved))
        if ctx.has_sky:
            scene_t["sky"] = saved[len(PARAM_NAMES)]
        grads = ctx.renderer.backward(scene_t, [ctx.cam], ctx.frame,
                                      [dict(rgb=g_rgb, depth=g_depth, alpha=g_alpha)])
        ctx.frame.close()
        return (None, None) + tuple(grads[k] for k in PARAM_NAMES) + (grads.get("sky"),)


def render_differentiable(params, cam, renderer=None):
    """params: dict of tensors (may require grad; an optional "sky" cube map
    [6, R, R, 3]).  Returns rgb, depth, alpha."""
    r = renderer or default_renderer()
    return PVGRender.apply(cam, r, *[params[k] for k in PARAM_NAMES], params.get("sky"))


def flat_gradients(scene_t):
    """(flat, grads): one float32 buffer and the per-parameter gradient
    tensors (shaped like ``scene_t``'s nine parameter arrays) as views of
    it, ready for :meth:`Renderer.backward` and a single all-reduce."""
    n = sum(scene_t[k].numel() for k in PARAM_NAMES)
    flat = torch.empty(n, dtype=torch.float32, device=scene_t["mu"].device)
    grads, o = {}, 0
    for k in PARAM_NAMES:
        t = scene_t[k]
        grads[k] = flat[o:o + t.numel()].view(t.shape)
        o += t.numel()
    return flat, grads


def allreduce_gradients(flat, group=None):
    """Sums a flat gradient buffer over the ranks of ``group`` in place (the
    exchange step of data-parallel training: every rank renders its own
    views of the shared scene and the per-Gaussian gradients are added).
    Uses the process group's backend (NCCL on GPUs, gloo on CPU)."""
    import torch.distributed as dist

    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    return flat


def l1_loss(renderer, pred, target, dl=None, loss=None, scale=None, stream=None):
    """loss = scale * sum|pred - target| (default scale = 1/numel) and
    dl = scale * sign(pred - target), computed by ``pvg_l1_loss`` with the
    renderer's workspace (fixed-order sum: bit-reproducible)."""
    if pred.shape != target.shape or not pred.is_contiguous() or not target.is_contiguous():
        raise ValueError("pred and target must be contiguous tensors of one shape")
    n = pred.numel()
    if dl is None:
        dl = torch.empty_like(pred)
    if loss is None:
        loss = torch.empty(1, device=pred.device, dtype=torch.float32)
    s = 1.0 / max(n, 1) if scale is None else float(scale)
    st = abi.lib().pvg_l1_loss(renderer.handle, pred.data_ptr(), target.data_ptr(), n, s, dl.data_ptr(),
                              loss.data_ptr(), _stream_ptr(stream))
    abi.check(st, "pvg_l1_loss")
    return loss, dl


def rgb_loss(renderer, pred, target, lambda_r=0.2, dl=None, loss=None, stream=None):
    """(1 - lambda_r) L1 + lambda_r (1 - SSIM) of planar [C, H, W] images
    (``pvg_rgb_loss``); returns (loss [3] = (L, L1, SSIM), dL/dpred)."""
    if (pred.shape != target.shape or pred.dim() != 3 or not pred.is_contiguous() or not target.is_contiguous()
            or pred.dtype != torch.float32 or target.dtype != torch.float32):
        raise ValueError("pred and target must be contiguous float32 tensors [C, H, W] of one shape")
    if dl is None:
        dl = torch.empty_like(pred)
    if loss is None:
        loss = torch.empty(3, device=pred.device, dtype=torch.float32)
    C_, H, W = pred.shape
    st = abi.lib().pvg_rgb_loss(renderer.handle, pred.data_ptr(), target.data_ptr(), int(C_), int(H), int(W),
                               float(lambda_r), dl.data_ptr(), loss.data_ptr(), _stream_ptr(stream))
    abi.check(st, "pvg_rgb_loss")
    return loss, dl


def kernel_launches() -> int:
    return int(abi.lib().pvg_kernel_launches())


def device_sm_count() -> int:
    """SM count of the current device, as the library sizes its grids."""
    return int(abi.lib().pvg_device_sm_count())


def fma_probe(dst, blocks, iters, a=0.9999, b=1e-3, stream=None):
    """Launches the FP32 throughput probe (``pvg_fma_probe``): blocks x 256
    threads x iters x 128 lane FMAs; dst holds blocks * 256 floats."""
    if dst.numel() < blocks * 256 or dst.dtype != torch.float32 or not dst.is_cuda:
        raise ValueError("dst must be a CUDA float32 tensor of blocks * 256 elements")
    abi.check(abi.lib().pvg_fma_probe(dst.data_ptr(), int(blocks), int(iters), float(a), float(b),
                                      _stream_ptr(stream)), "pvg_fma_probe")
    return int(blocks) * 256 * int(iters) * 128


def profile_enable(renderer, on=True):
    abi.check(abi.lib().pvg_profile_enable(renderer.handle, 1 if on else 0), "pvg_profile_enable")


def profile_read(renderer):
    """{stage: (total ms, calls)} since the last read (synchronises)."""
    ms = (C.c_double * 8)()
    calls = (C.c_int64 * 8)()
    abi.check(abi.lib().pvg_profile_read(renderer.handle, ms, calls), "pvg_profile_read")
    return {name: (float(ms[k]), int(calls[k])) for k, name in enumerate(abi.STAGES)}


def eval_count(renderer, frame):
    """(E, blended): list entries each pixel evaluated inside their footprint
    box up to its stop, and how many of them had alpha >= 1/255."""
    e, b = C.c_int64(), C.c_int64()
    abi.check(abi.lib().pvg_frame_eval_count(renderer.handle, frame.handle, C.byref(e), C.byref(b)),
              "pvg_frame_eval_count")
    return int(e.value), int(b.value)


def sort_pairs(renderer, keys, vals, begin_bit=0, end_bit=32, stream=None):
    """Stable in-place radix sort of int32/uint32 CUDA tensors ``keys`` /
    ``vals`` by key bits [begin_bit, end_bit) (``pvg_sort_pairs``)."""
    if keys.shape != vals.shape or keys.dim() != 1 or not keys.is_contiguous() or not vals.is_contiguous():
        raise ValueError("keys and vals must be contiguous 1-D tensors of one length")
    st = abi.lib().pvg_sort_pairs(renderer.handle, keys.data_ptr(), vals.data_ptr(), keys.numel(), int(begin_bit),
                                  int(end_bit), _stream_ptr(stream))
    abi.check(st, "pvg_sort_pairs")
    return keys, vals


def render_multi(renderer, scenes, cams, outs=None, frame=None, stream=None):
    """View v renders scenes[v] (``pvg_render_fwd_multi``); scenes may repeat."""
    if len(scenes) != len(cams):
        raise ValueError("one scene per camera")
    if outs is None:
        outs = renderer.alloc_images(cams)
    sc = (abi.Scene * len(cams))()
    for k, s in enumerate(scenes):
        sc[k] = abi_scene(s)
    ca = abi.cameras(cams)
    imgs = (abi.Image * len(cams))()
    _fill_images(imgs, outs, 0)
    st = abi.lib().pvg_render_fwd_multi(renderer.handle, sc, ca, len(cams), imgs,
                                        frame.handle if frame is not None else None, _stream_ptr(stream))
    abi.check(st, "pvg_render_fwd_multi")
    return outs

"""Batched rendering: many views of one scene, with uneven sizes and their
own times t, rendered (and optionally differentiated) as one CUDA graph.

Every view goes through one launch sequence (the views share the depth
sort and the tile sort; tile ids are global over the views), and the whole
sequence -- forward, L1 loss against per-view targets, backward -- is
captured once into a ``torch.cuda.CUDAGraph`` and replayed.  Capture needs
fixed sizes: the batch is first rendered uncaptured with the pair count
read back, the pair capacity is set from it (with headroom), and the
context runs without host round trips (``sync_sizes = 0``); an overflow is
reported by :meth:`BatchGraph.overflowed`.  The compositing configuration
may be picked by the autotuner beforehand (it does not change the images).
"""
from __future__ import annotations

import torch

from . import render as R
from . import tune as T


class BatchGraph:
    """``host_targets``: optional pinned host tensors, one per view; the
    graph then copies them into the device targets on a side stream that
    runs beside the forward pass and joins before the loss, so a training
    loop writes each step's targets into those host buffers and replays."""

    def __init__(self, scene_t, cams, targets=None, backward=True, config=None, autotune=True,
                 headroom=1.25, stream=None, tune_configs=T.CONFIGS, host_targets=None):
        self.scene_t = scene_t
        self.cams = list(cams)
        self.backward = backward
        if config is None:
            config = (T.tune(scene_t, self.cams, backward=backward, use_cache=False, configs=tune_configs)[0]
                      if autotune else (16, 16, 1))
        self.config = tuple(config)
        tw, th, px = self.config
        # measure the pair count once with a size read-back
        probe = R.Renderer(tile=(tw, th), pixels_per_thread=px)
        pf = R.Frame()
        probe.forward(scene_t, self.cams, frame=pf)
        _, K, _ = pf.stats()
        pf.close()
        probe.close()
        self.pair_capacity = max(1024, int(K * headroom))
        self.r = R.Renderer(tile=(tw, th), pixels_per_thread=px, sync_sizes=False,
                            pair_capacity=self.pair_capacity)
        self.frame = R.Frame()
        self.outs = self.r.alloc_images(self.cams)
        dev = scene_t["mu"].device
        if backward:
            self.targets = targets if targets is not None else [torch.rand_like(o["rgb"]) for o in self.outs]
            self.dls = [torch.empty_like(o["rgb"]) for o in self.outs]
            self.losses = torch.zeros(len(self.cams), device=dev)
            self.grads = {k: torch.empty_like(scene_t[k]) for k in R.PARAM_NAMES}
        self.host_targets = None
        if host_targets is not None:
            if not backward or len(host_targets) != len(self.cams):
                raise ValueError("host_targets: one pinned host tensor per view, with backward=True")
            for h, t in zip(host_targets, self.targets):
                if h.device.type != "cpu" or not h.is_pinned() or h.shape != t.shape or h.dtype != t.dtype:
                    raise ValueError("host_targets must be pinned CPU tensors shaped like the targets")
            self.host_targets = list(host_targets)
            self.copy_stream = torch.cuda.Stream(device=dev)
        self.stream = stream or torch.cuda.Stream(device=dev)
        self.graph = None
        # uncaptured run: allocates every buffer at its final size
        with torch.cuda.stream(self.stream):
            self._enqueue()
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._enqueue()
        torch.cuda.synchronize()

    def _enqueue(self):
        if self.host_targets is not None:  # target copies beside the forward pass
            cur = torch.cuda.current_stream()
            self.copy_stream.wait_stream(cur)
            with torch.cuda.stream(self.copy_stream):
                for t, h in zip(self.targets, self.host_targets):
                    t.copy_(h, non_blocking=True)
        self.r.forward(self.scene_t, self.cams, outs=self.outs, frame=self.frame)
        if self.host_targets is not None:
            torch.cuda.current_stream().wait_stream(self.copy_stream)
        if self.backward:
            for v, o in enumerate(self.outs):
                R.l1_loss(self.r, o["rgb"], self.targets[v], dl=self.dls[v], loss=self.losses[v:v + 1])
            self.r.backward(self.scene_t, self.cams, self.frame, [dict(rgb=d) for d in self.dls], grads=self.grads)

    def replay(self):
        self.graph.replay()

    def overflowed(self) -> bool:
        return self.frame.stats()[2] != 0

    @property
    def pixels(self) -> int:
        return sum(int(c["width"]) * int(c["height"]) for c in self.cams)

"""Python side of the render server (``pvg_serve_*`` in include/pvg.h).

Marshalling only: the queue, the batching workers and every kernel are in
the CUDA library.  A :class:`Server` keeps references to the scene tensors
it was given so they outlive it.
"""
from __future__ import annotations

import ctypes as C

from . import abi
from .render import abi_scene


class Server:
    def __init__(self, max_batch_views=16, n_streams=4, memory_budget=8 << 30, max_pending=4096, tile=(16, 16),
                 pixels_per_thread=1, gate_timeout_us=1_000_000, pipeline_depth=1, pair_capacity=0):
        self._lib = abi.lib()
        c = abi.ServeConfig()
        self._lib.pvg_serve_config_default(C.byref(c))
        c.max_batch_views = int(max_batch_views)
        c.n_streams = int(n_streams)
        c.memory_budget = int(memory_budget)
        c.max_pending = int(max_pending)
        c.tile_w, c.tile_h = int(tile[0]), int(tile[1])
        c.pixels_per_thread = int(pixels_per_thread)
        c.gate_timeout_us = int(gate_timeout_us)
        c.pipeline_depth = int(pipeline_depth)
        c.pair_capacity = int(pair_capacity)
        h = C.c_void_p()
        abi.check(self._lib.pvg_serve_create(C.byref(h), C.byref(c)), "pvg_serve_create")
        self.handle = h
        self._scenes = []
        self._outs = {}

    def add_scene(self, scene_t) -> int:
        sid = C.c_int32()
        abi.check(self._lib.pvg_serve_add_scene(self.handle, C.byref(abi_scene(scene_t)), C.byref(sid)),
                  "pvg_serve_add_scene")
        self._scenes.append(scene_t)
        return int(sid.value)

    def submit(self, scene_id, cam, out):
        """Queue a request; ``out`` = dict(rgb=[3,H,W] tensor, depth=None|[H,W],
        alpha=None|[H,W]).  Returns the request id or raises PVGError (BUSY
        when the queue is full)."""
        img = abi.Image()
        img.rgb = out["rgb"].data_ptr()
        img.depth = out["depth"].data_ptr() if out.get("depth") is not None else None
        img.alpha = out["alpha"].data_ptr() if out.get("alpha") is not None else None
        rid = C.c_uint64()
        st = self._lib.pvg_serve_submit(self.handle, int(scene_id), C.byref(abi.camera(cam)), C.byref(img),
                                        C.byref(rid))
        abi.check(st, "pvg_serve_submit")
        self._outs[int(rid.value)] = out
        return int(rid.value)

    @staticmethod
    def _stats(s):
        return dict(submit_ms=s.submit_ms, start_ms=s.start_ms, done_ms=s.done_ms, batch_views=s.batch_views,
                    status=s.status, gpu_ms=s.gpu_ms, attempts=s.attempts)

    def poll(self, rid):
        done, s = C.c_int32(), abi.ReqStats()
        abi.check(self._lib.pvg_serve_poll(self.handle, C.c_uint64(rid), C.byref(done), C.byref(s)), "pvg_serve_poll")
        return bool(done.value), self._stats(s)

    def wait(self, rid, timeout_s=60.0):
        s = abi.ReqStats()
        st = self._lib.pvg_serve_wait(self.handle, C.c_uint64(rid), float(timeout_s * 1e3), C.byref(s))
        abi.check(st, "pvg_serve_wait")
        return self._stats(s)

    def release(self, rid):
        abi.check(self._lib.pvg_serve_release(self.handle, C.c_uint64(rid)), "pvg_serve_release")
        self._outs.pop(rid, None)

    def counters(self):
        q, b, v, m = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        abi.check(self._lib.pvg_serve_counters(self.handle, C.byref(q), C.byref(b), C.byref(v), C.byref(m)),
                  "pvg_serve_counters")
        return dict(queued=q.value, batches=b.value, views=v.value, in_flight_bytes=m.value)

    def arena(self):
        """Requeues so far and the per-worker arena: Gaussians, pixels and
        pairs per batch, and the free device memory measured at creation."""
        v = [C.c_int64() for _ in range(5)]
        abi.check(self._lib.pvg_serve_arena(self.handle, *[C.byref(x) for x in v]), "pvg_serve_arena")
        return dict(zip(("requeues", "items_per_batch", "pixels_per_batch", "pairs_per_batch", "free_bytes"),
                        (x.value for x in v)))

    def debug_withhold(self, n):
        """Test hook: the next n submitted requests are never published in
        the ring, so the gather kernel's bounded wait runs out for them."""
        abi.check(self._lib.pvg_serve_debug_withhold(self.handle, int(n)), "pvg_serve_debug_withhold")

    def close(self):
        if self.handle:
            self._lib.pvg_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

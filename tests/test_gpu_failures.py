"""Failure handling, tested without faulting the GPU: bad arguments come
back as PVG_ERR_INVALID before anything is enqueued, injected allocation
failures (pvg_debug_fail_allocations) come back as PVG_ERR_OOM and the next
call recovers, the render server marks the requests of a failed launch with
that status and keeps serving, and a bounded wait on an unfinished request
returns PVG_ERR_TIMEOUT.  GPU only."""
import math

import numpy as np
import pytest
import torch

from paper_2311_18561_gb300 import abi
from paper_2311_18561_gb300 import render as R
from paper_2311_18561_gb300 import serve as S
from paper_2311_18561_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

INVALID, OOM, TIMEOUT = 1, 2, 4


@pytest.fixture(autouse=True)
def _clear_hook():
    yield
    abi.lib().pvg_debug_fail_allocations(0)


def _status(fn):
    with pytest.raises(abi.PVGError) as e:
        fn()
    return e.value.status


def _done_status(srv, rid, limit_s=60.0):
    """Status of a finished request (polling: wait() raises on a failed launch)."""
    import time

    t0 = time.time()
    while time.time() - t0 < limit_s:
        done, st = srv.poll(rid)
        if done:
            return st["status"]
        time.sleep(0.001)
    raise AssertionError("request did not finish")


def test_bad_arguments_are_rejected():
    st = R.scene_to_device(synth.make_plain_scene(seed=0, n=200))
    r = R.Renderer()
    good = synth.plain_camera(64, 48)
    for bad in (dict(good, width=0), dict(good, height=-3), dict(good, fx=float("nan")),
                dict(good, t=math.inf), dict(good, z_near=-1.0), dict(good, dt=float("nan")),
                dict(good, viewmat=np.full((3, 4), np.nan, np.float32))):
        outs = r.alloc_images([good])  # right-sized buffers: only the camera is wrong
        assert _status(lambda: r.forward(st, [bad], outs=outs)) == INVALID
    # the renderer is still usable
    out = r.forward(st, [good])[0]
    torch.cuda.synchronize()
    assert torch.isfinite(out["rgb"]).all()


def test_backward_without_saved_state_is_rejected():
    st = R.scene_to_device(synth.make_plain_scene(seed=0, n=200))
    cam = synth.plain_camera(64, 48)
    r = R.Renderer()
    r.forward(st, [cam])  # inference only: no frame, no state for a backward pass

    class _NoFrame:
        handle = None

    dl = [dict(rgb=torch.ones(3, 48, 64, device="cuda"))]
    assert _status(lambda: r.backward(st, [cam], _NoFrame(), dl)) == INVALID
    # with a frame the same call works
    fr = R.Frame()
    r.forward(st, [cam], frame=fr)
    g = r.backward(st, [cam], fr, dl)
    torch.cuda.synchronize()
    assert torch.isfinite(g["mu"]).all() and g["mu"].abs().sum().item() > 0


def test_empty_scene_renders_the_background():
    scene = {k: v[:0] for k, v in synth.make_plain_scene(seed=0, n=4).items()}
    st = R.scene_to_device(scene)
    cam = synth.plain_camera(40, 30, bg=(0.25, 0.5, 0.75))
    out = R.Renderer().forward(st, [cam])[0]
    torch.cuda.synchronize()
    expect = torch.tensor([0.25, 0.5, 0.75], device="cuda").view(3, 1, 1).expand(3, 30, 40)
    assert torch.equal(out["rgb"], expect) and out["alpha"].abs().max().item() == 0.0


def test_allocation_failure_is_reported_and_the_next_call_recovers():
    st = R.scene_to_device(synth.make_plain_scene(seed=1, n=2000))
    cam = synth.plain_camera(160, 120)
    ref = R.Renderer().forward(st, [cam])[0]["rgb"].clone()
    r = R.Renderer()  # fresh workspace: its first forward must allocate
    abi.lib().pvg_debug_fail_allocations(1)
    assert _status(lambda: r.forward(st, [cam])) == OOM
    out = r.forward(st, [cam])[0]
    torch.cuda.synchronize()
    assert torch.equal(out["rgb"], ref)


def test_server_survives_allocation_failures():
    scenes = [R.scene_to_device(synth.make_urban_scene(20_000, seed=3))]
    # a 1 MiB budget reserves almost no arena: every first request of a size
    # grows the worker's workspace while serving
    srv = S.Server(max_batch_views=1, n_streams=1, memory_budget=1 << 20)
    sid = srv.add_scene(scenes[0])
    cams = [synth.street_camera(0.1 * k, 248, 75) for k in range(6)]
    abi.lib().pvg_debug_fail_allocations(2)  # the worker's first launches cannot grow their workspace
    outs = [dict(rgb=torch.empty(3, 75, 248, device="cuda")) for _ in cams]
    rids = [srv.submit(sid, c, o) for c, o in zip(cams, outs)]
    statuses = [_done_status(srv, rid) for rid in rids]
    assert OOM in statuses, statuses
    assert statuses[-1] == 0, statuses  # later launches succeed
    abi.lib().pvg_debug_fail_allocations(0)
    # and the server still renders what a direct call renders
    for k, (c, o) in enumerate(zip(cams, outs)):
        o2 = dict(rgb=torch.empty(3, 75, 248, device="cuda"))
        assert _done_status(srv, srv.submit(sid, c, o2)) == 0
        ref = R.Renderer().forward(scenes[0], [c])[0]["rgb"]
        torch.cuda.synchronize()
        assert torch.equal(o2["rgb"], ref)
        if statuses[k] == 0:
            assert torch.equal(o["rgb"], ref)
    srv.close()


def test_bounded_wait_times_out_then_completes():
    scene = R.scene_to_device(synth.make_urban_scene(300_000, seed=4))
    srv = S.Server(max_batch_views=1, n_streams=1)
    sid = srv.add_scene(scene)
    cam = synth.street_camera(0.5, 1920, 1280)
    out = dict(rgb=torch.empty(3, 1280, 1920, device="cuda"))
    rid = srv.submit(sid, cam, out)
    assert _status(lambda: srv.wait(rid, 0.0)) == TIMEOUT
    st = srv.wait(rid, 60.0)
    assert st["status"] == 0
    srv.close()

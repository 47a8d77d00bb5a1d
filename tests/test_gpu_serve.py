"""The render server (pvg_serve_*): continuous batching over several
resident scenes with requests of mixed resolution, time and pose.  Each
request's image is bit-identical alone and in the mix, and equals a direct
pvg_render_fwd call; the memory budget limits batches; a full queue
answers BUSY; the gather kernel's bounded wait for an unpublished ring slot
runs out with PVG_ERR_TIMEOUT while the server goes on; a pair count above
a batch's reservation requeues its requests; the arenas follow the free
device memory.  GPU only."""
import numpy as np
import pytest
import torch

from paper_2311_18561_gb300 import abi
from paper_2311_18561_gb300 import render as R
from paper_2311_18561_gb300 import serve as S
from paper_2311_18561_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

RES = ((160, 120), (248, 75), (384, 256))


def _scenes():
    return [R.scene_to_device(synth.make_urban_scene(n, seed=20 + k)) for k, n in enumerate((20_000, 40_000,
                                                                                              80_000))]


def _requests(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        sid = int(rng.integers(0, 3))
        w, h = RES[int(rng.integers(0, len(RES)))]
        t = float(rng.uniform(0, 1))
        out.append((sid, synth.street_camera(t, w, h, lateral=float(rng.uniform(-2, 2)))))
    return out


def _out(cam):
    return dict(rgb=torch.empty(3, cam["height"], cam["width"], device="cuda"),
                depth=torch.empty(cam["height"], cam["width"], device="cuda"),
                alpha=torch.empty(cam["height"], cam["width"], device="cuda"))


def test_each_request_is_identical_alone_and_in_the_mix():
    scenes = _scenes()
    reqs = _requests(24)
    srv = S.Server(max_batch_views=8, n_streams=2)
    ids = [srv.add_scene(s) for s in scenes]
    # alone: one request at a time
    alone = []
    for sid, cam in reqs:
        o = _out(cam)
        rid = srv.submit(ids[sid], cam, o)
        st = srv.wait(rid, 30.0)
        assert st["batch_views"] == 1
        alone.append(o)
    # the mix: everything at once
    mixed, rids = [], []
    for sid, cam in reqs:
        o = _out(cam)
        rids.append(srv.submit(ids[sid], cam, o))
        mixed.append(o)
    sizes = [srv.wait(r, 60.0)["batch_views"] for r in rids]
    assert max(sizes) > 1, "no request was batched"
    for a, b in zip(alone, mixed):
        for k in ("rgb", "depth", "alpha"):
            assert torch.equal(a[k], b[k])
    # and equal to a direct render
    r = R.Renderer()
    for (sid, cam), a in zip(reqs, alone):
        d = r.forward(scenes[sid], [cam])[0]
        for k in ("rgb", "depth", "alpha"):
            assert torch.equal(a[k], d[k])
    srv.close()


def test_memory_budget_limits_batches():
    scenes = _scenes()
    srv = S.Server(max_batch_views=8, n_streams=1, memory_budget=1)  # nothing fits beside anything else
    ids = [srv.add_scene(s) for s in scenes]
    rids = []
    for sid, cam in _requests(10, seed=1):
        rids.append(srv.submit(ids[sid], cam, _out(cam)))
    for rid in rids:
        st = srv.wait(rid, 30.0)
        assert st["batch_views"] == 1 and st["status"] == 0
    srv.close()


def test_full_queue_answers_busy_and_everything_accepted_completes():
    scenes = _scenes()
    srv = S.Server(max_batch_views=1, n_streams=1, max_pending=1)
    sid = srv.add_scene(scenes[2])
    cam = synth.street_camera(0.5, 384, 256)
    accepted, busy = [], 0
    for _ in range(200):
        try:
            accepted.append(srv.submit(sid, cam, _out(cam)))
        except abi.PVGError as e:
            assert e.status == 3  # PVG_ERR_BUSY
            busy += 1
    assert busy > 0
    for rid in accepted:
        assert srv.wait(rid, 30.0)["status"] == 0
    srv.close()


def test_unknown_scene_and_request():
    srv = S.Server()
    cam = synth.street_camera(0.5, 64, 48)
    with pytest.raises(abi.PVGError) as e:
        srv.submit(3, cam, _out(cam))
    assert e.value.status == 7  # PVG_ERR_NOT_FOUND
    with pytest.raises(abi.PVGError) as e:
        srv.poll(12345)
    assert e.value.status == 7
    srv.close()


def test_unpublished_slot_times_out_on_the_device_and_the_server_goes_on():
    """The gather kernel waits (bounded, 20 ms here) for every slot of its
    batch; two requests whose slots are never published complete with
    PVG_ERR_TIMEOUT, the requests batched with them render normally, and so
    does everything after them."""
    scenes = _scenes()
    srv = S.Server(max_batch_views=8, n_streams=1, gate_timeout_us=20_000)
    ids = [srv.add_scene(s) for s in scenes]
    reqs = _requests(6, seed=3)
    srv.debug_withhold(2)
    outs, rids = [], []
    for sid, cam in reqs:
        o = _out(cam)
        rids.append(srv.submit(ids[sid], cam, o))
        outs.append(o)
    stats = []
    for rid in rids:
        try:
            srv.wait(rid, 30.0)
        except abi.PVGError as e:  # wait returns the request's status
            assert e.status == 4
        stats.append(srv.poll(rid)[1])
    assert [st["status"] for st in stats[:2]] == [4, 4]  # PVG_ERR_TIMEOUT
    assert all(st["status"] == 0 for st in stats[2:])
    assert stats[0]["gpu_ms"] >= 15.0  # the device waited out its bound
    r = R.Renderer()
    for (sid, cam), o, st in zip(reqs[2:], outs[2:], stats[2:]):
        d = r.forward(scenes[sid], [cam])[0]
        for k in ("rgb", "depth", "alpha"):
            assert torch.equal(o[k], d[k])
    for sid, cam in _requests(3, seed=4):
        o = _out(cam)
        assert srv.wait(srv.submit(ids[sid], cam, o), 30.0)["status"] == 0
        d = r.forward(scenes[sid], [cam])[0]
        assert torch.equal(o["rgb"], d["rgb"])
    srv.close()


def test_pair_count_above_the_reservation_requeues():
    """With 3,000 pairs per batch reserved, the GPU's pair count of the
    first batches exceeds the reservation: their requests go back to the
    queue with the measured density and are rendered again with a larger
    reservation, ending bit-identical to direct renders."""
    scenes = _scenes()
    srv = S.Server(max_batch_views=8, n_streams=1, pair_capacity=3000)
    ids = [srv.add_scene(s) for s in scenes]
    reqs = _requests(8, seed=5)
    outs = [_out(cam) for _, cam in reqs]
    rids = [srv.submit(ids[sid], cam, o) for (sid, cam), o in zip(reqs, outs)]
    stats = [srv.wait(rid, 60.0) for rid in rids]
    assert all(st["status"] == 0 for st in stats)
    assert max(st["attempts"] for st in stats) >= 2
    assert srv.arena()["requeues"] >= 1
    r = R.Renderer()
    for (sid, cam), o in zip(reqs, outs):
        d = r.forward(scenes[sid], [cam])[0]
        for k in ("rgb", "depth", "alpha"):
            assert torch.equal(o[k], d[k])
    srv.close()


def test_arenas_follow_the_free_device_memory():
    free, _ = torch.cuda.mem_get_info()
    srv = S.Server(n_streams=2, memory_budget=2 << 30)
    a = srv.arena()
    assert 0.5 * free <= a["free_bytes"] <= 1.5 * free
    budget = min(2 << 30, a["free_bytes"] // 10 * 9)
    assert a["items_per_batch"] == (budget // 2) * 45 // 100 // 204
    assert a["pixels_per_batch"] == (budget // 2) * 10 // 100 // 16
    srv.close()
    # a budget above the free memory is clamped to 90 % of it
    big = S.Server(n_streams=1, memory_budget=1 << 50, max_pending=16)
    b = big.arena()
    assert b["items_per_batch"] <= (b["free_bytes"] // 10 * 9) * 45 // 100 // 204
    big.close()

"""Batched views in one captured CUDA graph: the replayed graph produces the
same images and gradients as the uncaptured calls; views of uneven size
and time in one call equal the same views rendered one by one; the
multi-scene entry point equals per-scene calls.  GPU only."""
import numpy as np
import pytest
import torch

from paper_2311_18561_gb300 import batch as B
from paper_2311_18561_gb300 import render as R
from paper_2311_18561_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _cams():
    return [synth.street_camera(0.2, 320, 200), synth.street_camera(0.55, 248, 75, fx=144.0),
            synth.street_camera(0.8, 192, 128), synth.street_camera(0.41, 320, 200, lateral=1.0)]


def test_graph_replay_equals_uncaptured_calls():
    scene = synth.make_urban_scene(60_000, seed=3)
    st = R.scene_to_device(scene)
    cams = _cams()
    g = B.BatchGraph(st, cams, autotune=False, config=(16, 16, 2))
    g.replay()
    torch.cuda.synchronize()
    assert not g.overflowed()
    # reference: plain calls with a size read-back, same configuration
    r = R.Renderer(tile=(16, 16), pixels_per_thread=2)
    fr = R.Frame()
    outs = r.forward(st, cams, frame=fr)
    dls, losses = [], []
    for v, o in enumerate(outs):
        loss, dl = R.l1_loss(r, o["rgb"], g.targets[v])
        dls.append(dict(rgb=dl))
        losses.append(loss)
    grads = r.backward(st, cams, fr, dls)
    torch.cuda.synchronize()
    for v in range(len(cams)):
        for k in ("rgb", "depth", "alpha"):
            assert torch.equal(g.outs[v][k], outs[v][k]), (v, k)
    # gradients are summed with float atomics in no fixed order: equal up to
    # rounding, relative to each parameter group's scale
    for k in R.PARAM_NAMES:
        scale = float(grads[k].abs().max())
        assert float((g.grads[k] - grads[k]).abs().max()) <= 1e-4 * scale + 1e-12, k


def test_graph_replays_are_repeatable():
    scene = synth.make_urban_scene(40_000, seed=4)
    st = R.scene_to_device(scene)
    g = B.BatchGraph(st, _cams(), autotune=False, config=(16, 16, 1))
    g.replay()
    torch.cuda.synchronize()
    first = [o["rgb"].clone() for o in g.outs]
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for a, o in zip(first, g.outs):
        assert torch.equal(a, o["rgb"])


def test_graph_copies_host_targets_each_replay():
    """With pinned host targets the graph copies them in on every replay
    (beside the forward pass): new host values give the loss of those
    values, equal to the loss against device copies of them."""
    scene = synth.make_urban_scene(40_000, seed=6)
    st = R.scene_to_device(scene)
    cams = _cams()[:2]
    hosts = [torch.empty(3, int(c["height"]), int(c["width"])).pin_memory() for c in cams]
    g = B.BatchGraph(st, cams, autotune=False, config=(16, 16, 1), host_targets=hosts)
    r = R.Renderer()
    for trial in range(2):
        gen = torch.Generator().manual_seed(10 + trial)
        for h in hosts:
            h.copy_(torch.rand(h.shape, generator=gen))
        g.replay()
        torch.cuda.synchronize()
        for v, h in enumerate(hosts):
            assert torch.equal(g.targets[v].cpu(), h)
            loss, _ = R.l1_loss(r, g.outs[v]["rgb"], h.cuda())
            torch.cuda.synchronize()
            # the L1 sum is taken in a fixed order: the same value bit for bit
            assert float(loss[0]) == float(g.losses[v]), (trial, v)
    with pytest.raises(ValueError):
        B.BatchGraph(st, cams, autotune=False, config=(16, 16, 1), host_targets=[hosts[0]])


def test_uneven_views_in_one_call_equal_single_calls():
    scene = synth.make_urban_scene(50_000, seed=5)
    st = R.scene_to_device(scene)
    cams = _cams()
    r = R.Renderer()
    many = r.forward(st, cams)
    for v, cam in enumerate(cams):
        one = r.forward(st, [cam])[0]
        for k in ("rgb", "depth", "alpha"):
            assert torch.equal(many[v][k], one[k]), (v, k)


def test_multi_scene_call_equals_per_scene_calls():
    scenes = [R.scene_to_device(synth.make_urban_scene(n, seed=s)) for n, s in ((20_000, 1), (35_000, 2))]
    cams = _cams()[:3]
    which = [0, 1, 0]
    r = R.Renderer()
    many = R.render_multi(r, [scenes[w] for w in which], cams)
    for v, cam in enumerate(cams):
        one = r.forward(scenes[which[v]], [cam])[0]
        for k in ("rgb", "depth", "alpha"):
            assert torch.equal(many[v][k], one[k]), (v, k)


def test_graph_keeps_its_view_descriptors_after_later_calls_on_the_frame():
    """A captured forward replays with the cameras and images of its
    capture after a later capture and a later uncaptured call on the same
    frame with other cameras and images (each capture keeps its own copy of
    the view descriptors)."""
    scene = synth.make_urban_scene(40_000, seed=8)
    st = R.scene_to_device(scene)
    cams_a = _cams()[:2]
    cams_b = [synth.street_camera(0.7, 320, 200, lateral=-1.0), synth.street_camera(0.1, 248, 75, fx=144.0)]
    r = R.Renderer(sync_sizes=False, pair_capacity=1 << 22)
    fr = R.Frame()
    outs_a, outs_b, outs_c = r.alloc_images(cams_a), r.alloc_images(cams_b), r.alloc_images(cams_b)
    graphs = []
    for cams, outs in ((cams_a, outs_a), (cams_b, outs_b)):
        r.forward(st, cams, outs=outs, frame=fr)  # uncaptured first: buffers at their final sizes
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            r.forward(st, cams, outs=outs, frame=fr)
        graphs.append(g)
    ref_a = [o["rgb"].clone() for o in outs_a]
    ref_b = [o["rgb"].clone() for o in outs_b]
    for o in outs_a + outs_b:
        o["rgb"].zero_()
    r.forward(st, cams_b, outs=outs_c, frame=fr)
    graphs[1].replay()
    graphs[0].replay()
    torch.cuda.synchronize()
    for o, ref in zip(outs_a, ref_a):
        assert torch.equal(o["rgb"], ref)
    for o, ref in zip(outs_b, ref_b):
        assert torch.equal(o["rgb"], ref)
    assert not torch.equal(ref_a[0], ref_b[0])
    r.close()
    fr.close()

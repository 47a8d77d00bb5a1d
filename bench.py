#!/usr/bin/env python
"""Benchmark of the PVG rasterizer on one GB300 (or N replicas).

One step = one pass of the whole hot path over one synthetic frame: the
forward render (time evaluation, projection, depth + tile sort,
compositing), the L1 loss against a target image, and the backward pass
(compositing adjoint and chain rule to every PVG parameter).  Workload: the
urban scene of 1.5M Gaussians (SH degree 3) seen at 1920x1280 from frame
25 of the 50-frame street path.  ``value`` is whole-job Mpix/s of such
steps; the forward-only render rate is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 launch one process per GPU (torchrun): each rank renders its
own frame of the same scene (replicas, no collective on the data path).
``--impl reference`` times the FP64 CPU oracle on a bounded pixel sample of
the same workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "render Mpix/s & fwd+bwd step ms at 1.5M Gaussians 1920x1280; served p50/p99 latency"
FRAME = 25
# name: (Gaussians, width, height, focal or None (hfov 50 deg), description)
WORKLOADS = {
    "urban": (1_500_000, 1920, 1280, None,
              "urban scene, 1.5M Gaussians, SH-3, 1920x1280, street-path frame 25 (t=25/49): "
              "forward render + L1 loss + backward"),
    "training": (1_000_000, 1242, 375, 720.0,
                 "training config: urban-distribution scene, 1M Gaussians, SH-3, 1242x375 (f=720), "
                 "street-path frame 25: forward render + L1 loss + backward"),
}
N_GAUSS, W_PIX, H_PIX, FOCAL, WORKLOAD = WORKLOADS["urban"]


def select_workload(name):
    global N_GAUSS, W_PIX, H_PIX, FOCAL, WORKLOAD
    N_GAUSS, W_PIX, H_PIX, FOCAL, WORKLOAD = WORKLOADS[name]


def workload_camera(frame):
    from paper_2311_18561_gb300 import synth

    if FOCAL is None:
        return synth.urban_frame_camera(frame, W_PIX, H_PIX)
    return synth.street_camera(frame / 49.0, W_PIX, H_PIX, fx=FOCAL)


SM_MAX_MHZ = 2070.0  # nominal maximum SM clock (MEASURED_PEAKS.json's sm_max_mhz when present)
# Algorithmic FP32 lane-instructions of the compositor:
# every in-footprint evaluation: dy, the falloff exponent as two FFMA
# around the terms of the entry's pixel column (a' dx^2 and b' dx, shared
# by the column's pixels), o~ G, the 1/255 test, min(0.99, .) = 6;
# every blended evaluation in addition, forward: alpha T, T - alpha T, the
# stop test, 4 FFMA (r g b depth), O += w = 8; backward: 1 - alpha,
# T_i, w, X (4), dL/dalpha (2), colour and depth terms (4), opacity term,
# dL/dpower, 2 moments' bases, 5 moments, suffix sum = 23.
OPS_PER_LOSS_PIXEL = 207
OPS_PER_EVAL = 6
OPS_PER_BLEND = {"composite": 8, "composite_bwd": 23}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS) + ("batched", "serving"), default="urban")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", default="", help="tile_w,tile_h,pixels_per_thread (default: autotune)")
    ap.add_argument("--serve-rate", type=float, default=None,
                    help="request rate of a single serving leg (req/s; default: sweep 200, 500, 1000, 2000)")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="seconds of arrivals per serving rate (default 5 after the headline step, 10 for "
                         "--workload serving)")
    ap.add_argument("--dp", action="store_true",
                    help="with N > 1 ranks: data-parallel training step, the per-Gaussian gradients "
                         "summed over ranks in the step (default: independent replicas)")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the legs timed after the headline step: paper loss, extra channels, the "
                         "training (1M, 1242x375) and batched (3M, 64 views) configurations")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="wall-clock budget of the oracle's bounded sample")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_frame(rank):
    """Frame of the street path that replica `rank` renders (replicas only:
    every rank holds the whole scene and renders its own frame)."""
    return (FRAME + rank) % 50


def max_over_ranks(values, world, device):
    """Element-wise maximum of per-rank timings over the job (a job is as
    slow as its slowest replica); `world` = 1 returns them unchanged."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_value(world, mpix_per_rank, ms):
    """Whole-job throughput in Mpix/s: every rank renders mpix_per_rank per
    step, the step takes the slowest rank's `ms`."""
    return world * mpix_per_rank / (ms * 1e-3)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured", sm_max_mhz=float(d.get("sm_max_mhz", SM_MAX_MHZ)))
    except Exception:
        return dict(hbm_gbs=6800.0, source="fallback", sm_max_mhz=SM_MAX_MHZ)


def measure_fp32_peak(dev, seconds=1.2):
    """FP32 lane-FMA rate of the part, measured with the library's FMA probe
    (independent fused multiply-add chains, 2048 threads per SM), timed with
    CUDA events over about `seconds`; the best launch counts.  Returns the
    rate beside the SM count and the derived figure SMs x 128 lanes x the
    maximum SM clock."""
    import torch

    from paper_2311_18561_gb300 import render as R

    sms = R.device_sm_count()
    props_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 8 * sms
    dst = torch.empty(blocks * 256, device=dev)
    iters = 2000
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    R.fma_probe(dst, blocks, iters)  # warm-up
    torch.cuda.synchronize()
    best, total, launches = 0.0, 0.0, 0
    while total < seconds * 1e3 or launches < 5:
        a.record()
        lanes = R.fma_probe(dst, blocks, iters)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b)
        total += ms
        launches += 1
        best = max(best, lanes / (ms * 1e-3))
        if ms < 40.0:  # grow the launch to about 50 ms
            iters = int(iters * min(8.0, 50.0 / max(ms, 1e-3)))
    derived = sms * 128 * peaks()["sm_max_mhz"] * 1e6
    return {"lane_fma_per_s": best, "sm_count": sms, "sm_count_torch": props_sms, "launches": launches,
            "derived_lane_per_s": derived, "ratio_to_derived": best / derived,
            "how": "pvg_fma_probe: %d blocks x 256 threads, 8 independent FMA chains per thread, best of %d "
                   "launches of about 50 ms (CUDA events)" % (blocks, launches)}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms; start()
    returns once the first sample is written, so that the samples cover the
    region that follows."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t_end = time.time() + 5.0
        while time.time() < t_end and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return parse_clock_lines(lines)


def parse_clock_lines(lines):
    """The `clocks` summary of nvidia-smi samples (csv, noheader, nounits,
    the fields of ClockSampler.FIELDS): median SM clock over the samples
    under load (above half the highest), the maximum SM clock, and the
    slowdown reasons seen active; None without samples."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
    loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
    return {"sm_mhz": statistics.median(loaded) if loaded else None,
            "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


# the sources that decide the compositor kernels' memory traffic
COMPOSITOR_SOURCES = ("pvg_internal.cuh", "raster_common.cuh", "raster.cu", "raster_bwd.cu")


def kernel_source_hash(files=COMPOSITOR_SOURCES):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2311_18561_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, config):
    """DRAM bytes (read + write) per launch of `kernel` in compositing
    configuration `config` ("16x32x4") on the urban workload, from the
    committed ncu summary, if it was taken on the current kernel sources
    (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("source_hash") != kernel_source_hash():
            return None
        return d["kernels"][kernel][config]
    except Exception:
        return None


# --------------------------------------------------------------------------- shared timing helpers

def timed_steps(fn, steps, flush=None):
    """Per-step CUDA events around fn on the current stream (L2 flushed
    before each step, outside the events); returns the summed milliseconds."""
    import torch

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        if flush is not None:
            flush.zero_()
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def capture_graph(fn, dev):
    """fn's launches as one CUDA graph (its buffers are already sized) and
    the number of library kernels it holds."""
    import torch

    from paper_2311_18561_gb300 import render as R

    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    n0 = R.kernel_launches()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g, R.kernel_launches() - n0


def alu_roof(stage, stage_ms, E, B, fp32, traffic=None):
    """ALU roofline of a compositing stage: E in-footprint evaluations x 6
    + B blends x the stage's per-blend FP32 instructions, per launch, over
    the measured lane-FMA rate of the FMA probe."""
    ops = E * OPS_PER_EVAL + B * OPS_PER_BLEND[stage]
    ach = ops / (stage_ms[stage] * 1e-3)
    peak = fp32["lane_fma_per_s"]
    kern = "k_composite" if stage == "composite" else "k_composite_bwd"
    return {"kernel": kern, "bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12,
            "unit": "T FP32-lane-instr/s", "frac": ach / peak, "traffic": traffic,
            "work": "E=%d in-footprint evaluations x %d + %d blended x %d FP32 instructions"
                    % (E, OPS_PER_EVAL, B, OPS_PER_BLEND[stage]),
            "peak_kind": "measured (FMA probe)",
            "peak_source": "FP32 lane-FMA rate of the FMA probe in this run (%d SMs; %.1f T/s derived from "
                           "%d SMs x 128 lanes x %.0f MHz)" % (fp32["sm_count"], fp32["derived_lane_per_s"] / 1e12,
                                                              fp32["sm_count"], peaks()["sm_max_mhz"])}


def hbm_algo_bytes(stage, n_gauss, M, K):
    """Algorithmic bytes per launch of the HBM-bound stages."""
    return {"project": n_gauss * 68 + n_gauss * 8, "finalize": M * (68 + 192 + 48 + 8 + 4),
            "preprocess_bwd": M * (260 + 40 + 260) + (n_gauss - M) * 260, "depth_sort": M * 4 * 20,
            "pairs": M * 12 + K * 8, "tile_sort": K * 40}.get(stage, 0)


def dominant_roof(stage_ms, E, B, n_gauss, M, K, fp32, traffic=None):
    dominant = max(stage_ms, key=stage_ms.get)
    if dominant in ("composite", "composite_bwd"):
        return alu_roof(dominant, stage_ms, E, B, fp32, traffic)
    pk = peaks()
    b = hbm_algo_bytes(dominant, n_gauss, M, K)
    ach = b / (stage_ms[dominant] * 1e-3) / 1e9
    return {"kernel": dominant, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": ach / pk["hbm_gbs"], "traffic": None, "peak_kind": pk["source"]}


def stage_profile(r, fn, steps, flush=None):
    """Per-stage milliseconds (library event timer) per eager call of fn,
    summed over the library calls fn makes."""
    from paper_2311_18561_gb300 import render as R

    R.profile_enable(r, True)
    R.profile_read(r)
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        fn()
    stages = R.profile_read(r)
    R.profile_enable(r, False)
    return {k: v[0] / max(steps, 1) for k, v in stages.items()}


def tuned_step(dev, st, cams, targets, tile_arg="", tune_configs=None):
    """A renderer in the autotuned (or given) configuration whose pair
    capacity comes from one sized render (2x headroom), and its training
    step over `cams`: forward, L1 against `targets`, backward, never reading
    a size back (one CUDA graph)."""
    import torch

    from paper_2311_18561_gb300 import render as R

    if tile_arg:
        best, table = tuple(int(v) for v in tile_arg.split(",")), None
    else:
        from paper_2311_18561_gb300 import tune

        kw = {} if tune_configs is None else {"configs": tune_configs}
        best, table = tune.tune(st, cams, backward=True, use_cache=False, **kw)
    probe, pfr = R.Renderer(tile=best[:2], pixels_per_thread=best[2]), R.Frame()
    probe.forward(st, cams, frame=pfr)
    pair_capacity = max(1 << 20, 2 * pfr.stats()[1])
    probe.close()
    pfr.close()
    r = R.Renderer(tile=best[:2], pixels_per_thread=best[2], sync_sizes=False, pair_capacity=pair_capacity)
    fr = R.Frame()
    outs = r.alloc_images(cams)
    grad_flat, grads = R.flat_gradients(st)
    dls = [torch.empty_like(o["rgb"]) for o in outs]
    losses = torch.empty(len(cams), device=dev)

    def step():
        r.forward(st, cams, outs=outs, frame=fr)
        for v, o in enumerate(outs):
            R.l1_loss(r, o["rgb"], targets[v], dl=dls[v], loss=losses[v:v + 1])
        r.backward(st, cams, fr, [dict(rgb=d) for d in dls], grads=grads)

    return dict(best=best, table=table, r=r, fr=fr, outs=outs, grads=grads, grad_flat=grad_flat, dls=dls,
                losses=losses, step=step, pair_capacity=pair_capacity)


# --------------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2311_18561_gb300 import render as R
    from paper_2311_18561_gb300 import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    scene = synth.make_urban_scene(N_GAUSS, seed=0)
    frame_idx = replica_frame(rank)
    cam = workload_camera(frame_idx)
    st = R.scene_to_device(scene, dev)
    target_host = torch.from_numpy(synth.random_image(H_PIX, W_PIX, seed=1)).pin_memory()
    target = target_host.to(dev)
    ts = tuned_step(dev, st, [cam], [target], args.tile)
    best, table, r, fr, outs = ts["best"], ts["table"], ts["r"], ts["fr"], ts["outs"]
    grad_flat, grads, pair_capacity = ts["grad_flat"], ts["grads"], ts["pair_capacity"]
    dl, loss = ts["dls"][0], ts["losses"][0:1]
    dp = args.dp and world > 1
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def step():
        ts["step"]()
        if dp:
            R.allreduce_gradients(grad_flat)

    def fwd_only():
        r.forward(st, [cam], outs=outs, frame=fr)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    # (a data-parallel step keeps its collective outside a captured graph)
    step_graph, launches_per_step = capture_graph(step, dev) if not dp else (None, 35)
    fwd_graph, _ = capture_graph(fwd_only, dev)
    barrier()

    # ---- timed region: K full steps, each one replay of the captured step
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t0 = time.perf_counter()
    step_ms = timed_steps(step_graph.replay if step_graph is not None else step, args.steps, flush)
    barrier()
    wall = time.perf_counter() - t0
    launches = launches_per_step * args.steps
    # forward-only rate (same protocol)
    fwd_ms = timed_steps(fwd_graph.replay, args.steps, flush) / args.steps
    # the FP32 peak of the ALU rooflines, at the clocks sampled here
    fp32 = measure_fp32_peak(dev)
    clk = clocks.stop()
    # per-stage times from the library's event timer, in eager steps after
    # the timed region (the events add a little time of their own)
    stage_ms = stage_profile(r, step, args.steps, flush)

    M, K, ov = fr.stats()
    if ov:
        raise RuntimeError("pair capacity %d overflowed (K = %d)" % (pair_capacity, K))
    r.forward(st, [cam], outs=outs, frame=fr)
    E, B = R.eval_count(r, fr)
    ms_step = step_ms / args.steps
    ms_step, fwd_ms = max_over_ranks([ms_step, fwd_ms], world, dev)
    mpix = W_PIX * H_PIX / 1e6

    # ---- end to end through the public API: every step copies its target
    # in from pinned host memory and reads the loss back.  `e2e` uses the
    # captured training step of the batch API (BatchGraph: forward + L1 +
    # backward as one CUDA graph, here for the one view); `e2e_eager` the
    # per-call API (Renderer.forward, l1_loss, Renderer.backward).  With
    # --dp the gradient all-reduce is outside the graph: both use the
    # per-call path.
    def e2e_time(step_fn, copy_in, loss_t, stream):
        loss_host = torch.empty(1, pin_memory=True)
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                copy_in()
                step_fn()
                loss_host.copy_(loss_t, non_blocking=True)
                stream.synchronize()
        return (time.perf_counter() - e0) / args.steps

    e2e_eager_s = e2e_time(step, lambda: target.copy_(target_host, non_blocking=True), loss,
                           torch.cuda.current_stream())
    if dp:
        e2e_s, e2e_api = e2e_eager_s, "Renderer.forward + l1_loss + Renderer.backward + all-reduce"
    else:
        from paper_2311_18561_gb300.batch import BatchGraph

        # the graph copies the pinned host target in on a side stream that
        # overlaps the forward pass (host_targets), so copy_in is empty
        bg = BatchGraph(st, [cam], targets=[target], config=best, autotune=False, host_targets=[target_host])
        with torch.cuda.stream(bg.stream):
            for _ in range(max(3, args.warmup)):
                bg.replay()
        e2e_s = e2e_time(bg.replay, lambda: None, bg.losses[0:1], bg.stream)
        e2e_api = ("BatchGraph.replay (one CUDA graph: the pinned target's host-to-device copy beside "
                   "the forward pass, then L1 and backward)")
        del bg
    e2e_s, e2e_eager_s = max_over_ranks([e2e_s, e2e_eager_s], world, dev)

    # ---- the same step with the paper's photometric loss (1 - 0.2) L1 + 0.2 (1 - SSIM)
    def step_paper_loss():
        r.forward(st, [cam], outs=outs, frame=fr)
        R.rgb_loss(r, outs[0]["rgb"], target, lambda_r=0.2, dl=dl, loss=loss3)
        r.backward(st, [cam], fr, [dict(rgb=dl)], grads=grads)

    loss3 = torch.empty(3, device=dev)
    paper_loss = features = None
    for _ in range(0 if args.no_legs else 3):
        step_paper_loss()
    if not args.no_legs:
        paper_graph, _ = capture_graph(step_paper_loss, dev)
        paper_step_ms = timed_steps(paper_graph.replay, args.steps, flush) / args.steps
        loss_graph, _ = capture_graph(lambda: R.rgb_loss(r, outs[0]["rgb"], target, lambda_r=0.2, dl=dl,
                                                         loss=loss3), dev)
        loss_ms = timed_steps(loss_graph.replay, args.steps, flush) / args.steps
        # separable filtering: 5 moments and 3 derivative maps x 2 passes x 11 taps,
        # 3 products, ~20 for S and its derivatives, 5 for the gradient, 3 for L1
        loss_ops = 3 * W_PIX * H_PIX * OPS_PER_LOSS_PIXEL
        alu_peak = fp32["lane_fma_per_s"]
        paper_loss = {"step_ms": paper_step_ms, "loss_ms": loss_ms,
                      "roofline_loss": {"kernel": "k_rgb_loss", "bound": "alu",
                                        "achieved": loss_ops / (loss_ms * 1e-3) / 1e12, "peak": alu_peak / 1e12,
                                        "unit": "T FP32-lane-instr/s", "peak_kind": "measured (FMA probe)",
                                        "frac": loss_ops / (loss_ms * 1e-3) / alu_peak,
                                        "work": "%d FP32 instructions per pixel and channel" % OPS_PER_LOSS_PIXEL,
                                        "hbm_bytes": 3 * W_PIX * H_PIX * 12,
                                        "note": "includes the fixed-order reduction kernel"}}

        # ---- the same step rendering and differentiating the extra channels:
        # velocity (3), staticness (1) and 19 semantic classes
        from paper_2311_18561_gb300 import abi as A
        st_f = dict(st)
        st_f["sem"] = torch.tensor(synth.make_semantics(N_GAUSS, 19, seed=5), device=dev)
        fmask = A.FEAT_VBAR | A.FEAT_RHO | A.FEAT_SEM
        outs_f = r.alloc_images([cam], features=fmask, n_sem=19)
        dl_feat = torch.randn(23, H_PIX, W_PIX, device=dev) * 1e-6
        grads_f = dict(grads)
        grads_f["sem"] = torch.empty_like(st_f["sem"])

        def step_features():
            r.forward(st_f, [cam], outs=outs_f, frame=fr, features=fmask)
            R.l1_loss(r, outs_f[0]["rgb"], target, dl=dl, loss=loss)
            r.backward(st_f, [cam], fr, [dict(rgb=dl, feat=dl_feat)], grads=grads_f)

        for _ in range(3):
            step_features()
        feat_graph, _ = capture_graph(step_features, dev)
        features = {"channels": "v_bar (3) + rho (1) + 19 semantic classes",
                    "step_ms": timed_steps(feat_graph.replay, args.steps, flush) / args.steps}
        del st_f, outs_f, dl_feat, grads_f, feat_graph

    # ---- roofline of the dominant stage
    roof = dominant_roof(stage_ms, E, B, N_GAUSS, M, K, fp32,
                         traffic=ncu_traffic("k_composite_bwd", "%dx%dx%d" % best) if args.workload == "urban"
                         else None)
    pk = peaks()
    out = {
        "metric": METRIC, "value": job_value(world, mpix, ms_step), "unit": "Mpix/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded urban-shaped PVG scene, random-init parameters)",
        "config": {"workload": WORKLOAD, "gaussians": N_GAUSS, "width": W_PIX, "height": H_PIX,
                   "name": args.workload, "sh_degree": 3,
                   "tile": "%dx%d, %d px/thread (%s)" % (best[0], best[1], best[2],
                                                         "given" if table is None else "autotuned"),
                   "l2": "flushed before every step (256 MB write)",
                   "step": "one CUDA-graph replay of forward + L1 + backward (pair capacity %d = 2x the measured K, no host round trip)" % pair_capacity,
                   "parallelism": ("data parallel, gradients all-reduced" if dp else "replicas")
                   if world > 1 else "single GPU"},
        "fwd_bwd_step_ms": ms_step,
        "autotune_ms": None if table is None else {"%dx%dx%d" % k: round(v, 4) for k, v in table.items()},
        "render_fwd": {"ms": fwd_ms, "mpix_s": job_value(world, mpix, fwd_ms)},
        "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
        "visible": M, "pairs": K, "evals": E, "blended_evals": B, "overflow": ov,
        "roofline_composite_fwd": alu_roof("composite", stage_ms, E, B, fp32),
        "sm_count": fp32["sm_count"],
        "fp32_peak": {"value": fp32["lane_fma_per_s"] / 1e12, "unit": "T lane-FMA/s", "kind": "measured",
                      **{k: v for k, v in fp32.items() if k != "lane_fma_per_s"}},
        "hbm_peak": {"value": pk["hbm_gbs"], "unit": "GB/s", "kind": pk["source"]},
        "wall_s_timed_region": wall,
        "roofline": roof,
        "e2e": {"value": job_value(world, mpix, e2e_s * 1e3), "unit": "Mpix/s",
                "h2d_bytes_per_step": target_host.numel() * 4,
                "d2h_bytes_per_step": 4,
                "api": e2e_api + "; only the 4-byte loss is read back (images and gradients stay on the device)"},
        "e2e_eager": {"value": job_value(world, mpix, e2e_eager_s * 1e3), "unit": "Mpix/s",
                      "h2d_bytes_per_step": target_host.numel() * 4, "d2h_bytes_per_step": 4,
                      "api": "Renderer.forward + l1_loss + Renderer.backward; only the 4-byte loss is read back"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "paper_loss_step": paper_loss,
        "features_step": features,
    }
    del flush
    if rank == 0 and not args.no_legs and args.workload == "urban":
        # the other configurations, each with its own roofline
        del st, grads, grad_flat, ts, r, fr, outs
        torch.cuda.empty_cache()
        out["training"] = training_leg(dev, max(3, args.steps // 2), fp32)
        torch.cuda.empty_cache()
        out["batched"] = batched_leg(dev, max(3, args.steps // 4), fp32)
        torch.cuda.empty_cache()
    if not args.no_serve and rank == 0:
        torch.cuda.empty_cache()
        rates = [args.serve_rate] if args.serve_rate else [200.0, 500.0, 1000.0, 2000.0]
        out["serving"] = {"legs": [serving_leg(dev, rt, args.serve_seconds or 5.0, config=(16, 16, 1))
                                   for rt in rates]}
        release_serve_scenes()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(scene, cam, args.cpu_seconds)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def training_leg(dev, steps, fp32):
    """The training configuration: a 1M-Gaussian urban-distribution scene
    at 1242x375 (f = 720), frame 25, forward + L1 + backward as one CUDA
    graph in the autotuned configuration; stage times, K / E counts and
    the roofline of its dominant stage."""
    import torch

    from paper_2311_18561_gb300 import render as R
    from paper_2311_18561_gb300 import synth

    n, w, h, f = WORKLOADS["training"][:4]
    scene = R.scene_to_device(synth.make_urban_scene(n, seed=0), dev)
    cam = synth.street_camera(FRAME / 49.0, w, h, fx=f)
    target = torch.from_numpy(synth.random_image(h, w, seed=1)).to(dev)
    ts = tuned_step(dev, scene, [cam], [target])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(3):
        ts["step"]()
    g, launches = capture_graph(ts["step"], dev)
    ms = timed_steps(g.replay, steps, flush) / steps
    stage_ms = stage_profile(ts["r"], ts["step"], steps, flush)
    M, K, ov = ts["fr"].stats()
    ts["r"].forward(scene, [cam], outs=ts["outs"], frame=ts["fr"])
    E, B = R.eval_count(ts["r"], ts["fr"])
    mpix = w * h / 1e6
    best = ts["best"]
    return {"workload": WORKLOADS["training"][4], "ms_per_step": ms, "mpix_s": mpix / (ms * 1e-3),
            "tile": "%dx%d, %d px/thread (autotuned)" % best, "steps": steps, "gpu_launches_per_step": launches,
            "l2": "flushed before every step", "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
            "visible": M, "pairs": K, "evals": E, "blended_evals": B, "overflow": ov,
            "roofline": dominant_roof(stage_ms, E, B, n, M, K, fp32),
            "roofline_composite_bwd": alu_roof("composite_bwd", stage_ms, E, B, fp32)}


def batched_leg(dev, steps, fp32):
    """64 views (22 x 1920x1280, 21 x 1242x375, 21 x 960x640, own t each) of
    a 3M-Gaussian urban scene: forward + L1 + backward replayed as one CUDA
    graph, against one launch sequence per view; the stage split of both
    (where the batched step spends its time against 64 single views)."""
    import torch

    from paper_2311_18561_gb300 import batch as Bt
    from paper_2311_18561_gb300 import render as R
    from paper_2311_18561_gb300 import synth

    scene = R.scene_to_device(synth.make_urban_scene(3_000_000, seed=0), dev)
    cams = synth.batched_views(seed=0, n_views=64)
    g = Bt.BatchGraph(scene, cams, autotune=True,
                      tune_configs=((16, 16, 1), (16, 16, 2), (16, 16, 4), (32, 16, 4), (16, 32, 4), (32, 32, 4)))
    mpix = g.pixels / 1e6
    for _ in range(3):
        g.replay()
    ms_graph = timed_steps(g.replay, steps) / steps
    over = g.overflowed()
    tw, th, px = g.config
    # the same 64-view step eagerly, for the stage split
    stages_batched = stage_profile(g.r, g._enqueue, 2)
    M, K, _ = g.frame.stats()
    g.r.forward(scene, cams, outs=g.outs, frame=g.frame)
    E, B = R.eval_count(g.r, g.frame)
    # one launch sequence per view
    r1 = R.Renderer(tile=(tw, th), pixels_per_thread=px)
    f1 = R.Frame()
    o1 = {}
    grads = {k: torch.empty_like(scene[k]) for k in R.PARAM_NAMES}

    def per_view():
        for v, cam in enumerate(cams):
            key = (cam["width"], cam["height"])
            if key not in o1:
                o1[key] = r1.alloc_images([cam])
            o = r1.forward(scene, [cam], outs=o1[key], frame=f1)[0]
            dl = R.l1_loss(r1, o["rgb"], g.targets[v])[1]
            r1.backward(scene, [cam], f1, [dict(rgb=dl)], grads=grads)

    per_view()
    ms_per_view = timed_steps(per_view, max(2, steps // 2)) / max(2, steps // 2)
    stages_per_view = stage_profile(r1, per_view, 1)
    r1.close()
    f1.close()
    return {"workload": "batched: 64 views (22x1920x1280, 21x1242x375, 21x960x640), 3M Gaussians SH-3, "
                        "fwd + L1 + bwd", "mpix_per_batch": mpix, "tile": "%dx%d, %d px/thread (autotuned)" % g.config,
            "pair_capacity": g.pair_capacity, "overflow": over, "visible": M, "pairs": K, "evals": E,
            "blended_evals": B,
            "graph": {"ms": ms_graph, "mpix_s": mpix / (ms_graph * 1e-3)},
            "one_launch_per_view": {"ms": ms_per_view, "mpix_s": mpix / (ms_per_view * 1e-3)},
            "stages_ms_batched": {k: round(v, 3) for k, v in stages_batched.items()},
            "stages_ms_per_view_sum": {k: round(v, 3) for k, v in stages_per_view.items()},
            "roofline": dominant_roof(stages_batched, E, B, 64 * 3_000_000, M, K, fp32)}


# --------------------------------------------------------------------------- serving

SERVE_SCENES = None


def release_serve_scenes():
    global SERVE_SCENES
    SERVE_SCENES = None


def serve_scenes(dev):
    """The four resident scenes of the serving config (0.5M, 1M, 2M, 4M
    Gaussians, urban distribution, SH-3)."""
    global SERVE_SCENES
    if SERVE_SCENES is None:
        from paper_2311_18561_gb300 import render as R
        from paper_2311_18561_gb300 import synth

        SERVE_SCENES = [R.scene_to_device(synth.make_urban_scene(n, seed=10 + k), dev)
                        for k, n in enumerate(synth.SERVE_SCENE_SIZES)]
    return SERVE_SCENES


def _percentiles(lat_ms):
    import numpy as np

    a = np.asarray(lat_ms, dtype=np.float64)
    return float(np.percentile(a, 50)), float(np.percentile(a, 99))


def serving_leg(dev, rate, seconds, config=(16, 16, 1), max_batch_views=16, n_streams=4, pipeline_depth=1, seed=0):
    """Poisson arrivals at `rate` req/s for `seconds` (random scene, pose on
    the street path +-2 m, t ~ U[0,1], resolution from {640x480, 1242x375,
    1920x1280}) served by the continuous-batching server, then the same
    schedule served one request per launch, synchronously (the plain path:
    one pvg_render_fwd call per request and a wait for its image)."""
    import collections

    import torch

    from paper_2311_18561_gb300 import render as R
    from paper_2311_18561_gb300 import serve as S
    from paper_2311_18561_gb300 import synth

    scenes = serve_scenes(dev)
    reqs = synth.serve_requests(rate, seconds, n_scenes=len(scenes), seed=seed)
    pool = collections.defaultdict(list)

    def buf(cam):
        key = (cam["width"], cam["height"])
        return pool[key].pop() if pool[key] else torch.empty(3, cam["height"], cam["width"], device=dev)

    srv = S.Server(max_batch_views=max_batch_views, n_streams=n_streams, memory_budget=24 << 30,
                   tile=config[:2], pixels_per_thread=config[2], pipeline_depth=pipeline_depth)
    ids = [srv.add_scene(sc) for sc in scenes]
    # warm-up: every scene at every resolution once (the server learns each
    # scene's pairs per pixel), then a burst of full batches
    warm = []
    for sid in ids:
        for w, h in synth.SERVE_RESOLUTIONS:
            cam = synth.street_camera(0.5, w, h)
            warm.append((srv.submit(sid, cam, dict(rgb=buf(cam))), cam))
    for k in range(2 * n_streams * max_batch_views):
        cam = synth.street_camera(0.5, 1920, 1280)
        warm.append((srv.submit(ids[k % len(ids)], cam, dict(rgb=buf(cam))), cam))
    for rid, cam in warm:
        srv.wait(rid, 120.0)
        srv.release(rid)
    torch.cuda.synchronize()
    c0 = srv.counters()
    requeues0 = srv.arena()["requeues"]
    stats, outstanding, i = [], collections.deque(), 0
    t0 = time.perf_counter()
    while i < len(reqs) or outstanding:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i][0] <= now:
            _, sid, cam = reqs[i]
            b = buf(cam)
            outstanding.append((srv.submit(ids[sid], cam, dict(rgb=b)), cam, b))
            i += 1
        while outstanding:
            rid, cam, b = outstanding[0]
            done, st = srv.poll(rid)
            if not done:
                break
            stats.append((st, cam))
            pool[(cam["width"], cam["height"])].append(b)
            srv.release(rid)
            outstanding.popleft()
        time.sleep(0.0002)
    counters = srv.counters()
    arena = srv.arena()
    srv.close()
    lat = [st["done_ms"] - st["submit_ms"] for st, _ in stats]
    span_ms = max(st["done_ms"] for st, _ in stats) - min(st["submit_ms"] for st, _ in stats)
    pix = sum(c["width"] * c["height"] for _, c in stats)
    p50, p99 = _percentiles(lat)
    batches = counters["batches"] - c0["batches"]
    views = counters["views"] - c0["views"]
    served = {"p50_ms": p50, "p99_ms": p99, "mpix_s": pix / (span_ms * 1e-3) / 1e6, "requests": len(stats),
              "launches": batches, "mean_views_per_launch": views / max(1, batches),
              "mean_gpu_ms_per_request": sum(st["gpu_ms"] for st, _ in stats) / max(1, len(stats)),
              "requeues": arena["requeues"] - requeues0,
              "errors": sum(1 for st, _ in stats if st["status"] != 0)}
    # one request per launch, synchronous, same schedule
    r = R.Renderer(tile=config[:2], pixels_per_thread=config[2])
    for k in range(3):
        r.forward(scenes[-1], [synth.street_camera(0.5, 1920, 1280)])
    torch.cuda.synchronize()
    lat1, outs1 = [], {}
    t0 = time.perf_counter()
    for arr, sid, cam in reqs:
        now = time.perf_counter() - t0
        if now < arr:
            time.sleep(arr - now)
        key = (cam["width"], cam["height"])
        if key not in outs1:
            outs1[key] = r.alloc_images([cam])
        r.forward(scenes[sid], [cam], outs=outs1[key])
        torch.cuda.synchronize()
        lat1.append((time.perf_counter() - t0 - arr) * 1e3)
    span1 = time.perf_counter() - t0 - reqs[0][0]
    r.close()
    q50, q99 = _percentiles(lat1)
    one = {"p50_ms": q50, "p99_ms": q99, "mpix_s": pix / span1 / 1e6}
    return {"rate_req_s": rate, "seconds": seconds, "scenes": list(synth.SERVE_SCENE_SIZES),
            "max_batch_views": max_batch_views, "streams": n_streams, "pipeline_depth": pipeline_depth,
            "arena_per_worker": {k: arena[k] for k in ("items_per_batch", "pixels_per_batch", "pairs_per_batch")},
            "free_bytes_at_create": arena["free_bytes"], "served": served, "one_request_per_launch": one}


def run_serving(args):
    """Serving sweep over request rates (report only)."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rates = [args.serve_rate] if args.serve_rate else [200.0, 500.0, 1000.0, 2000.0]
    res = [serving_leg(dev, rt, args.serve_seconds or 10.0) for rt in rates]
    if rank == 0:
        print(json.dumps({"metric": METRIC, "workload": "serving sweep", "legs": res}), flush=True)


def run_batched(args):
    """The batched configuration on its own (see batched_leg)."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fp32 = measure_fp32_peak(dev)
    res = batched_leg(dev, max(3, args.steps), fp32)
    if rank == 0:
        print(json.dumps({"metric": METRIC, **res}), flush=True)


# --------------------------------------------------------------------------- oracle

def oracle_sample_step(scene, cam, pixels, w_rgb):
    """One bounded-sample step of the FP64 oracle: forward on the sampled
    pixels (culled mode) and the backward of L = sum w . rgb there."""
    import numpy as np

    import oracle

    oracle.render(scene, cam, mode="culled", pixels=pixels)
    P = pixels.shape[0]
    oracle.render_bwd(scene, cam, w_rgb, np.zeros(P), np.zeros(P), mode="culled", pixels=pixels)


def _sample_pixels(n, seed=0):
    import numpy as np

    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, W_PIX, n), rng.integers(0, H_PIX, n)], axis=1).astype(np.int32)


def cpu_baseline(scene, cam, seconds):
    """Time the oracle (as it stands) on a pixel sample sized so one step
    takes about `seconds` of wall time on the host cores."""
    import numpy as np

    import oracle

    oracle.build()
    cores = oracle.num_threads()
    n = 64
    pix = _sample_pixels(n)
    t0 = time.perf_counter()
    oracle_sample_step(scene, cam, pix, np.ones((n, 3)) / n)
    t_small = time.perf_counter() - t0
    # the per-call preprocess + sort of all N Gaussians is a fixed cost
    n2 = 4 * n
    pix2 = _sample_pixels(n2)
    t0 = time.perf_counter()
    oracle_sample_step(scene, cam, pix2, np.ones((n2, 3)) / n2)
    t_big = time.perf_counter() - t0
    per_px = max((t_big - t_small) / (n2 - n), 1e-6)
    fixed = max(t_small - per_px * n, 0.0)
    n3 = int(min(max((seconds - fixed) / per_px, 64), 200_000))
    pix3 = _sample_pixels(n3, seed=1)
    t0 = time.perf_counter()
    oracle_sample_step(scene, cam, pix3, np.ones((n3, 3)) / n3)
    t = time.perf_counter() - t0
    return {"value": n3 / t / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "sample": "%d random pixels of the 1920x1280 frame; FP64 oracle forward (culled) + backward on "
                      "those pixels, including its per-call preprocess and depth sort of all %d Gaussians "
                      "(%.1f s)" % (n3, N_GAUSS, t),
            "other_configs": oracle_other_configs()}


def oracle_other_configs():
    """The rest of the oracle's timing plan, bounded to a few seconds: the
    plain configuration (2,000 Gaussians, 160x120) rendered whole by brute
    force (every Gaussian for every pixel), and the training configuration
    (1M Gaussians, 1242x375) forward + backward on a pixel sample."""
    import numpy as np

    import oracle
    from paper_2311_18561_gb300 import synth

    out = {}
    scene = synth.make_plain_scene(seed=0, n=2000)
    cam = synth.plain_camera()
    t0 = time.perf_counter()
    oracle.render(scene, cam, mode="brute")
    t = time.perf_counter() - t0
    out["plain_brute_force"] = {"mpix_s": 160 * 120 / t / 1e6, "seconds": t,
                                "workload": "2,000 Gaussians, 160x120, every Gaussian at every pixel"}
    n, w, h, f = WORKLOADS["training"][:4]
    scene = synth.make_urban_scene(n, seed=0)
    cam = synth.street_camera(FRAME / 49.0, w, h, fx=f)
    rng = np.random.default_rng(3)
    P = 2000
    pix = np.stack([rng.integers(0, w, P), rng.integers(0, h, P)], axis=1).astype(np.int32)
    t0 = time.perf_counter()
    oracle_sample_step(scene, cam, pix, np.ones((P, 3)) / P)
    t = time.perf_counter() - t0
    out["training_backward"] = {"mpix_s": P / t / 1e6, "seconds": t,
                                "workload": "1M Gaussians, 1242x375: forward (culled) + backward on %d random "
                                            "pixels, including the per-call preprocess of all Gaussians" % P}
    return out


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2311_18561_gb300 import synth

    oracle.build()
    scene = synth.make_urban_scene(N_GAUSS, seed=0)
    cam = workload_camera(FRAME)
    # size each step's sample so that warmup + steps stay within a few minutes
    per_step_budget = max(2.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    cb = cpu_baseline(scene, cam, per_step_budget)
    n = int(cb["sample"].split()[0])
    pix = _sample_pixels(n, seed=2)
    w = np.ones((n, 3)) / n
    for _ in range(args.warmup):
        oracle_sample_step(scene, cam, pix, w)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample_step(scene, cam, pix, w)
    dt = (time.perf_counter() - t0) / args.steps
    v = n / dt / 1e6
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpix/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "gaussians": N_GAUSS, "width": W_PIX, "height": H_PIX,
                      "sample_pixels_per_step": n},
           "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": "%d random pixels per step, FP64 oracle forward + backward" % n},
           "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    select_workload(args.workload)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

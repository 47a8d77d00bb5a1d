"""Host logic of the autotuner, with the GPU timing replaced by a fake:
the fastest configuration wins, results are cached per workload shape and
reused without timing again, and the key tells workloads apart.  No GPU."""
import json

import numpy as np
import torch

from paper_2311_18561_gb300 import synth
from paper_2311_18561_gb300 import tune as T


def _scene(n, deg):
    sc = synth.make_plain_scene(seed=0, n=n, sh_degree=deg)
    return {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in sc.items() if not k.startswith("_")}


def test_fastest_config_is_cached_and_reused(tmp_path, monkeypatch):
    times = {cfg: 1.0 + i for i, cfg in enumerate(T.CONFIGS)}
    times[(32, 32, 4)] = 0.5
    calls = []

    def fake(cfg, scene_t, cams, backward, warmup, iters):
        calls.append(cfg)
        return times[tuple(cfg)]

    monkeypatch.setattr(T, "_time_config", fake)
    path = str(tmp_path / "tune.json")
    st, cams = _scene(50, 1), [synth.plain_camera()]
    best, table = T.tune(st, cams, backward=True, cache_path=path)
    assert best == (32, 32, 4) and len(calls) == len(T.CONFIGS) and table[(32, 32, 4)] == 0.5
    cache = json.load(open(path))
    assert list(cache) == [T.workload_key(st, cams, True)]
    # the same workload again: read from the cache, nothing timed
    best2, table2 = T.tune(st, cams, backward=True, cache_path=path)
    assert best2 == best and table2 == table and len(calls) == len(T.CONFIGS)
    # a forward-only tuning of the same scene is another workload
    T.tune(st, cams, backward=False, cache_path=path)
    assert len(calls) == 2 * len(T.CONFIGS) and len(json.load(open(path))) == 2
    # use_cache=False times again and leaves the file alone
    T.tune(st, cams, backward=True, cache_path=path, use_cache=False)
    assert len(calls) == 3 * len(T.CONFIGS) and len(json.load(open(path))) == 2


def test_workload_key_tells_shapes_apart():
    cams = [synth.plain_camera(160, 120), synth.plain_camera(64, 48)]
    k = T.workload_key(_scene(50, 1), cams, True)
    assert k != T.workload_key(_scene(51, 1), cams, True)
    assert k != T.workload_key(_scene(50, 2), cams, True)
    assert k != T.workload_key(_scene(50, 1), cams[:1], True)
    assert k != T.workload_key(_scene(50, 1), cams, False)
    assert k == T.workload_key(_scene(50, 1), cams, True)


def test_corrupt_cache_is_ignored(tmp_path, monkeypatch):
    monkeypatch.setattr(T, "_time_config", lambda cfg, *a: 2.0 if tuple(cfg) != (16, 16, 1) else 1.0)
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    best, _ = T.tune(_scene(20, 0), [synth.plain_camera()], cache_path=str(path))
    assert best == (16, 16, 1)
    assert json.loads(path.read_text())  # rewritten as valid JSON

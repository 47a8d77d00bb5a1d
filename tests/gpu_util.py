"""Helpers shared by the GPU tests: run the CUDA path through the C ABI
and compare with the FP64 oracle."""
import numpy as np
import torch

import oracle
from oracle import binning

from . import parity_log

# Image tolerance: max-abs 1e-3 per channel in [0, 1] (rgb, alpha) on
# pixels the oracle does not flag; flagged pixels (a gate within 1e-5
# relative of its threshold, or two blended depths within 1e-6 relative:
# FP32 may decide those differently) are held to 1/255 + 1e-3 and must be
# rare.  Depth (metres, not in [0, 1]) is held to 1e-3 relative.
TOL = 1e-3
FLAG_TOL = 1.0 / 255.0 + 1e-3
# Flagged pixels may be at most 0.1 % of the compared pixels (the 1.5M
# urban frame at 1920x1280 flags 0.08 % of its sampled pixels).  Nearly all
# flags are near-ties in depth (two blended Gaussians within 1e-6 relative)
# and one such pair flags every pixel of its overlap, so scenes dense in
# such pairs pass DENSE_TIE_FLAG_FRAC (2 %) explicitly: the small synthetic
# scenes (a few hundred to 2,000 large Gaussians on a few thousand pixels:
# up to 1.4 %) and the urban distribution at 1242x375 (200k to 1M
# Gaussians: 0.5 to 1.8 %).  Either cap still holds at least 98 % of the
# pixels to the 1e-3 bound; the real fractions are printed in the run's
# terminal summary.
MAX_FLAG_FRAC = 1e-3
DENSE_TIE_FLAG_FRAC = 0.02


def to_numpy_images(out):
    return dict(rgb=out["rgb"].permute(1, 2, 0).cpu().numpy().astype(np.float64),
                depth=out["depth"].cpu().numpy().astype(np.float64),
                alpha=out["alpha"].cpu().numpy().astype(np.float64))


def compare_to_oracle(got, ref, pixels=None, max_flag_frac=MAX_FLAG_FRAC):
    """got: dict of numpy arrays [H,W,(3)] or [P,(3)] if pixels given."""
    flag = ref["flag"] != 0
    e_rgb = np.abs(got["rgb"] - ref["rgb"]).max(axis=-1)
    e_a = np.abs(got["alpha"] - ref["alpha"])
    zscale = np.maximum(1.0, np.abs(ref["depth"]))
    e_d = np.abs(got["depth"] - ref["depth"]) / zscale
    ok = ~flag
    report = dict(max_rgb=float(e_rgb[ok].max(initial=0)), max_alpha=float(e_a[ok].max(initial=0)),
                  max_depth_rel=float(e_d[ok].max(initial=0)), flagged=int(flag.sum()),
                  flagged_max=float(max(e_rgb[flag].max(initial=0), e_a[flag].max(initial=0))),
                  flagged_frac=float(flag.mean()))
    parity_log.record("image", flag.size, flag.sum(), rgb=report["max_rgb"], alpha=report["max_alpha"],
                      depth_rel=report["max_depth_rel"], flagged_max=report["flagged_max"])
    assert report["max_rgb"] <= TOL, report
    assert report["max_alpha"] <= TOL, report
    assert report["max_depth_rel"] <= TOL, report
    assert report["flagged_max"] <= FLAG_TOL, report
    assert flag.mean() <= max_flag_frac, report
    return report


def gpu_render(renderer, scene_t, cams, frame=None):
    outs = renderer.forward(scene_t, cams, frame=frame)
    torch.cuda.synchronize()
    return outs


def check_tile_lists(ex, scene, cam, tile, tiles_x, tiles_y):
    """The GPU's per-tile lists (exported frame `ex`) against what is fixed:
    each list is an ordered subset of the bounding-rectangle list (plain
    definition over the GPU's own rectangles and depth keys), it holds
    every tile where the FP64 oracle blends the Gaussian (level shrunk by
    1e-3 against rounding), and the ranges partition the pairs in tile
    order.  Returns (pairs kept, pairs of the rectangle lists)."""
    gid, zk, rect = ex["sorted_gid"], ex["depth_key"], ex["rect"]
    z = zk.view(np.float32)
    values, ranges = binning.tile_lists(gid, z, rect[:, [0, 1, 2, 3]], tiles_x, tiles_y)
    got_vals = gid[ex["pair_vals"]].astype(np.int64)
    got_r = ex["ranges"].astype(np.int64)
    lens = got_r[:, 1] - got_r[:, 0]
    assert np.all(lens >= 0) and lens.sum() == got_vals.size
    nonempty = lens > 0
    np.testing.assert_array_equal(got_r[nonempty, 0], np.concatenate([[0], np.cumsum(lens[nonempty])[:-1]]))
    pp = oracle.preprocess(scene, cam)
    need = binning.contributing_tiles(pp["uv"][gid], pp["conic"][gid], pp["ot"][gid], cam["width"],
                                      cam["height"], tile[0], tile[1], shrink=1 - 1e-3)
    kept = {}
    for t in range(tiles_x * tiles_y):
        full = values[ranges[t, 0]:ranges[t, 1]]
        got = got_vals[got_r[t, 0]:got_r[t, 1]]
        pos = {int(g): i for i, g in enumerate(full)}
        idx = np.array([pos.get(int(g), -1) for g in got])
        assert np.all(idx >= 0) and np.all(np.diff(idx) > 0), t
        for g in got:
            kept.setdefault(int(g), set()).add(t)
    for k, g in enumerate(gid):
        assert need[k] <= kept.get(int(g), set()), int(g)
    return got_vals.size, values.size

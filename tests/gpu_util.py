"""Helpers shared by the GPU tests: run the CUDA path through the C ABI
and compare with the FP64 oracle."""
import numpy as np
import torch

# Image tolerance: max-abs 1e-3 per channel in [0, 1] (rgb, alpha) on
# pixels the oracle does not flag; flagged pixels (a gate within 1e-5
# relative of its threshold, or two blended depths within 1e-6 relative:
# FP32 may decide those differently) are held to 1/255 + 1e-3 and must be
# rare.  Depth (metres, not in [0, 1]) is held to 1e-3 relative.
TOL = 1e-3
FLAG_TOL = 1.0 / 255.0 + 1e-3


def to_numpy_images(out):
    return dict(rgb=out["rgb"].permute(1, 2, 0).cpu().numpy().astype(np.float64),
                depth=out["depth"].cpu().numpy().astype(np.float64),
                alpha=out["alpha"].cpu().numpy().astype(np.float64))


def compare_to_oracle(got, ref, pixels=None, max_flag_frac=0.05):
    """got: dict of numpy arrays [H,W,(3)] or [P,(3)] if pixels given."""
    flag = ref["flag"] != 0
    e_rgb = np.abs(got["rgb"] - ref["rgb"]).max(axis=-1)
    e_a = np.abs(got["alpha"] - ref["alpha"])
    zscale = np.maximum(1.0, np.abs(ref["depth"]))
    e_d = np.abs(got["depth"] - ref["depth"]) / zscale
    ok = ~flag
    report = dict(max_rgb=float(e_rgb[ok].max(initial=0)), max_alpha=float(e_a[ok].max(initial=0)),
                  max_depth_rel=float(e_d[ok].max(initial=0)), flagged=int(flag.sum()),
                  flagged_max=float(max(e_rgb[flag].max(initial=0), e_a[flag].max(initial=0))))
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

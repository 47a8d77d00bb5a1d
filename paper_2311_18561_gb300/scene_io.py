"""Scene files: a PVG scene's parameter arrays (structure of arrays,
float32) and a JSON header in one ``.npz``, so that a benchmark or a test
can be rerun on the same bytes.

Header: format version, point count N, SH degree, the array names with
their shapes, and free-form metadata (the generator and seed, say).
Optional arrays: ``sem`` [N, S] and ``sky`` [6, R, R, 3].
"""
from __future__ import annotations

import json

import numpy as np

FORMAT = "pvg-scene/1"
PARAMS = ("mu", "vel", "tau", "beta", "period", "scale", "quat", "opacity", "sh")
OPTIONAL = ("sem", "sky")


def _shapes(n, k):
    return dict(mu=(n, 3), vel=(n, 3), tau=(n,), beta=(n,), period=(n,), scale=(n, 3), quat=(n, 4),
                opacity=(n,), sh=(n, k, 3))


def save_scene(path, scene, meta=None):
    """Writes ``scene`` (dict of arrays, or torch tensors) to ``path``."""
    arrs = {}
    for name in PARAMS + OPTIONAL:
        v = scene.get(name)
        if v is None:
            continue
        if hasattr(v, "detach"):
            v = v.detach().cpu().numpy()
        arrs[name] = np.ascontiguousarray(v, dtype=np.float32)
    n = int(arrs["mu"].shape[0])
    k = int(arrs["sh"].shape[1])
    deg = int(round(np.sqrt(k))) - 1
    if (deg + 1) ** 2 != k or not 0 <= deg <= 3:
        raise ValueError("sh must be [N, (D+1)^2, 3] with D in 0..3")
    for name, shape in _shapes(n, k).items():
        if arrs[name].shape != shape:
            raise ValueError("scene[%r] has shape %s, expected %s" % (name, arrs[name].shape, shape))
    header = dict(format=FORMAT, n=n, sh_degree=deg, arrays={k_: list(v.shape) for k_, v in arrs.items()},
                  meta=meta or {})
    with open(path, "wb") as f:
        np.savez(f, header=np.frombuffer(json.dumps(header).encode(), dtype=np.uint8), **arrs)


def load_scene(path):
    """(scene, header): the arrays of a file written by :func:`save_scene`."""
    with np.load(path) as z:
        header = json.loads(bytes(z["header"]).decode())
        if header.get("format") != FORMAT:
            raise ValueError("not a %s file" % FORMAT)
        scene = {name: np.array(z[name]) for name in header["arrays"]}
    for name, shape in header["arrays"].items():
        if list(scene[name].shape) != shape:
            raise ValueError("array %r does not match the header" % name)
    return scene, header

"""Scene files round-trip bit for bit, with their header.  No GPU."""
import numpy as np
import pytest

from paper_2311_18561_gb300 import scene_io, synth


def test_round_trip(tmp_path):
    scene = synth.make_fd_scene(seed=3, n=37, sh_degree=2)
    scene["sem"] = synth.make_semantics(37, 5)
    scene["sky"] = np.random.default_rng(0).uniform(size=(6, 4, 4, 3)).astype(np.float32)
    p = tmp_path / "s.npz"
    scene_io.save_scene(p, scene, meta=dict(generator="make_fd_scene", seed=3))
    back, header = scene_io.load_scene(p)
    assert header["n"] == 37 and header["sh_degree"] == 2 and header["meta"]["seed"] == 3
    assert set(back) == set(scene)
    for k, v in scene.items():
        assert back[k].dtype == np.float32
        np.testing.assert_array_equal(back[k], np.asarray(v, np.float32))


def test_rejects_bad_shapes(tmp_path):
    scene = synth.make_fd_scene(seed=0, n=5, sh_degree=1)
    scene["quat"] = scene["quat"][:, :3]
    with pytest.raises(ValueError):
        scene_io.save_scene(tmp_path / "bad.npz", scene)

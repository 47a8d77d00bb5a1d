"""Pins of the oracle's integer side (depth order, tile lists, ranges)
against a brute-force scan on tiny inputs, and against invariants that hold
at any size (permutation of the pairs, monotone keys).  No GPU."""
import numpy as np

from oracle import binning


def _random_case(rng, m, tiles_x, tiles_y):
    gid = np.sort(rng.choice(10 * m, size=m, replace=False))
    z = rng.uniform(0.5, 3.0, m).astype(np.float32)
    z[rng.integers(0, m, m // 5)] = z[0]  # plenty of exact ties
    tx0 = rng.integers(0, tiles_x, m)
    ty0 = rng.integers(0, tiles_y, m)
    tx1 = np.minimum(tiles_x, tx0 + rng.integers(0, 4, m))
    ty1 = np.minimum(tiles_y, ty0 + rng.integers(0, 4, m))
    return gid, z, np.stack([tx0, ty0, tx1, ty1], axis=1)


def test_tile_lists_match_brute_force():
    rng = np.random.default_rng(0)
    for _ in range(5):
        gid, z, rect = _random_case(rng, 60, 5, 4)
        values, ranges = binning.tile_lists(gid, z, rect, 5, 4)
        brute = binning.tile_lists_brute(gid, z, rect, 5, 4)
        for t, lst in enumerate(brute):
            s, e = ranges[t]
            assert values[s:e].tolist() == lst


def test_depth_order_ties_by_index():
    gid = np.array([7, 3, 9, 1])
    z = np.array([2.0, 1.0, 1.0, 2.0], np.float32)
    assert binning.depth_order(gid, z).tolist() == [3, 9, 1, 7]


def test_pairs_are_a_permutation_and_sorted():
    rng = np.random.default_rng(1)
    gid, z, rect = _random_case(rng, 400, 12, 9)
    values, ranges = binning.tile_lists(gid, z, rect, 12, 9)
    counts = np.maximum(rect[:, 2] - rect[:, 0], 0) * np.maximum(rect[:, 3] - rect[:, 1], 0)
    assert values.size == counts.sum()
    # every Gaussian appears exactly count times
    got = np.bincount(np.searchsorted(gid, values), minlength=gid.size)
    np.testing.assert_array_equal(got, counts)
    zb = dict(zip(gid.tolist(), binning.zbits(z).tolist()))
    for t in range(12 * 9):
        s, e = ranges[t]
        keys = [(zb[int(g)], int(g)) for g in values[s:e]]
        assert keys == sorted(keys)
    assert ranges[-1, 1] == values.size


def test_contributing_tiles_of_a_disc():
    """A circular Gaussian (conic I / s^2) is blended inside the disc of
    radius s sqrt(2 ln(255 o~)) (closed form); its tiles are those holding a
    pixel centre within that radius, found here by a plain loop."""
    s, o = 3.0, 0.6
    r = s * np.sqrt(2.0 * np.log(255.0 * o))
    W, H, tw, th = 37, 29, 8, 4
    for (u, v) in [(10.3, 12.7), (0.0, 0.0), (36.9, 3.2), (20.0, 28.5)]:
        want = set()
        for py in range(H):
            for px in range(W):
                if (px + 0.5 - u) ** 2 + (py + 0.5 - v) ** 2 <= r * r * (1 - 1e-12):
                    want.add((py // th) * ((W + tw - 1) // tw) + px // tw)
        got = binning.contributing_tiles([[u, v]], [[1 / s**2, 0.0, 1 / s**2]], [o], W, H, tw, th)[0]
        assert got == want, (u, v)
    # below the skip threshold nothing is blended
    assert binning.contributing_tiles([[5, 5]], [[1, 0, 1]], [1 / 255.0], 16, 16, 8, 8)[0] == set()


def test_contributing_tiles_of_a_sheared_ellipse():
    """An anisotropic conic: a pixel centre is in the footprint iff its
    offset's quadratic form is under the level, checked per pixel."""
    a, b, c, o = 0.05, 0.04, 0.08, 0.9
    level = 2 * np.log(255 * o)
    W, H, tw, th = 40, 30, 16, 8
    u, v = 17.2, 14.9
    want = set()
    for py in range(H):
        for px in range(W):
            dx, dy = px + 0.5 - u, py + 0.5 - v
            if a * dx * dx + 2 * b * dx * dy + c * dy * dy <= level:
                want.add((py // th) * 3 + px // tw)
    got = binning.contributing_tiles([[u, v]], [[a, b, c]], [o], W, H, tw, th)[0]
    assert got == want and len(want) < 3 * 4

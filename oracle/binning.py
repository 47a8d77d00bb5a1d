"""Integer side of the oracle: depth order, tile lists and tile ranges.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Given, for each visible Gaussian of one view, its tile rectangle and the
float32 bits of its camera depth z (both taken from the renderer under test,
so that the integer work is compared on identical inputs), this builds the
plain definition of what binning plus sorting must produce (Sec. 3.1:
Gaussians are sorted by camera depth and blended per tile):

* the depth order of the visible Gaussians, by (z, index);
* for every tile, the list of Gaussians whose rectangle covers it, ordered
  by (z, index);
* per tile, the [start, end) range of its list in the concatenation of all
  lists in tile order.

z > 0 for every visible Gaussian, so the IEEE-754 bit pattern of z orders
like z itself.
"""
from __future__ import annotations

import numpy as np


def zbits(z):
    return np.ascontiguousarray(z, dtype=np.float32).view(np.uint32).astype(np.uint64)


def depth_order(gid, z):
    """gid sorted by (z bits, gid)."""
    gid = np.asarray(gid, np.int64)
    order = np.lexsort((gid, zbits(z)))
    return gid[order]


def tile_lists(gid, z, rect, tiles_x, tiles_y):
    """rect [M, 4] = (tx0, ty0, tx1, ty1), half-open in tiles.

    Returns (values, ranges): values = gid of every (tile, Gaussian) pair
    sorted by (tile, z, gid); ranges [tiles, 2] = start/end per tile.
    """
    gid = np.asarray(gid, np.int64)
    rect = np.asarray(rect, np.int64).reshape(-1, 4)
    zb = zbits(z)
    tiles, gids, zs = [], [], []
    for k in range(gid.shape[0]):
        tx0, ty0, tx1, ty1 = rect[k]
        if tx1 <= tx0 or ty1 <= ty0:
            continue
        ty, tx = np.meshgrid(np.arange(ty0, ty1), np.arange(tx0, tx1), indexing="ij")
        t = (ty * tiles_x + tx).reshape(-1)
        tiles.append(t)
        gids.append(np.full(t.shape, gid[k]))
        zs.append(np.full(t.shape, zb[k], dtype=np.uint64))
    ntiles = tiles_x * tiles_y
    if not tiles:
        return np.zeros(0, np.int64), np.zeros((ntiles, 2), np.int64)
    tiles = np.concatenate(tiles)
    gids = np.concatenate(gids)
    zs = np.concatenate(zs)
    order = np.lexsort((gids, zs, tiles))
    values = gids[order]
    counts = np.bincount(tiles, minlength=ntiles)
    ends = np.cumsum(counts)
    ranges = np.stack([ends - counts, ends], axis=1)
    return values, ranges


def tile_lists_brute(gid, z, rect, tiles_x, tiles_y):
    """The same lists built the slow way: for each tile, scan every Gaussian
    in depth order and keep those whose rectangle covers the tile."""
    order = depth_order(gid, z)
    pos = {int(g): k for k, g in enumerate(np.asarray(gid, np.int64))}
    rect = np.asarray(rect, np.int64).reshape(-1, 4)
    lists = []
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            lst = []
            for g in order:
                tx0, ty0, tx1, ty1 = rect[pos[int(g)]]
                if tx0 <= tx < tx1 and ty0 <= ty < ty1:
                    lst.append(int(g))
            lists.append(lst)
    return lists


def contributing_tiles(uv, conic, ot, width, height, tile_w, tile_h, shrink=1.0):
    """Per Gaussian, the set of tile ids (row-major, ``ceil(width / tile_w)``
    tiles a row) holding at least one pixel centre where it is blended:
    ``o~ exp(-q / 2) >= 1/255`` with ``q = d^T conic d`` and d the offset of
    the pixel centre (px + 0.5, py + 0.5) from ``uv`` (Sec. 3.1, with the
    1/255 skip of 3DGS), i.e. ``q <= 2 ln(255 o~)``.  ``shrink`` < 1 scales
    that level down, leaving out centres within rounding of the boundary.
    Brute force over every pixel; small images only."""
    uv = np.asarray(uv, np.float64).reshape(-1, 2)
    conic = np.asarray(conic, np.float64).reshape(-1, 3)
    ot = np.asarray(ot, np.float64).reshape(-1)
    tiles_x = (width + tile_w - 1) // tile_w
    py, px = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    tile = (py // tile_h) * tiles_x + px // tile_w
    cx, cy = px + 0.5, py + 0.5
    out = []
    for k in range(uv.shape[0]):
        if not ot[k] > 1.0 / 255.0:
            out.append(set())
            continue
        level = shrink * 2.0 * np.log(255.0 * ot[k])
        dx, dy = cx - uv[k, 0], cy - uv[k, 1]
        q = conic[k, 0] * dx * dx + 2.0 * conic[k, 1] * dx * dy + conic[k, 2] * dy * dy
        out.append(set(np.unique(tile[q <= level]).tolist()))
    return out

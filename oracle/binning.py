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

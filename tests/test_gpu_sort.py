"""The stable radix sort behind the depth and tile orders (Sec. 3.1:
Gaussians sorted by camera depth, per tile), bit-exact against numpy's
stable argsort, through the C ABI (pvg_sort_pairs).  GPU only."""
import numpy as np
import pytest
import torch

from paper_2311_18561_gb300 import render as R

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _check(renderer, keys_np, vals_np, begin, end):
    k = torch.from_numpy(keys_np.view(np.int32)).cuda()
    v = torch.from_numpy(vals_np.view(np.int32)).cuda()
    R.sort_pairs(renderer, k, v, begin, end)
    torch.cuda.synchronize()
    mask = np.uint64((1 << (end - begin)) - 1)
    sort_bits = (keys_np.astype(np.uint64) >> np.uint64(begin)) & mask
    order = np.argsort(sort_bits, kind="stable")
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint32), keys_np[order])
    np.testing.assert_array_equal(v.cpu().numpy().view(np.uint32), vals_np[order])


@pytest.fixture(scope="module")
def renderer():
    return R.Renderer()


@pytest.mark.parametrize("n", [0, 1, 7, 2047, 2048, 2049, 100_003])
@pytest.mark.parametrize("bits", [(0, 14), (0, 31), (0, 32), (3, 11), (0, 20)])
def test_sort_small_and_ragged(renderer, n, bits):
    rng = np.random.default_rng(n + 31 * bits[1])
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 3] = keys[0] if n else 0  # many equal keys: stability matters
    vals = np.arange(n, dtype=np.uint32)
    _check(renderer, keys, vals, *bits)


@pytest.mark.parametrize("width", range(1, 9))
def test_sort_every_last_digit_width(renderer, width):
    """A sort by 8 + width bits: the last digit pass has width 1..8 bits
    (each width ranks with its own number of ballots)."""
    rng = np.random.default_rng(40 + width)
    n = 300_001
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    keys[::5] = keys[3]
    _check(renderer, keys, np.arange(n, dtype=np.uint32), 0, 8 + width)
    _check(renderer, keys, np.arange(n, dtype=np.uint32), 5, 5 + width)


def test_sort_depth_keys_of_a_frame(renderer):
    """Positive float32 depths (31 significant bits), 2M of them."""
    rng = np.random.default_rng(1)
    z = rng.uniform(0.2, 300.0, 2_000_000).astype(np.float32)
    z[::7] = z[0]
    _check(renderer, z.view(np.uint32).copy(), np.arange(z.size, dtype=np.uint32), 0, 31)


def test_sort_tile_keys_full_size(renderer):
    """12M tile ids of a 1920x1280 frame (9600 tiles, 14 bits), values in
    depth order: the size of the urban benchmark's pair list."""
    rng = np.random.default_rng(2)
    keys = rng.integers(0, 9600, 12_000_000).astype(np.uint32)
    _check(renderer, keys, np.arange(keys.size, dtype=np.uint32), 0, 14)


@pytest.mark.parametrize("n,bits", [(13_000_000, (0, 17)), (20_000_017, (0, 32))])
def test_sort_long_with_late_value_reads(renderer, n, bits):
    """Sorts of 12M keys and more run the wide downsweep that reads the
    values late (four CTAs per SM): tile ids of a 64-view batch (17 bits,
    many equal keys) and full 32-bit keys with a ragged last tile."""
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2 ** bits[1], n, dtype=np.uint64).astype(np.uint32)
    keys[::9] = keys[4]
    _check(renderer, keys, np.arange(n, dtype=np.uint32), *bits)

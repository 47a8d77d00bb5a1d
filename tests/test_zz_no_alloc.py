"""pvg_sort_pairs_noalloc: the radix sort for callers that cannot allocate
device memory (graph capture, real-time threads, hosts with their own
memory pool).  Its output must equal the allocating entry point's
(pvg_sort_pairs) bit for bit -- the sort is integer work -- on two calls in
a row, the second with other data, other sizes and an odd number of digit
passes, so that contents left in the shared fixed scratch by the first call
cannot leak into the second.  Collected last (file name) so that a run
stopping at the first failure has run every other test.  GPU only."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2311_18561_gb300 import abi
from paper_2311_18561_gb300 import render as R

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

MAX_PAIRS = 1 << 20


def _noalloc(keys, vals, begin, end):
    st = abi.lib().pvg_sort_pairs_noalloc(keys.data_ptr(), vals.data_ptr(), keys.numel(), begin, end,
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    abi.check(st, "pvg_sort_pairs_noalloc")


def test_noalloc_sort_equals_allocating_sort_twice_in_a_row():
    renderer = R.Renderer()
    rng = np.random.default_rng(123)
    cases = [
        # (n, begin_bit, end_bit, key generator)
        (300_003, 0, 14, lambda n: rng.integers(0, 9600, n).astype(np.uint32)),          # 2 passes
        (MAX_PAIRS, 0, 20, lambda n: rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)),  # 3 passes
    ]
    for n, b, e, gen in cases:
        keys = gen(n)
        keys[: n // 4] = keys[0]  # long runs of equal keys: stability shows
        vals = rng.permutation(n).astype(np.uint32)
        k_ref = torch.from_numpy(keys.view(np.int32).copy()).cuda()
        v_ref = torch.from_numpy(vals.view(np.int32).copy()).cuda()
        k_new = k_ref.clone()
        v_new = v_ref.clone()
        R.sort_pairs(renderer, k_ref, v_ref, b, e)
        _noalloc(k_new, v_new, b, e)
        torch.cuda.synchronize()
        assert torch.equal(k_new, k_ref), (n, b, e)
        assert torch.equal(v_new, v_ref), (n, b, e)
        order = np.argsort((keys.astype(np.uint64) >> np.uint64(b)) & np.uint64((1 << (e - b)) - 1), kind="stable")
        np.testing.assert_array_equal(v_new.cpu().numpy().view(np.uint32), vals[order])
    renderer.close()


def test_noalloc_sort_rejects_sizes_beyond_its_maximum():
    k = torch.zeros(MAX_PAIRS + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros_like(k)
    st = abi.lib().pvg_sort_pairs_noalloc(k.data_ptr(), v.data_ptr(), k.numel(), 0, 8,
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1  # PVG_ERR_INVALID

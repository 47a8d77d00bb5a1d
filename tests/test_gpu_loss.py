"""Parity of the fused photometric loss (1 - lambda_r) L1 + lambda_r
(1 - SSIM) (Sec. 3.4) of the CUDA path with the FP64 oracle.  GPU only.

Tolerances (FP32 windowed sums against FP64): the loss, L1 and SSIM values
within 1e-5 relative (2e-6 absolute); the gradient within 1e-3 of its
largest magnitude per element and 1e-4 relative in norm.
"""
import numpy as np
import pytest
import torch

from oracle import loss as OL
from paper_2311_18561_gb300 import render as R

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def renderer():
    return R.Renderer()


def _images(shape, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, size=shape).astype(np.float32)
    # a target correlated with x, so that SSIM is far from 0 and 1
    y = np.clip(x + rng.normal(0, 0.15, size=shape), 0, 1).astype(np.float32)
    return x, y


def _check(renderer, x, y, lam):
    xt, yt = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
    loss, dl = R.rgb_loss(renderer, xt, yt, lambda_r=lam)
    torch.cuda.synchronize()
    L, l1, s, g = OL.rgb_loss(x, y, lambda_r=lam)
    got = loss.cpu().numpy().astype(np.float64)
    assert got[0] == pytest.approx(L, rel=1e-5, abs=2e-6)
    assert got[1] == pytest.approx(l1, rel=1e-5, abs=2e-6)
    assert got[2] == pytest.approx(s, rel=1e-5, abs=2e-6)
    d = dl.cpu().numpy().astype(np.float64)
    err = np.abs(d - g)
    assert err.max() <= 1e-3 * np.abs(g).max(), (err.max(), np.abs(g).max())
    assert np.linalg.norm(d - g) <= 1e-4 * np.linalg.norm(g)


@pytest.mark.parametrize("shape", [(3, 64, 48), (3, 45, 70), (1, 7, 5), (2, 33, 32), (3, 1, 40)])
@pytest.mark.parametrize("lam", [0.2, 0.0, 1.0])
def test_loss_matches_oracle(renderer, shape, lam):
    x, y = _images(shape, seed=sum(shape))
    _check(renderer, x, y, lam)


def test_loss_at_training_and_urban_resolutions(renderer):
    for shape, seed in (((3, 375, 1242), 1), ((3, 1280, 1920), 2)):
        x, y = _images(shape, seed)
        _check(renderer, x, y, 0.2)


def test_identical_images_and_determinism(renderer):
    x, _ = _images((3, 50, 61), 4)
    xt = torch.tensor(x, device="cuda")
    loss, dl = R.rgb_loss(renderer, xt, xt.clone())
    torch.cuda.synchronize()
    assert abs(loss[0].item()) < 1e-6 and loss[2].item() == pytest.approx(1.0, abs=1e-6)
    assert dl.abs().max().item() < 1e-9
    x, y = _images((3, 90, 77), 5)
    a = R.rgb_loss(renderer, torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"))
    b = R.rgb_loss(renderer, torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_loss_rejects_bad_arguments(renderer):
    x = torch.zeros(3, 8, 8, device="cuda")
    with pytest.raises(Exception):
        R.rgb_loss(renderer, x, x, lambda_r=1.5)
    with pytest.raises(Exception):
        R.rgb_loss(renderer, x, torch.zeros(3, 8, 9, device="cuda"))


@pytest.mark.parametrize("n", [1, 255, 257, 3 * 375 * 1242, 3 * 1280 * 1920])
def test_l1_loss_is_reproducible_and_matches_fp64(renderer, n):
    """pvg_l1_loss: the fixed-order sum gives the same loss bit for bit on
    every call (and from a second context), within 1e-6 relative of the FP64
    sum; the gradient is scale * sign(pred - target) exactly."""
    rng = np.random.default_rng(n)
    x = rng.uniform(0, 1, size=n).astype(np.float32)
    y = rng.uniform(0, 1, size=n).astype(np.float32)
    y[: n // 7] = x[: n // 7]  # equal entries: sign 0
    xt, yt = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
    other = R.Renderer()
    runs = [R.l1_loss(renderer, xt, yt)[0].clone() for _ in range(3)] + [R.l1_loss(other, xt, yt)[0].clone()]
    loss, dl = R.l1_loss(renderer, xt, yt)
    torch.cuda.synchronize()
    for r in runs:
        assert torch.equal(r, loss)
    ref = np.abs(x.astype(np.float64) - y.astype(np.float64)).sum() / n
    assert float(loss[0]) == pytest.approx(ref, rel=1e-6, abs=1e-9)
    d = x.astype(np.float64) - y.astype(np.float64)
    want = np.float32(1.0 / n) * np.sign(d).astype(np.float32)
    np.testing.assert_array_equal(dl.cpu().numpy(), want)
    other.close()


@pytest.mark.parametrize("n", [1003, 3 * 375 * 1242])
def test_l1_loss_of_unaligned_views(renderer, n):
    """Arrays that do not start on a 16-byte boundary take the kernel's
    one-element path (aligned ones take four elements at a time): the same
    loss within 1e-6 of the FP64 sum and the exact gradient."""
    rng = np.random.default_rng(n + 1)
    x = rng.uniform(0, 1, size=n + 1).astype(np.float32)
    y = rng.uniform(0, 1, size=n + 1).astype(np.float32)
    xt, yt = torch.tensor(x, device="cuda")[1:], torch.tensor(y, device="cuda")[1:]
    assert xt.data_ptr() % 16 != 0
    loss, dl = R.l1_loss(renderer, xt, yt)
    torch.cuda.synchronize()
    d = x[1:].astype(np.float64) - y[1:].astype(np.float64)
    assert float(loss[0]) == pytest.approx(np.abs(d).sum() / n, rel=1e-6, abs=1e-9)
    want = np.float32(1.0 / n) * np.sign(d).astype(np.float32)
    np.testing.assert_array_equal(dl.cpu().numpy(), want)


def test_l1_loss_of_nothing_is_zero(renderer):
    e = torch.empty(0, device="cuda")
    loss, _ = R.l1_loss(renderer, e, e)
    torch.cuda.synchronize()
    assert float(loss[0]) == 0.0

"""Pins of the oracle's photometric loss (1 - lambda_r) L1 + lambda_r L_ssim
(Sec. 3.4 loss, lambda_r = 0.2; SSIM with the 3DGS window).  No GPU.

* the window: symmetric, sums to 1, neighbouring taps in the ratio of the
  Gaussian;
* the separable zero-padded convolution equals scipy's 2-D convolution
  with the outer-product kernel, and a per-pixel brute-force SSIM written
  from the definition (explicit 11 x 11 window sums, no convolution);
* SSIM(x, x) = 1 with a zero gradient; SSIM is symmetric in its arguments;
  constant images give (2ab + C1) / (a^2 + b^2 + C1) away from the border;
  lambda_r = 0 and 1 reduce to L1 and 1 - SSIM;
* the gradient matches FP64 finite differences.
"""
import numpy as np
import pytest

from oracle import loss as OL


def test_window():
    g = OL.gaussian_window()
    assert len(g) == 11 and g.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(g, g[::-1], rtol=0, atol=0)
    assert g[5] / g[4] == pytest.approx(np.exp(1.0 / (2 * 1.5 ** 2)), rel=1e-14)
    assert g[5] / g[3] == pytest.approx(np.exp(4.0 / (2 * 1.5 ** 2)), rel=1e-14)


def test_conv_matches_scipy():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    img = rng.uniform(size=(2, 23, 31))
    g = OL.gaussian_window()
    k2 = np.outer(g, g)
    got = OL.conv_same(img, g)
    for c in range(2):
        ref = signal.convolve2d(img[c], k2, mode="same", boundary="fill", fillvalue=0.0)
        np.testing.assert_allclose(got[c], ref, rtol=0, atol=1e-14)


def _brute_ssim_pixel(x, y, r, c):
    g = OL.gaussian_window()
    w = np.outer(g, g)
    H, W = x.shape
    m = [0.0] * 5
    for i in range(-5, 6):
        for j in range(-5, 6):
            rr, cc = r + i, c + j
            if 0 <= rr < H and 0 <= cc < W:
                a, b, wt = x[rr, cc], y[rr, cc], w[i + 5, j + 5]
                m[0] += wt * a
                m[1] += wt * b
                m[2] += wt * a * a
                m[3] += wt * b * b
                m[4] += wt * a * b
    mx, my = m[0], m[1]
    vx, vy, cxy = m[2] - mx * mx, m[3] - my * my, m[4] - mx * my
    return ((2 * mx * my + OL.C1) * (2 * cxy + OL.C2)) / ((mx * mx + my * my + OL.C1) * (vx + vy + OL.C2))


def test_ssim_map_matches_brute_force():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(1, 17, 19))
    y = np.clip(x + rng.normal(0, 0.1, size=x.shape), 0, 1)
    S = OL.ssim_terms(x, y)[0][0]
    for r, c in [(0, 0), (3, 7), (8, 9), (16, 18), (10, 0), (0, 12)]:
        assert S[r, c] == pytest.approx(_brute_ssim_pixel(x[0], y[0], r, c), rel=1e-12, abs=1e-14)


def test_identity_symmetry_constants_and_limits():
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(3, 20, 24))
    y = rng.uniform(size=(3, 20, 24))
    L, l1, s, grad = OL.rgb_loss(x, x)
    assert L == pytest.approx(0.0, abs=1e-15) and s == pytest.approx(1.0, abs=1e-14)
    assert np.abs(grad).max() < 1e-15
    assert OL.ssim(x, y) == pytest.approx(OL.ssim(y, x), abs=1e-14)
    a, b = 0.3, 0.7
    S = OL.ssim_terms(np.full((1, 30, 30), a), np.full((1, 30, 30), b))[0][0]
    inner = S[5:-5, 5:-5]
    np.testing.assert_allclose(inner, (2 * a * b + OL.C1) / (a * a + b * b + OL.C1), rtol=1e-12)
    L0, l10, _, _ = OL.rgb_loss(x, y, lambda_r=0.0)
    assert L0 == pytest.approx(np.abs(x - y).mean(), rel=1e-15) and L0 == l10
    L1_, _, s1, _ = OL.rgb_loss(x, y, lambda_r=1.0)
    assert L1_ == pytest.approx(1.0 - s1, abs=1e-15)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.uniform(0.05, 0.95, size=(3, 14, 16))
    y = rng.uniform(0.05, 0.95, size=(3, 14, 16))
    L, _, _, grad = OL.rgb_loss(x, y)
    idx = [(0, 0, 0), (1, 7, 8), (2, 13, 15), (0, 3, 12), (1, 0, 9), (2, 10, 1)] + \
          [tuple(rng.integers(0, s) for s in x.shape) for _ in range(10)]
    for i in idx:
        if abs(x[i] - y[i]) < 1e-4:
            continue  # |x - y| has a kink there
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = (OL.rgb_loss(xp, y)[0] - OL.rgb_loss(xm, y)[0]) / (2 * h)
        assert grad[i] == pytest.approx(fd, rel=1e-6, abs=1e-11), i

"""FP64 oracle of the photometric training loss -- TEST INFRASTRUCTURE ONLY.

The paper supervises the RGB rendering with
    L = (1 - lambda_r) L_1 + lambda_r L_ssim,   lambda_r = 0.2
(Sec. 3.4, the loss equation and its implementation details), where L_1 and
L_ssim are the L1 and SSIM losses of 3D Gaussian Splatting.  The paper does
not restate them; this module takes the 3DGS reading:

  * L_1 = mean over channels and pixels of |x - y|;
  * L_ssim = 1 - SSIM, SSIM the mean over channels and pixels of the SSIM
    map of each channel, computed with an 11 x 11 Gaussian window
    (sigma = 1.5, normalised to sum 1) applied with zero padding ("same"
    size), C1 = 0.01^2, C2 = 0.03^2:
        S = (2 mu_x mu_y + C1)(2 s_xy + C2) /
            ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
    mu = G*x, s_x^2 = G*(x^2) - mu_x^2, s_xy = G*(x y) - mu_x mu_y;
  * the derivative of sign at 0 is 0.

dL/dx is the exact reverse mode: with m1 = G*x, m2 = G*(x^2),
m12 = G*(x y) (the window is symmetric, so its transpose is itself)
    dS/dx_p = sum_q G(q - p) [dS_q/dm1 + 2 x_p dS_q/dm2 + y_p dS_q/dm12].
Images are planar [C, H, W]; every function returns float64.
"""
from __future__ import annotations

import numpy as np

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA_R = 0.2


def gaussian_window(size=WINDOW, sigma=SIGMA):
    """1-D Gaussian taps exp(-(k - c)^2 / (2 sigma^2)), c = size // 2,
    normalised to sum 1."""
    k = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return g / g.sum()


def conv_same(img, g):
    """Separable 2-D convolution of the last two axes of img with the outer
    product g g^T, zero padding, output of the input's size."""
    img = np.asarray(img, np.float64)
    r = len(g) // 2
    H, W = img.shape[-2:]
    pad = np.zeros(img.shape[:-2] + (H + 2 * r, W + 2 * r))
    pad[..., r:r + H, r:r + W] = img
    rows = np.zeros(img.shape[:-2] + (H + 2 * r, W))
    for j in range(len(g)):  # along x
        rows += g[j] * pad[..., :, j:j + W]
    out = np.zeros(img.shape)
    for i in range(len(g)):  # along y
        out += g[i] * rows[..., i:i + H, :]
    return out


def ssim_terms(x, y):
    """SSIM map S [C,H,W] and its partial derivatives with respect to the
    windowed moments m1 = G*x, m2 = G*(x^2), m12 = G*(x y)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    g = gaussian_window()
    mx, my = conv_same(x, g), conv_same(y, g)
    exx, eyy, exy = conv_same(x * x, g), conv_same(y * y, g), conv_same(x * y, g)
    vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A1, A2 = 2 * mx * my + C1, 2 * cxy + C2
    B1, B2 = mx * mx + my * my + C1, vx + vy + C2
    S = A1 * A2 / (B1 * B2)
    # direct partials of S(mu_x, s_x^2, s_xy)
    dS_dmu = S * (2 * my / A1 - 2 * mx / B1)
    dS_dvx = -S / B2
    dS_dcxy = 2 * S / A2
    # through s_x^2 = m2 - m1^2 and s_xy = m12 - m1 mu_y
    d_m1 = dS_dmu - 2 * mx * dS_dvx - my * dS_dcxy
    d_m2 = dS_dvx
    d_m12 = dS_dcxy
    return S, d_m1, d_m2, d_m12


def ssim(x, y):
    return float(ssim_terms(x, y)[0].mean())


def rgb_loss(x, y, lambda_r=LAMBDA_R):
    """(L, L_1, SSIM, dL/dx) of (1 - lambda_r) L_1 + lambda_r (1 - SSIM)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    l1 = float(np.abs(x - y).mean())
    S, d_m1, d_m2, d_m12 = ssim_terms(x, y)
    s = float(S.mean())
    loss = (1.0 - lambda_r) * l1 + lambda_r * (1.0 - s)
    g = gaussian_window()
    dS_dx = conv_same(d_m1, g) + 2 * x * conv_same(d_m2, g) + y * conv_same(d_m12, g)
    grad = (1.0 - lambda_r) / n * np.sign(x - y) - lambda_r / n * dS_dx
    return loss, l1, s, grad

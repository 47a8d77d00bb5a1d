"""The geometry the tile binning relies on, in FP64 on the CPU: over a band
of rows, the ellipse a x^2 + 2 b x y + c y^2 <= Q spans exactly
[x_left(clamp(y_l)), x_right(clamp(-y_l))] with
x(y) = (-b y -+ sqrt(a Q - D y^2)) / a, D = ac - b^2, y_l = b sqrt(Q/(cD))
(the left edge is convex with its minimum at y_l, the right edge concave
with its maximum at -y_l).  Checked against brute force over dense rows.
No GPU."""
import numpy as np


def band_span(a, b, c, Q, lo, hi):
    D = a * c - b * b
    ym = np.sqrt(Q * a / D)
    lo, hi = max(lo, -ym), min(hi, ym)
    if lo > hi:
        return None
    yl = b * np.sqrt(Q / (c * D))
    y1 = min(max(yl, lo), hi)
    y2 = min(max(-yl, lo), hi)
    x1 = (-b * y1 - np.sqrt(max(a * Q - D * y1 * y1, 0.0))) / a
    x2 = (-b * y2 + np.sqrt(max(a * Q - D * y2 * y2, 0.0))) / a
    return x1, x2


def brute_span(a, b, c, Q, lo, hi, n=4001):
    ys = np.linspace(lo, hi, n)
    D = a * c - b * b
    disc = a * Q - D * ys * ys
    ok = disc >= 0
    if not ok.any():
        return None
    r = np.sqrt(disc[ok])
    return float(((-b * ys[ok] - r) / a).min()), float(((-b * ys[ok] + r) / a).max())


def test_band_spans_match_brute_force():
    rng = np.random.default_rng(0)
    for _ in range(400):
        # random covariance (long axis up to 40x the short one), any rotation
        s1, s2 = np.exp(rng.uniform(-1, 3)), np.exp(rng.uniform(-1, 3))
        th = rng.uniform(0, np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        cov = R @ np.diag([s1 * s1, s2 * s2]) @ R.T
        a, b2, c = np.linalg.inv(cov)[[0, 0, 1], [0, 1, 1]]
        Q = rng.uniform(0.1, 11.0)
        ext = np.sqrt(Q * cov[1, 1])
        lo = rng.uniform(-1.5 * ext, 1.2 * ext)
        hi = lo + rng.uniform(0.5, 2.0 * ext)
        got, want = band_span(a, b2, c, Q, lo, hi), brute_span(a, b2, c, Q, lo, hi)
        if want is None:
            assert got is None or got[1] - got[0] < 1e-6 * ext
            continue
        assert got is not None
        # the dense sampling can only under-estimate the extent
        tol = 1e-3 * max(ext, 1.0)
        assert got[0] <= want[0] + tol and got[1] >= want[1] - tol
        assert got[0] >= want[0] - 0.05 * max(ext, 1.0) and got[1] <= want[1] + 0.05 * max(ext, 1.0)


def test_span_contains_every_pixel_centre_inside():
    """Pixel centres (integer + 0.5 offsets) inside the ellipse fall in the
    band's span, for bands of 8 and 32 rows."""
    rng = np.random.default_rng(1)
    for _ in range(100):
        s1, s2 = np.exp(rng.uniform(0, 3)), np.exp(rng.uniform(0, 3))
        th = rng.uniform(0, np.pi)
        R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        cov = R @ np.diag([s1 * s1, s2 * s2]) @ R.T
        a, b2, c = np.linalg.inv(cov)[[0, 0, 1], [0, 1, 1]]
        Q = rng.uniform(1.0, 11.0)
        u, v = rng.uniform(0, 1, 2)
        for th_rows in (8, 32):
            for y0 in range(-80, 80, th_rows):
                py = np.arange(y0, y0 + th_rows) + 0.5 - v
                px = np.arange(-200, 200) + 0.5 - u
                X, Y = np.meshgrid(px, py)
                inside = a * X * X + 2 * b2 * X * Y + c * Y * Y <= Q
                span = band_span(a, b2, c, Q, py[0], py[-1])
                if not inside.any():
                    continue
                assert span is not None
                xs = X[inside]
                assert xs.min() >= span[0] - 1e-9 and xs.max() <= span[1] + 1e-9

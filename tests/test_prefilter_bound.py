"""The single-precision candidate prefilter of the neighbour passes never rejects a pair that
the exact FP64 test accepts (CPU emulation of the kernel's float arithmetic).

The kernels keep a candidate b of particle a when fma(dx, dx, dy*dy) <= bound in float32,
with dx = fl32(fl32(x_a - xmin) - fl32(x_b - xmin)); the bound adds twice the worst-case
rounding error for positions in [0, 2^B * 2h] to (2h)^2.  Here adversarial pairs sit just
inside r = 2h, far from the bounding-box corner, at every orientation.
"""
import numpy as np
import pytest


def prefilter_bound(h, B):
    u = 2.0 ** -24
    two_h = 2.0 * h
    L = float(1 << B) * two_h
    e = 2.0 * L * u + 2.0 * two_h * u + L * u
    err = 4.0 * two_h * e + 2.0 * e * e + 4.0 * u * two_h * two_h
    hi = two_h * two_h + 2.0 * err
    f = np.float32(hi)
    while float(f) < hi:
        f = np.nextafter(f, np.float32(1e30))
    return f


@pytest.mark.parametrize("h,B", [(0.3, 7), (0.5, 6), (0.3, 8), (0.1, 10)])
def test_prefilter_keeps_every_true_neighbour(h, B):
    rng = np.random.default_rng(B)
    bound = prefilter_bound(h, B)
    two_h = 2 * h
    L = (1 << B) * two_h
    m = 200000
    xa = rng.uniform(0.0, L, (m, 2))
    ang = rng.uniform(0, 2 * np.pi, m)
    r = two_h * (1.0 - rng.uniform(0, 1e-9, m))  # just inside the support
    xb = xa + np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
    ok = np.all((xb >= 0) & (xb <= L), axis=1)
    xa, xb = xa[ok], xb[ok]
    d = xa - xb
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
    inside = r2 < two_h * two_h
    fa = xa.astype(np.float32)  # xmin = 0 here: fl32(x - xmin) = fl32(x)
    fb = xb.astype(np.float32)
    dx = (fa[:, 0] - fb[:, 0]).astype(np.float32)
    dy = (fa[:, 1] - fb[:, 1]).astype(np.float32)
    p = (dy * dy).astype(np.float32)
    r2f = (dx.astype(np.float64) * dx.astype(np.float64) + p.astype(np.float64)).astype(np.float32)
    assert np.all(r2f[inside] <= bound)
    # and the margin stays small: the prefilter passes under 1 % more area than the exact test
    assert float(bound) / (two_h * two_h) - 1 < 1e-2


def prefilter_bounds(h, B):
    """(lo, hi): the same margin below and above (2h)^2 (float32, rounded outward)."""
    hi = prefilter_bound(h, B)
    two_h = 2.0 * h
    lo = two_h * two_h - (float(hi) - two_h * two_h)
    g = np.float32(lo)
    while float(g) > lo:
        g = np.nextafter(g, np.float32(0.0))
    return g, hi


@pytest.mark.parametrize("h,B", [(0.3, 7), (0.3, 10), (0.5, 6), (0.05, 12)])
def test_lower_bound_proves_neighbours(h, B):
    """A float r^2 below the lower bound proves r < 2h: pairs just outside the support never
    fall under it, so skipping the exact test for them keeps the neighbour set exact."""
    rng = np.random.default_rng(100 + B)
    lo, hi = prefilter_bounds(h, B)
    two_h = 2 * h
    L = (1 << B) * two_h
    m = 200000
    xa = rng.uniform(0.0, L, (m, 2))
    ang = rng.uniform(0, 2 * np.pi, m)
    r = two_h * (1.0 + rng.uniform(0, 1e-9, m))  # just outside (or on) the support
    xb = xa + np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
    ok = np.all((xb >= 0) & (xb <= L), axis=1)
    xa, xb = xa[ok], xb[ok]
    d = xa - xb
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
    outside = r2 >= two_h * two_h
    fa, fb = xa.astype(np.float32), xb.astype(np.float32)
    dx = (fa[:, 0] - fb[:, 0]).astype(np.float32)
    dy = (fa[:, 1] - fb[:, 1]).astype(np.float32)
    p = (dy * dy).astype(np.float32)
    r2f = (dx.astype(np.float64) * dx.astype(np.float64) + p.astype(np.float64)).astype(np.float32)
    assert np.all(r2f[outside] >= lo)
    assert lo < two_h * two_h < hi

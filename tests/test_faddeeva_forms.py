"""The approximations of Re w(x + i y) that the opacity kernel uses, written
out in FP64 and checked against SciPy's Faddeeva function over the regions
where the kernel applies each one, with the truncation bounds the kernel's
design relies on (the FP32 rounding of about ten operations comes on top and
is covered by the GPU tests):

* one-pole truncation of the Laplace continued fraction, |z| >= 24:
  Re w = (y / sqrt pi) (u + 1) / (u^2 + 2 y^2), u = x^2 + y^2 - 1/2;
  relative error <= 2.52 / |z|^4 <= 7.6e-6;
* the continued fraction to depth 4 (|z| >= 8) or 6 (5 <= |z| < 8) plus the
  Gaussian term exp(y^2 - x^2) cos(2 x y) near the real axis: <= 1e-7 and
  <= 5e-7 (depth 3 would give <= 1e-6 for |z| >= 8);
* the closed real form of the depth-2 fraction, 14 <= |z| < 24: <= 7.3e-7;
* the eight-term Taylor expansion about the nearest node of a grid of
  spacing 1/8 (|z - z0| <= 0.089), |z| < 5: <= 3e-7;
* the shifted Lorentz form (y / sqrt pi) / (x^2 + y^2 - 3/2): relative error
  (2 y^2 + 3/2) / (x^2 + y^2)^2 to leading order (at most 0.6% more), below
  2e-6 where the kernel uses it (x^2 + y^2 >= 1.001 sqrt((2 y^2 + 3/2) / 2e-6));
* its degree-5 expansion over a block of 16 G points about the block centre,
  for |x_c| >= 12 h (h the half-width of the block) where the shifted Lorentz
  form holds on the whole block: a further <= 2.6e-6.

A dropped term of a form, a wrong depth or a wrong coefficient of the
expansion's recurrence breaks its bound.  The Taylor coefficients are built
here from wofz at the nodes and the derivative recurrence
w' = -2 z w + 2i / sqrt(pi), w^(n+1) = -2 z w^(n) - 2 n w^(n-1)."""
import math

import numpy as np
import pytest

wofz = pytest.importorskip("scipy.special").wofz
SQRTPI = math.sqrt(math.pi)


def _grid(xs, ys):
    X, Y = np.meshgrid(xs, ys)
    return X.ravel(), Y.ravel()


def _ref(x, y):
    return wofz(x + 1j * y).real


def _near_axis():
    return np.array([1e-10, 1e-6, 1e-3])


def test_one_pole_form():
    x, y = _grid(np.linspace(0.0, 100.0, 2001), np.concatenate([_near_axis(), np.linspace(0.01, 100.0, 800)]))
    s = x * x + y * y
    m = (s >= 576.0) & (s <= 1e4)                 # beyond, FP64 rounding of the reference dominates
    x, y, s = x[m], y[m], s[m]
    u = s - 0.5
    rel = np.abs(y / SQRTPI * (u + 1.0) / (u * u + 2.0 * y * y) / _ref(x, y) - 1.0)
    assert np.all(rel <= 2.52 / (s * s))
    assert rel.max() <= 7.6e-6


def _cf(x, y, depth):
    z = x + 1j * y
    t = z.copy()
    for k in range(depth, 0, -1):
        t = z - 0.5 * k / t
    v = t.imag / (SQRTPI * np.abs(t) ** 2)
    g = y * y - x * x
    return v + np.where((y < 1.0) & (g > -87.0), np.exp(g) * np.cos(2.0 * x * y), 0.0)


@pytest.mark.parametrize("lo,hi,depth,bound", [(8.0, 24.0, 4, 1e-7), (5.0, 8.0, 6, 5e-7), (8.0, 24.0, 3, 1e-6)])
def test_continued_fraction_with_gaussian_term(lo, hi, depth, bound):
    x, y = _grid(np.linspace(0.0, 24.0, 961), np.concatenate([_near_axis(), np.linspace(0.02, 24.0, 480)]))
    s = x * x + y * y
    m = (s >= lo * lo) & (s < hi * hi)
    assert np.max(np.abs(_cf(x[m], y[m], depth) / _ref(x[m], y[m]) - 1.0)) <= bound


def test_closed_depth_two_form():
    x, y = _grid(np.linspace(0.0, 24.0, 1201), np.concatenate([_near_axis(), np.linspace(0.02, 24.0, 600)]))
    s = x * x + y * y
    m = (s >= 196.0) & (s < 576.0)
    x, y = x[m], y[m]
    x2, y2 = x * x, y * y
    u, v2 = x2 - y2, 4.0 * x2 * y2
    um = u - 1.5
    re = y * (x2 + v2 + (u - 1.0) * um) / (SQRTPI * (x2 + y2) * (um * um + v2))
    assert np.max(np.abs(re / _ref(x, y) - 1.0)) <= 7.3e-7


def test_taylor_table_form():
    H, NT = 0.125, 8
    x, y = _grid(np.linspace(0.0, 5.0, 641), np.linspace(0.0, 5.0, 641))
    m = x * x + y * y < 25.0
    x, y = x[m], y[m]
    ix = np.minimum((x / H + 0.5).astype(int), 40)
    iy = np.minimum((y / H + 0.5).astype(int), 40)
    z0 = ix * H + 1j * iy * H
    dz = (x + 1j * y) - z0
    assert np.abs(dz).max() <= 0.089
    c = [wofz(z0), None]
    c[1] = -2.0 * z0 * c[0] + 2j / SQRTPI
    for n in range(1, NT - 1):
        c.append((-2.0 * z0 * c[n] - 2.0 * c[n - 1]) / (n + 1))
    acc = c[NT - 1]
    for n in range(NT - 2, -1, -1):
        acc = acc * dz + c[n]
    assert np.max(np.abs(acc.real / _ref(x, y) - 1.0)) <= 3e-7


def test_shifted_lorentz_form():
    x, y = _grid(np.concatenate([np.linspace(0.0, 100.0, 1001), np.geomspace(100.0, 1e4, 200)]),
                 np.concatenate([_near_axis(), np.geomspace(0.05, 300.0, 300)]))
    s = x * x + y * y
    bound = (2.0 * y * y + 1.5) / (s * s)
    m = s >= 1.001 * np.sqrt((2.0 * y * y + 1.5) / 2e-6)     # the kernel's selection of the form
    x, y, s, bound = x[m], y[m], s[m], bound[m]
    rel = np.abs(y / SQRTPI / (s - 1.5) / _ref(x, y) - 1.0)
    assert np.all(rel <= 1.006 * bound + 1e-13)
    assert rel.max() <= 2e-6


def test_degree_five_expansion_of_the_shifted_lorentz_term():
    rng = np.random.default_rng(3)
    worst, cases = 0.0, 0
    for _ in range(6000):
        G = int(rng.choice([1, 2, 4, 8]))
        dx = 10 ** rng.uniform(-3.5, 0.5)
        y = 10 ** rng.uniform(-5, 2)
        h = (16 * G - 1) * dx / 2
        xc = rng.choice([-1.0, 1.0]) * 12.0 * h * 10 ** rng.uniform(0.0, 1.0)
        t = np.arange(16 * G) - (16 * G - 1) / 2
        x = xc + t * dx
        if np.any((2 * y * y + 1.5) / (x * x + y * y) ** 2 > 2e-6):
            continue                               # the kernel expands only where the form holds
        cases += 1
        s = xc * xc + y * y - 1.5
        alpha, beta = 2.0 * xc * dx / s, dx * dx / s
        P = [1.0, -alpha]
        for _n in range(2, 6):
            P.append(-alpha * P[-1] - beta * P[-2])
        poly = sum(P[n] * t ** n for n in range(6)) / s
        exact = 1.0 / (s + 2.0 * xc * dx * t + dx * dx * t * t)
        worst = max(worst, float(np.max(np.abs(poly / exact - 1.0))))
    assert cases > 1000
    assert worst <= 2.6e-6

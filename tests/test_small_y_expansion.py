"""The small-y form of Re w that the opacity kernel uses for lines with
y <= 0.02 (Doppler-dominated cells), checked on the CPU against SciPy's
Faddeeva function: the expansion of Re w(x + i y) in y about the real axis,

  Re w = e^{-x^2} (1 + y^2 (1 - 2 x^2)) + y G(x)
         + (y^3 / 6) (4 / sqrt(pi) + G(x) (6 - 4 x^2)),  G = -Im w'(x),

with G and e^{-x^2} below x = 5 from the real-axis Taylor coefficients of w
(derived here independently, from wofz and the derivative recurrence
w' = -2 z w + 2i / sqrt(pi)), above x = 5 from the asymptotic series of G
and a compensated exponent; the y^3 term only below x = 40 (its bracket
4 / sqrt(pi) + G (6 - 4 x^2) cancels like x^2 eps in FP32, and a line's
fixup range can reach its cutoff edge, thousands of Doppler widths out).  The arithmetic is emulated in FP32 step by
step as the kernel performs it, which pins the relative error bound stated
for the kernel (2.3e-6) and catches a dropped or mis-signed term."""
import math

import numpy as np
import pytest

wofz = pytest.importorskip("scipy.special").wofz

F32 = np.float32
H = 0.125          # node spacing of the Taylor table
NT = 8             # terms per node
SQRTPI = math.sqrt(math.pi)


def _real_axis_coefficients(x0):
    """Taylor coefficients c_n = w^(n)(x0) / n! on the real axis (FP64)."""
    z0 = complex(x0, 0.0)
    c = [complex(math.exp(-x0 * x0), wofz(z0).imag)]
    c.append(-2.0 * z0 * c[0] + 2j / SQRTPI)
    for n in range(1, NT - 1):
        c.append((-2.0 * z0 * c[n] - 2.0 * c[n - 1]) / (n + 1))
    return np.array(c, dtype=np.complex64)


TABLE = {ix: _real_axis_coefficients(ix * H) for ix in range(41)}
# (2k-1)!! / 2^k, k = 1 .. 10
SERIES = [1.0]
for k in range(1, 11):
    SERIES.append(SERIES[-1] * (2 * k - 1) / 2.0)


def small_y_re(x, y):
    """FP32 emulation of the kernel's evaluation (ex2 taken as exact)."""
    x, y = F32(abs(x)), F32(y)
    if x < 5.0:
        ix = min(int(x * F32(1.0 / H) + F32(0.5)), 40)
        a = F32(x - F32(ix * H))
        c = TABLE[ix]
        r = F32(c[NT - 1].real)
        d = F32(F32(NT - 1) * F32(c[NT - 1].imag))
        for n in range(NT - 2, 0, -1):
            r = F32(r * a + F32(c[n].real))
            d = F32(d * a + F32(n) * F32(c[n].imag))
        e = F32(r * a + F32(c[0].real))
        g = F32(-d)
    else:
        l2e = F32(1.4426950408889634)
        l2e_lo = F32(1.4426950408889634 - float(l2e))
        hi = F32(x * x)
        lo = F32(float(x) * float(x) - float(hi))
        ah = F32(-hi * l2e)
        al = F32(-(float(hi) * float(l2e) + float(ah)) - float(lo) * float(l2e) - float(hi) * float(l2e_lo))
        e = F32(F32(2.0 ** float(ah)) * F32(1.0 + al * F32(0.6931471805599453)))
        t = F32(F32(1.0) / hi)
        s = F32(SERIES[10])
        for k in range(9, 0, -1):
            s = F32(s * t + F32(SERIES[k]))
        g = F32(F32(2.0 / SQRTPI) * t * s)
    x2, y2 = F32(x * x), F32(y * y)
    cub = F32(g * F32(6.0 - 4.0 * x2) + F32(4.0 / SQRTPI)) if x < 40.0 else F32(0.0)
    gy = F32(y2 * F32(1.0 / 6.0)) * cub + g
    return float(F32(e * F32(F32(1.0) + y2 * F32(1.0 - 2.0 * x2)) + y * F32(gy)))


def test_small_y_form_against_wofz():
    worst = 0.0
    xs = np.concatenate([np.linspace(0.0, 7.0, 1401), np.linspace(7.0, 40.0, 167), np.geomspace(40.0, 5000.0, 120)])
    for y in (1e-10, 1e-8, 1e-6, 1e-4, 1e-3, 5e-3, 1e-2, 2e-2):
        for x in xs:
            ref = wofz(complex(x, y)).real
            worst = max(worst, abs(small_y_re(x, y) - ref) / ref)
    print(f"small-y form: max relative error {worst:.2e}")
    assert worst < 2.5e-6


def test_small_y_form_needs_every_term():
    """The terms of the expansion matter on its range: without the y^3 term
    the error at y = 0.02 reaches ~8e-5 (near x = 2.9), and with G from
    2 x F(x) - 1 evaluated in FP32 (cancellation) instead of the table's
    derivative coefficients the far wings lose their accuracy."""
    dawsn = pytest.importorskip("scipy.special").dawsn
    y = 0.02
    worst_cubic = 0.0
    for x in np.linspace(0.0, 40.0, 801):
        g = 2 / SQRTPI * (2 * x * dawsn(x) - 1)
        cubic = y ** 3 / 6 * (4 / SQRTPI + g * (6 - 4 * x * x))
        ref = wofz(complex(x, y)).real
        worst_cubic = max(worst_cubic, abs(small_y_re(x, y) - cubic - ref) / ref)
    assert worst_cubic > 5e-5
    # G from Dawson's integral in FP32: 2 x F - 1 cancels to ~1/(2 x^2)
    x = 4.9
    f32_g = float(F32(2.0 / SQRTPI) * (F32(2.0) * F32(x) * F32(dawsn(x)) - F32(1.0)))
    exact_g = 2 / SQRTPI * (2 * x * dawsn(x) - 1)
    assert abs(f32_g - exact_g) / abs(exact_g) > 1e-6

"""Pins of the oracle's Voigt profile (Sec. 6.1.1, Eqs. 2-11) to its limits,
its normalisation and a brute-force convolution integral."""
import numpy as np
import pytest
from scipy import integrate

from oracle import voigt as V


def test_gaussian_limit():
    # gamma -> 0: V -> G (Eq. 2)
    sig = 0.01
    d = np.linspace(-6 * sig, 6 * sig, 241)
    v = V.voigt(d, sig, 1e-16 * sig)
    g = V.gaussian(d, sig)
    assert np.max(np.abs(v - g) / g) < 1e-9


def test_lorentz_limit():
    # sigma -> 0: V -> L (Eq. 3)
    gam = 0.07
    d = np.linspace(-100 * gam, 100 * gam, 401)
    v = V.voigt(d, 1e-7 * gam, gam)
    lz = V.lorentzian(d, gam)
    assert np.max(np.abs(v - lz) / lz) < 1e-6


@pytest.mark.parametrize("sig,gam", [(0.005, 1e-6), (0.005, 0.005), (0.002, 0.3)])
def test_unit_area(sig, gam):
    # Integral over +-X: 1 minus the Lorentzian tail mass beyond X, (2/pi) atan(gam/X)
    X = 2000.0 * max(sig, gam)
    val, _ = integrate.quad(lambda x: V.voigt(x, sig, gam), -X, X, points=[0.0],
                            limit=2000, epsabs=0, epsrel=1e-11)
    tail = 2.0 / np.pi * np.arctan(gam / X)
    assert abs(val + tail - 1.0) < 1e-7


def test_truncated_lorentz_mass():
    # With a 25 cm^-1 cutoff a pure Lorentzian keeps (2/pi) atan(25/gamma).
    gam = 0.08
    val, _ = integrate.quad(lambda x: V.voigt(x, 1e-9, gam), -25, 25, points=[0.0],
                            limit=2000, epsrel=1e-12)
    assert abs(val - 2 / np.pi * np.arctan(25 / gam)) < 1e-8


def _convolution(nu, sig, gam):
    # Eq. 10 written out: integral G(nu'; sigma) L(nu - nu'; gamma) dnu'
    f = lambda t: V.gaussian(t, sig) * V.lorentzian(nu - t, gam)
    lim = 12 * sig
    val, _ = integrate.quad(f, -lim, lim, points=sorted({0.0, float(np.clip(nu, -lim, lim))}),
                            limit=4000, epsabs=0, epsrel=1e-12)
    return val


@pytest.mark.parametrize("x", [0.0, 0.3, 1.0, 2.5, 4.0, 7.0, 20.0])
@pytest.mark.parametrize("y", [1e-3, 0.1, 1.0, 5.0])
def test_faddeeva_vs_brute_force_convolution(x, y):
    sig = 1.0 / np.sqrt(2.0)          # then z = nu + i gamma
    nu, gam = x, y
    ref = _convolution(nu, sig, gam)
    # the Gaussian factor is negligible beyond 12 sigma; the Lorentz mass
    # outside is accounted for by comparing relative to the peak scale
    got = V.voigt(nu, sig, gam)
    assert abs(got - ref) <= 1e-8 * got + 1e-12 * V.voigt(0.0, sig, gam)


@pytest.mark.parametrize("x,y", [(0.0, 1e-3), (0.7, 0.05), (2.2, 0.6), (5.5, 2.0), (30.0, 0.3), (1.3, 8.0)])
def test_faddeeva_re_is_the_voigt_function(x, y):
    # Re w(x + i y) = K(x, y) = (y / pi) int exp(-t^2) / ((x - t)^2 + y^2) dt,
    # by quadrature; on the real axis K(x, 0) = exp(-x^2).
    f = lambda t: np.exp(-t * t) / ((x - t) ** 2 + y * y)
    val, _ = integrate.quad(f, -12.0, 12.0, points=sorted({0.0, min(x, 11.9)}), limit=4000,
                            epsabs=0, epsrel=1e-12)
    k = y / np.pi * val
    assert abs(V.faddeeva_re(x, y) / k - 1) < 1e-9
    assert abs(V.faddeeva_re(x, 0.0) - np.exp(-x * x)) <= 1e-15 * max(np.exp(-x * x), 1e-300)

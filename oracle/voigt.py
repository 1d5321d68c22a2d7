"""Voigt line profile (Sec. 6.1.1, test f04broadening, Eqs. 2-11).

G(nu; sigma) = exp(-nu^2 / 2 sigma^2) / (sigma sqrt(2 pi))        (Eq. 2)
L(nu; gamma) = gamma / (pi (nu^2 + gamma^2))                       (Eq. 3)
V(nu; sigma, gamma) = Re w(z) / (sigma sqrt(2 pi)),
z = (nu + i gamma) / (sigma sqrt 2)                                (Eqs. 4-11)

w(z) is the Faddeeva function.  As in the paper's own test suite, its reference
value is scipy.special.wofz.
"""
import numpy as np
from scipy.special import wofz

SQRT2 = np.sqrt(2.0)
SQRT2PI = np.sqrt(2.0 * np.pi)


def faddeeva_re(x, y):
    """Re w(x + i y), the Voigt function K(x, y), in FP64."""
    return wofz(np.asarray(x, np.float64) + 1j * np.asarray(y, np.float64)).real


def voigt(dnu, sigma, gamma):
    """V(dnu; sigma, gamma) in units of 1/cm^-1 (Eqs. 4-11)."""
    dnu = np.asarray(dnu, np.float64)
    z = (dnu + 1j * gamma) / (sigma * SQRT2)
    return wofz(z).real / (sigma * SQRT2PI)


def gaussian(dnu, sigma):
    """Eq. 2."""
    dnu = np.asarray(dnu, np.float64)
    return np.exp(-dnu * dnu / (2.0 * sigma * sigma)) / (sigma * SQRT2PI)


def lorentzian(dnu, gamma):
    """Eq. 3."""
    dnu = np.asarray(dnu, np.float64)
    return gamma / (np.pi * (dnu * dnu + gamma * gamma))

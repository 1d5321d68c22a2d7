"""Emission (eclipse) radiative transfer, band integration and quadrature.

The paper implements the emergent-ray geometry of an eclipse observation
(Sec. 3) and tests it against closed forms: the isothermal atmosphere emits the
Planck function (test f08isothermal, Sec. 6.1.3) and the optically thin line
depth scales with abundance (test f05abundance, Sec. 6.1.2, Eqs. 12-13).  The
discretisation itself is in the companion paper (its Eqs. 14-18); the reading
taken here makes the isothermal case exact:

* levels k = 0 (top) .. L-1 (bottom), tau_0 = 0,
  dtau_k = (chi_k + chi_{k+1}) / 2 * (P_{k+1} - P_k) / g     (chi in cm^2 g^-1);
* I(mu) = sum_k (B_k + B_{k+1}) / 2 * (t_k - t_{k+1}) + B_{L-1} t_{L-1},
  t_k = exp(-tau_k / mu): layer-averaged source, blackbody interior below the
  deepest level, no incident or reflected starlight;
* F = 2 pi sum_i w_i mu_i I(mu_i), Gauss-Legendre nodes on mu in [0, 1];
* B is the Planck function per unit wavenumber,
  B(nu, T) = 2 h c^2 nu^3 / (exp(c2 nu / T) - 1)  [erg s^-1 cm^-2 sr^-1 (cm^-1)^-1].

Band values are trapezoid-weighted means of the spectrum over a filter's
transmission curve on the wavenumber grid (the spectrum integrator, Sec. 3).
"""
import math
import numpy as np

from .constants import H_PLANCK, C_LIGHT, C2, BAR


def planck(nu, T):
    """B(nu, T) per unit wavenumber (nu in cm^-1)."""
    nu = np.asarray(nu, np.float64)
    return 2.0 * H_PLANCK * C_LIGHT ** 2 * nu ** 3 / np.expm1(C2 * nu / T)


def gauss_legendre_mu(n):
    """Nodes and weights of n-point Gauss-Legendre quadrature on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def optical_depth(chi, p_bar, g):
    """tau at each level [.., L] from opacity chi[.., L] (cm^2 g^-1)."""
    chi = np.asarray(chi, np.float64)
    dp = np.diff(np.asarray(p_bar, np.float64) * BAR)
    dtau = 0.5 * (chi[..., :-1] + chi[..., 1:]) * dp / g
    tau = np.zeros(chi.shape)
    tau[..., 1:] = np.cumsum(dtau, axis=-1)
    return tau


def intensity(tau, B, mu):
    """I(mu) from tau[L] and B[L] (or [.., L] arrays, levels last)."""
    t = np.exp(-np.asarray(tau) / mu)
    Bbar = 0.5 * (B[..., :-1] + B[..., 1:])
    return np.sum(Bbar * (t[..., :-1] - t[..., 1:]), axis=-1) + B[..., -1] * t[..., -1]


def emission_flux(chi, p_bar, T, nu, g, n_angles, tau_max=None):
    """Planetary flux F(nu) for chi[L][n_nu], T[L]; returns FP64 [n_nu].

    tau_max (Sec. 4 item 7, the integration goes down to a chosen optical depth):
    at each wavenumber the integration stops at the first level whose vertical
    optical depth exceeds tau_max, and that level is the bottom boundary (its
    blackbody seen through the layers above)."""
    tau = optical_depth(np.asarray(chi).T, p_bar, g)           # [n_nu][L]
    B = planck(np.asarray(nu)[:, None], np.asarray(T)[None, :])  # [n_nu][L]
    mu, w = gauss_legendre_mu(n_angles)
    F = np.zeros(len(nu))
    if tau_max is None:
        for i in range(n_angles):
            F += w[i] * mu[i] * intensity(tau, B, mu[i])
        return 2.0 * math.pi * F
    L = tau.shape[1]
    for r in range(len(nu)):
        over = np.nonzero(tau[r, 1:] > tau_max)[0]
        k = over[0] + 1 if over.size else L - 1
        for i in range(n_angles):
            F[r] += w[i] * mu[i] * intensity(tau[r, :k + 1], B[r, :k + 1], mu[i])
    return 2.0 * math.pi * F


def trapezoid_weights(n):
    """Trapezoid weights (in units of the grid step) on n uniform points."""
    w = np.ones(n)
    if n >= 1:
        w[0] = 0.5
        w[-1] = 0.5
    if n == 1:
        w[0] = 1.0
    return w


def band_integrate(spec, filters, nu_lo=0):
    """Band means sum_j W_bj F_j dw_j / sum_j W_bj dw_j on the span starting at
    grid index nu_lo with len(spec) points; filters are [n_bands][n_nu_grid].
    A band whose weight sum over the span is zero yields 0."""
    spec = np.asarray(spec, np.float64)
    n = spec.size
    dw = trapezoid_weights(n)
    W = np.asarray(filters, np.float64)[:, nu_lo:nu_lo + n]
    num = np.array([math.fsum(W[b] * spec * dw) for b in range(W.shape[0])])
    den = np.array([math.fsum(W[b] * dw) for b in range(W.shape[0])])
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)


def emission_contributions(chi, p_bar, T, nu, g, n_angles, tau_max=None):
    """Contribution functions of the emission spectrum (post-processing, Sec. 3),
    FP64 [L][n_nu].

    Reading: the flux is a sum of one term per layer plus the bottom boundary,
    F = sum_{k < kb} C_k + C_kb, with
    C_k = 2 pi sum_i w_i mu_i (B_k + B_{k+1}) / 2 (t_k(mu_i) - t_{k+1}(mu_i))
    the emission of the layer between levels k and k+1 that reaches the top,
    and C_kb = 2 pi sum_i w_i mu_i B_kb t_kb(mu_i) the bottom level's blackbody
    seen through the column; kb is the last level integrated (L - 1, or the
    level where the optical-depth limit stops).  Entries after kb are 0."""
    tau = optical_depth(np.asarray(chi).T, p_bar, g)           # [n_nu][L]
    B = planck(np.asarray(nu)[:, None], np.asarray(T)[None, :])  # [n_nu][L]
    mu, w = gauss_legendre_mu(n_angles)
    n_nu, L = tau.shape
    C = np.zeros((L, n_nu))
    for r in range(n_nu):
        kb = L - 1
        if tau_max is not None:
            over = np.nonzero(tau[r, 1:] > tau_max)[0]
            kb = over[0] + 1 if over.size else L - 1
        for i in range(n_angles):
            t = np.exp(-tau[r, :kb + 1] / mu[i])
            C[:kb, r] += w[i] * mu[i] * 0.5 * (B[r, :kb] + B[r, 1:kb + 1]) * (t[:-1] - t[1:])
            C[kb, r] += w[i] * mu[i] * B[r, kb] * t[kb]
    return 2.0 * math.pi * C

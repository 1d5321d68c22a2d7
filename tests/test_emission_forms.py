"""The emission kernel's rearrangements of the radiative transfer, written
out in FP64 and checked against the oracle's plain definitions (Sec. 3 with
the layer-averaged source; the isothermal case exact, Sec. 6.1.3):

* angle-summed transmittance: instead of one intensity per Gauss-Legendre
  angle, the kernel keeps Tw_k = sum_i (2 pi w_i mu_i / 2) t_i(k) with
  t_i(k) = 2^(tau_k a_i), a_i = -log2(e) / mu_i, from the running vertical
  optical depth, and forms
    F = sum_{k>=1} (B_{k-1} + B_k) (Tw_{k-1} - Tw_k) + 2 B_bottom Tw_bottom,
  the same sum as 2 pi sum_i w_i mu_i I(mu_i) regrouped;
* the Planck function of a wavenumber pair (nu_a, nu_b = nu_a + dnu) from one
  exponential and one reciprocal: e_a = 2^(nu_a y), e_b = e_a r with
  y = (c2 / T) log2(e), r = 2^(y dnu),
    B_a = c1 nu_a^3 (e_b - 1) R,  B_b = c1 nu_b^3 (e_a - 1) R,
    R = 1 / ((e_a - 1)(e_b - 1)),
  with c1 = 2 h c^2 per unit wavenumber.
Both are exact identities, so they agree with the oracle to rounding."""
import math

import numpy as np

from oracle import radiation as R

H_PLANCK = 6.62607015e-27      # erg s (CODATA 2018, exact)
C_LIGHT = 2.99792458e10        # cm s^-1 (exact)
K_B = 1.380649e-16             # erg K^-1 (exact)


def _atmosphere(seed, L=50, n_nu=17):
    rng = np.random.default_rng(seed)
    p = np.logspace(-6, 2, L)
    T = rng.uniform(600.0, 2400.0, L)
    nu = np.linspace(1000.0, 3000.0, n_nu)
    chi = 10 ** rng.uniform(-4, 1, (L, n_nu))
    return p, T, nu, chi


def test_angle_summed_transmittance_regroups_the_flux():
    g = 2182.73
    for seed, n_angles in ((1, 1), (2, 4), (3, 8), (4, 16)):
        p, T, nu, chi = _atmosphere(seed)
        tau = R.optical_depth(chi.T, p, g)                      # [n_nu][L]
        B = R.planck(nu[:, None], T[None, :])
        mu, w = R.gauss_legendre_mu(n_angles)
        a = -math.log2(math.e) / mu                             # log2 transmittance per unit tau
        Tw = sum(math.pi * w[i] * mu[i] * np.exp2(tau * a[i]) for i in range(n_angles))
        F = np.sum((B[:, :-1] + B[:, 1:]) * (Tw[:, :-1] - Tw[:, 1:]), axis=1) + 2.0 * B[:, -1] * Tw[:, -1]
        ref = R.emission_flux(chi, p, T, nu, g, n_angles)
        assert np.max(np.abs(F / ref - 1)) < 1e-12


def test_planck_pair_from_one_exponential_and_one_reciprocal():
    c1 = 2.0 * H_PLANCK * C_LIGHT ** 2
    c2 = H_PLANCK * C_LIGHT / K_B
    dnu = 0.02
    nu_a = np.arange(1000.0, 3000.0, 7.77)
    nu_b = nu_a + dnu
    for T in (300.0, 500.0, 1200.0, 3000.0):
        y = c2 / T * math.log2(math.e)
        r = 2.0 ** (y * dnu)
        ea = np.exp2(nu_a * y)
        eb = ea * r
        Rr = 1.0 / ((ea - 1.0) * (eb - 1.0))
        Ba = c1 * nu_a ** 3 * (eb - 1.0) * Rr
        Bb = c1 * nu_b ** 3 * (ea - 1.0) * Rr
        assert np.max(np.abs(Ba / R.planck(nu_a, T) - 1)) < 1e-12
        assert np.max(np.abs(Bb / R.planck(nu_b, T) - 1)) < 1e-12

"""Pins of the oracle's emission RT, Planck function, quadrature and band
integration: f08isothermal (Sec. 6.1.3), f05abundance (Sec. 6.1.2, Eqs. 12-13,
the varying-abundance table), Stefan-Boltzmann and Wien laws."""
import json
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import radiation as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SIGMA_SB = 5.670374419e-5          # erg cm^-2 s^-1 K^-4 (CODATA 2018)
WIEN_X = 2.821439372122079         # peak of x^3/(e^x - 1)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_gauss_legendre_exactness(n):
    mu, w = R.gauss_legendre_mu(n)
    for k in range(2 * n):
        assert abs(np.sum(w * mu ** k) - 1.0 / (k + 1)) < 1e-14
    assert np.all((mu > 0) & (mu < 1))


def test_isothermal_emits_planck():
    # Without scattering an isothermal atmosphere emits pi B(T) for any opacity.
    rng = np.random.default_rng(3)
    p = np.logspace(-6, 2, 60)
    nu = np.linspace(1000, 3000, 37)
    chi = 10 ** rng.uniform(-4, 4, (60, 37))
    for n_ang in (1, 4, 8):
        F = R.emission_flux(chi, p, np.full(60, 1234.5), nu, 2182.73, n_ang)
        exp = np.pi * R.planck(nu, 1234.5)
        assert np.max(np.abs(F / exp - 1)) < 1e-12


def test_transparent_atmosphere_shows_interior():
    p = np.logspace(-6, 2, 30)
    T = np.linspace(600, 1700, 30)
    nu = np.linspace(1000, 3000, 11)
    F = R.emission_flux(np.zeros((30, 11)), p, T, nu, 2182.73, 4)
    assert np.max(np.abs(F / (np.pi * R.planck(nu, 1700.0)) - 1)) < 1e-13


def _thin_layer_flux(tau_layer, n_ang, B_top=1.0, B_bot=3.0):
    # two levels: a single layer of optical depth tau over a hot interior
    chi = np.array([[tau_layer], [tau_layer]])       # dtau = chi * dP / g with dP/g = 1
    p = np.array([0.0, 1e-6])                        # bar -> dP = 1 dyn cm^-2
    g = 1.0
    tau = R.optical_depth(chi.T, p, g)
    mu, w = R.gauss_legendre_mu(n_ang)
    B = np.array([[B_top, B_bot]])
    return 2 * np.pi * sum(w[i] * mu[i] * R.intensity(tau, B, mu[i])[0] for i in range(n_ang))


def test_f05_thin_layer_ratio_closed_form():
    # Per angle F0 - F = (Bbar - B_bot)(1 - exp(-tau/mu)) with Bbar the layer mean,
    # so f(n) = sum w mu (1 - e^{-n tau/mu}) / sum w mu (1 - e^{-tau/mu}).
    mu, w = R.gauss_legendre_mu(4)
    tau = 2e-5
    F0 = _thin_layer_flux(0.0, 4)
    Fl = _thin_layer_flux(tau, 4)
    for n in range(2, 11):
        Fh = _thin_layer_flux(n * tau, 4)
        f = (F0 - Fh) / (F0 - Fl)
        closed = np.sum(w * mu * -np.expm1(-n * tau / mu)) / np.sum(w * mu * -np.expm1(-tau / mu))
        assert abs(f - closed) < 1e-9


def test_f05_trend_matches_paper_table():
    # The varying-abundance table (f05abundance) prints f slightly below the abundance ratio n with
    # a deficit growing with n; the thin-layer law gives the same signature.
    with open(os.path.join(GOLDEN, "f05_abundance_table.json")) as fh:
        table = json.load(fh)["f_vs_0.01pct"]
    n_vals = sorted(int(k) for k in table)
    deficits = [n - table[str(n)] for n in n_vals]
    assert all(d > 0 for d in deficits) and all(np.diff(deficits) > 0)
    tau = 1e-4
    F0, Fl = _thin_layer_flux(0.0, 4), _thin_layer_flux(tau, 4)
    ours = [n - (F0 - _thin_layer_flux(n * tau, 4)) / (F0 - Fl) for n in n_vals]
    assert all(d > 0 for d in ours) and all(np.diff(ours) > 0)
    assert max(abs(d) / n for d, n in zip(deficits, n_vals)) < 1e-3   # "closely obey"


@pytest.mark.parametrize("T", [300.0, 1000.0, 2500.0])
def test_planck_integral_stefan_boltzmann(T):
    val, _ = integrate.quad(lambda nu: R.planck(nu, T), 1e-3, 200 * T, limit=500, epsrel=1e-12)
    assert abs(val / (SIGMA_SB * T ** 4 / np.pi) - 1) < 1e-8


def test_planck_wien_peak():
    T = 1500.0
    k_over_hc = 1.0 / 1.438776877        # cm^-1 per K
    nu = np.linspace(2000, 4000, 200001)
    peak = nu[np.argmax(R.planck(nu, T))]
    assert abs(peak - WIEN_X * k_over_hc * T) < 0.02


def test_band_constant_and_linear():
    nu = 1000 + np.arange(2000) * 1.0
    W = np.zeros((2, 2000), np.float32)
    W[0, 200:601] = 1.0
    W[1] = np.exp(-0.5 * ((nu - 1800) / 100) ** 2)
    assert np.allclose(R.band_integrate(np.full(2000, 7.25), W), 7.25, rtol=1e-14)
    lin = 3.0 + 0.01 * nu
    out = R.band_integrate(lin, W)
    assert abs(out[0] - (3.0 + 0.01 * nu[200:601].mean())) < 1e-12
    a, b = np.random.default_rng(0).normal(size=(2, 2000))
    assert np.allclose(R.band_integrate(2 * a - b, W), 2 * R.band_integrate(a, W) - R.band_integrate(b, W),
                       rtol=1e-12, atol=1e-12)


def test_optical_depth_exact_for_opacity_linear_in_pressure():
    # tau(P) = int_{P0}^{P} chi dP' / g; for chi = a + b P the layer trapezoid
    # is exact, so every level's tau equals the integral in closed form.
    p = np.sort(np.random.default_rng(8).uniform(1e-3, 50.0, 23))
    a, b, g = 0.7, 0.031, 2182.73
    P = p * 1e6
    tau = R.optical_depth(a + b * P, p, g)
    exact = (a * (P - P[0]) + 0.5 * b * (P ** 2 - P[0] ** 2)) / g
    assert tau[0] == 0.0
    assert np.max(np.abs(tau - exact) / np.maximum(exact, 1e-300)) < 1e-13


@pytest.mark.parametrize("n,nu_lo", [(1, 4), (2, 0), (3, 5), (7, 11), (40, 3)])
def test_band_of_linear_spectrum_over_whole_span_is_the_continuous_mean(n, nu_lo):
    # A top-hat covering the whole span and a spectrum linear in nu: the band
    # value is the mean of the linear function over [nu_first, nu_last],
    # (f_first + f_last) / 2, which the trapezoid reproduces exactly only with
    # half weights at both ends of the span.
    W = np.zeros((1, 64), np.float32)
    W[0, nu_lo:nu_lo + n] = 1.0
    nu = 1000.0 + np.arange(nu_lo, nu_lo + n)
    f = 5.0 + 0.37 * nu
    got = R.band_integrate(f, W, nu_lo=nu_lo)[0]
    assert abs(got / (0.5 * (f[0] + f[-1])) - 1) < 1e-14


def test_band_value_is_invariant_to_the_filter_scale():
    # B_b is a weighted mean: scaling a filter by any positive factor, however
    # small its weight sum becomes, leaves the band value unchanged.
    rng = np.random.default_rng(9)
    f = rng.uniform(1, 2, 50)
    W = rng.uniform(0, 1, (3, 50))
    ref = R.band_integrate(f, W)
    for s in (1e-3, 1e-9, 1e6):
        assert np.allclose(R.band_integrate(f, W * s), ref, rtol=1e-13)
    one = np.zeros((1, 50))
    one[0, 17] = 1e-4                       # a single point of small weight
    assert abs(R.band_integrate(f, one)[0] / f[17] - 1) < 1e-15


def test_band_on_span_with_no_overlap_is_zero():
    W = np.zeros((1, 100), np.float32)
    W[0, 80:] = 1.0
    assert R.band_integrate(np.ones(30), W, nu_lo=10)[0] == 0.0


# ---- optical-depth limit (Sec. 4 item 7)

def test_tau_limit_keeps_isothermal_planck():
    # The level where the integration stops becomes the blackbody bottom:
    # an isothermal atmosphere still emits pi B(T) exactly.
    rng = np.random.default_rng(4)
    p = np.logspace(-6, 2, 60)
    nu = np.linspace(1000, 3000, 23)
    chi = 10 ** rng.uniform(-2, 4, (60, 23))
    for tau_max in (0.5, 3.0, 20.0):
        F = R.emission_flux(chi, p, np.full(60, 987.0), nu, 2182.73, 4, tau_max=tau_max)
        assert np.max(np.abs(F / (np.pi * R.planck(nu, 987.0)) - 1)) < 1e-12


def test_tau_limit_equals_truncated_atmosphere():
    # Opacity constant across wavenumbers: every column stops at the same
    # level k, and the result is the untruncated flux of levels 0..k.
    p = np.logspace(-6, 2, 40)
    T = np.linspace(700, 1600, 40)
    nu = np.linspace(1000, 3000, 9)
    chi = np.repeat(np.logspace(-1, 1, 40)[:, None], 9, axis=1)
    tau = R.optical_depth(chi[:, 0], p, 2182.73)
    tau_max = 7.0
    k = int(np.nonzero(tau[1:] > tau_max)[0][0]) + 1
    got = R.emission_flux(chi, p, T, nu, 2182.73, 8, tau_max=tau_max)
    exp = R.emission_flux(chi[:k + 1], p[:k + 1], T[:k + 1], nu, 2182.73, 8)
    assert np.max(np.abs(got / exp - 1)) < 1e-14


def test_tau_limit_beyond_the_column_changes_nothing():
    rng = np.random.default_rng(5)
    p = np.logspace(-6, 2, 30)
    T = rng.uniform(600, 1800, 30)
    nu = np.linspace(1000, 3000, 13)
    chi = 10 ** rng.uniform(-3, 1, (30, 13))
    a = R.emission_flux(chi, p, T, nu, 2182.73, 4)
    b = R.emission_flux(chi, p, T, nu, 2182.73, 4, tau_max=1e300)
    assert np.max(np.abs(a / b - 1)) < 1e-15


def test_tau_limit_stops_at_the_first_level_that_exceeds_it():
    # g = 1e6 and pressures 1, 2, 3, ... bar with chi = 1 give tau_k = k
    # exactly.  A level whose tau equals the limit does not stop the
    # integration; the first level with tau > tau_max is the bottom.
    L = 12
    p = np.arange(1.0, L + 1.0)
    T = np.linspace(600.0, 1500.0, L)
    nu = np.linspace(1000, 3000, 5)
    chi = np.ones((L, 5))
    assert np.array_equal(R.optical_depth(chi[:, 0], p, 1e6), np.arange(L, dtype=float))
    got = R.emission_flux(chi, p, T, nu, 1e6, 4, tau_max=3.0)
    exp = R.emission_flux(chi[:5], p[:5], T[:5], nu, 1e6, 4)       # levels 0..4 (tau = 4 > 3)
    assert np.max(np.abs(got / exp - 1)) < 1e-14


def test_tau_limit_above_a_thin_column_keeps_every_level():
    # A column thin enough that its bottom level shows: a finite limit above
    # the column's total optical depth changes nothing.
    p = np.logspace(-6, 2, 30)
    T = np.linspace(1800, 600, 30)
    nu = np.linspace(1000, 3000, 7)
    chi = np.full((30, 7), 1e-6)
    tau = R.optical_depth(chi[:, 0], p, 2182.73)
    assert 0.01 < tau[-1] < 0.1
    a = R.emission_flux(chi, p, T, nu, 2182.73, 4)
    b = R.emission_flux(chi, p, T, nu, 2182.73, 4, tau_max=5.0)
    assert np.max(np.abs(a / b - 1)) < 1e-15

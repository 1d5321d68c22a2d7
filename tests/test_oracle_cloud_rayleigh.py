"""Pins of the oracle's gray cloud deck and Rayleigh opacity (Sec. 3, the
transit code's cloud and scattering capabilities) against closed forms: the
blackbody of the deck seen through a transparent atmosphere, the isothermal
hydrostatic radius of the deck, the isothermal Planck invariance, and the
Rayleigh transit radius of an isothermal atmosphere (slant optical depth
e^-gamma_E at the effective radius, slope 4 H per e-fold of wavenumber)."""
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import forward as Fw, radiation as R
from oracle.cloud_rayleigh import deck_levels, rayleigh_chi
from oracle.constants import K_BOLTZ, AMU, BAR

G = 2182.73
MU = 2.3
RP = 1.138 * 7.1492e9
RS = 0.756 * 6.957e10
A_H2 = 8.4e-45                       # cm^2 (cm^-1)^-4: sigma_R ~ 5e-30 cm^2 at 5000 cm^-1


def _cfg(**kw):
    c = dict(g=G, mu=MU, n_angles=4, x0=[1e-4], t_int=100.0, t_star=5000.0, r_star_tp=RS,
             a_orbit=0.0312 * 1.495978707e13, t_min=500.0, t_max=3000.0, p_ref=0.1, p_top=1e-8, p_bot=100.0)
    c.update(kw)
    return c


def test_deck_level_rule():
    p = np.logspace(-6, 2, 9)                          # 1e-6 .. 100 bar, one per decade
    assert deck_levels(p, None) == 9 and deck_levels(p, 0.0) == 9 and deck_levels(p, -1.0) == 9
    assert deck_levels(p, 1e3) == 9                    # below the column: no deck
    assert deck_levels(p, 100.0) == 9                  # on the last level
    assert deck_levels(p, 1e-2) == 5                   # on a level: it is the last one kept
    assert deck_levels(p, 1.5e-2) == 6                 # between levels: the deeper one
    assert deck_levels(p, 1e-9) == 2 and deck_levels(p, 1e-6) == 2   # at least two levels


def _emission_case(L=30):
    p = np.logspace(-6, 2, L)
    T = np.linspace(900.0, 2100.0, L)                  # hotter with depth
    nu = np.linspace(1500.0, 6000.0, 7)
    grid = np.zeros((1, L, 1, nu.size))
    return p, T, nu, grid


@pytest.mark.parametrize("k", [1, 4, 17, 29])
def test_transparent_atmosphere_shows_the_deck(k):
    # no opacity above an opaque deck: F = 2 pi sum w mu B(T_k) = pi B(T_k)
    p, T, nu, grid = _emission_case()
    F = Fw.emission_spectrum(grid, p, [1000.0], nu, np.zeros(6), _cfg(p_cloud=p[k]), T=T)
    assert np.allclose(F, np.pi * R.planck(nu, T[k]), rtol=1e-13)
    # a deck between levels k-1 and k acts at level k
    F2 = Fw.emission_spectrum(grid, p, [1000.0], nu, np.zeros(6), _cfg(p_cloud=p[k] * 0.97), T=T)
    assert np.allclose(F2, F, rtol=1e-15)


def test_deck_off_or_below_changes_nothing():
    p, T, nu, _ = _emission_case()
    rng = np.random.default_rng(5)
    grid = rng.uniform(0, 3e-22, (1, 30, 1, nu.size))
    ref = Fw.emission_spectrum(grid, p, [1000.0], nu, np.zeros(6), _cfg(), T=T)
    for pc in (None, 0.0, 150.0, 100.0):
        got = Fw.emission_spectrum(grid, p, [1000.0], nu, np.zeros(6), _cfg(p_cloud=pc), T=T)
        assert np.array_equal(got, ref)


def test_rayleigh_keeps_isothermal_planck():
    p, _, nu, grid = _emission_case()
    T = np.full(30, 1400.0)
    for a in (A_H2, 1e3 * A_H2, 1e8 * A_H2):
        F = Fw.emission_spectrum(grid, p, [1000.0], nu, np.zeros(6), _cfg(rayleigh_coef=a), T=T)
        assert np.allclose(F, np.pi * R.planck(nu, 1400.0), rtol=1e-12)


def test_rayleigh_opaque_first_layer():
    # the first layer opaque at every angle: I = (B_0 + B_1) / 2, F = pi (B_0 + B_1) / 2
    p, T, nu, grid = _emission_case()
    F = Fw.emission_spectrum(grid, p, [1000.0], nu, np.zeros(6), _cfg(rayleigh_coef=1e6), T=T)
    assert np.allclose(F, 0.5 * np.pi * (R.planck(nu, T[0]) + R.planck(nu, T[1])), rtol=1e-13)


def test_rayleigh_chi_law():
    # nu^4 per molecule, divided by the mean molecular mass in grams
    nu = np.array([1000.0, 2000.0, 8000.0])
    chi = rayleigh_chi(nu, A_H2, MU)
    assert np.allclose(chi * MU * AMU / A_H2, nu ** 4, rtol=1e-15)
    assert np.all(rayleigh_chi(nu, 0.0, MU) == 0.0)


def _iso_transit(nu, L=500, T=1200.0, rayleigh=A_H2, p_cloud=None):
    """Isothermal (T clamped) instance with Rayleigh and/or a deck, no lines."""
    n_nu = nu.size
    dnu = nu[1] - nu[0] if n_nu > 1 else 1.0
    grid = np.zeros((1, 2, 1, n_nu))
    inst = SimpleNamespace(n_levels=np.array([L]), theta=np.zeros((1, 6)), nu_lo=np.array([0]),
                           nu_hi=np.array([n_nu]), r_planet=np.array([RP]), r_star=np.array([RS]))
    cfg = _cfg(t_min=T, t_max=T, rayleigh_coef=rayleigh, p_cloud=p_cloud)
    return Fw.transmission_spectrum(grid, [1e-8, 100.0], [1000.0], float(nu[0]), dnu, inst, 0, cfg)


def _iso_radius(P, T=1200.0):
    C = K_BOLTZ * T / (MU * AMU * G * RP ** 2)
    return 1.0 / (1.0 / RP + C * np.log(P / 0.1))


@pytest.mark.parametrize("k", [3, 250, 420])
def test_transparent_transit_ends_at_the_deck(k):
    # no opacity above the deck: delta = r_deck^2 / R_star^2, r from the
    # isothermal hydrostatic closed form of the whole column (P_ref = 0.1 bar
    # may lie below the deck)
    P = np.logspace(-8, 2, 500)
    d = _iso_transit(np.array([3000.0, 3001.0]), rayleigh=0.0, p_cloud=P[k])
    assert np.allclose(d, _iso_radius(P[k]) ** 2 / RS ** 2, rtol=1e-12)


def _slant_tau(b, nu, T=1200.0):
    """Rayleigh slant optical depth of an isothermal atmosphere at impact b:
    sigma n(b) sqrt(2 pi b H(b)), H(b) = k T b^2 / (mu m_u g R_p^2)."""
    C = K_BOLTZ * T / (MU * AMU * G * RP ** 2)
    P = 0.1 * np.exp((1.0 / b - 1.0 / RP) / C)
    n = P * BAR / (K_BOLTZ * T)
    return A_H2 * nu ** 4 * n * np.sqrt(2 * np.pi * b * C * b * b)


def test_rayleigh_transit_radius_closed_form():
    # For an exponential atmosphere, integral (1 - exp(-tau0 e^{-x/H})) dx over
    # x >= 0 equals H (gamma_E + ln tau0 + E1(tau0)): the effective radius is
    # where the slant optical depth is e^-gamma_E = 0.5615.
    T = 1200.0
    for nu0 in (10000.0, 25000.0):                   # photosphere near 1 and 1e-2 bar
        d = _iso_transit(np.array([nu0, nu0 + 1.0]), T=T)[0]
        R_eff = np.sqrt(d) * RS
        H = K_BOLTZ * T * R_eff ** 2 / (MU * AMU * G * RP ** 2)
        lo, hi = RP * 0.9, RP * 1.2                  # bisection on tau(b) = e^-gamma
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if _slant_tau(mid, nu0, T) > np.exp(-np.euler_gamma):
                lo = mid
            else:
                hi = mid
        assert abs(R_eff - 0.5 * (lo + hi)) < 0.02 * H


def test_rayleigh_transit_slope_is_four_scale_heights():
    # dR_eff / d ln nu = 4 H
    T = 1200.0
    nus = np.array([10000.0, 10000.0 * np.e])
    R_eff = [np.sqrt(_iso_transit(np.array([v, v + 1.0]), T=T)[0]) * RS for v in nus]
    H = K_BOLTZ * T * (0.5 * (R_eff[0] + R_eff[1])) ** 2 / (MU * AMU * G * RP ** 2)
    assert abs((R_eff[1] - R_eff[0]) / (4 * H) - 1) < 0.01


def test_transit_span_maps_each_point_to_its_wavenumber():
    # A span starting inside the grid with a step other than 1: each point
    # of the instance's spectrum is the Rayleigh transit of the wavenumber
    # nu_start + (nu_lo + j) dnu, evaluated alone.
    n_grid, lo, hi, dnu, nu_start = 12, 3, 10, 750.0, 9000.0
    grid = np.zeros((1, 2, 1, n_grid))
    inst = SimpleNamespace(n_levels=np.array([300]), theta=np.zeros((1, 6)), nu_lo=np.array([lo]),
                           nu_hi=np.array([hi]), r_planet=np.array([RP]), r_star=np.array([RS]))
    cfg = _cfg(t_min=1200.0, t_max=1200.0, rayleigh_coef=A_H2)
    span = Fw.transmission_spectrum(grid, [1e-8, 100.0], [1000.0], nu_start, dnu, inst, 0, cfg)
    assert span.size == hi - lo
    for j in (0, 4, hi - lo - 1):
        v = nu_start + (lo + j) * dnu
        alone = _iso_transit(np.array([v, v + 1.0]), L=300)[0]
        assert abs(span[j] / alone - 1) < 1e-13
    assert np.all(np.diff(span) > 0)               # sigma_R grows with nu


def test_contributions_carry_rayleigh_and_the_deck():
    # The per-layer contributions of a cloudy, Rayleigh-scattering column add
    # up to its flux, and nothing below the deck contributes.
    p, T, nu, _ = _emission_case()
    rng = np.random.default_rng(6)
    grid = rng.uniform(0, 1e-24, (1, 30, 1, nu.size))
    cfg = _cfg(rayleigh_coef=1e4 * A_H2, p_cloud=p[21])
    C = Fw.emission_contributions(grid, p, [1000.0], nu, np.zeros(6), cfg, T=T)
    F = Fw.emission_spectrum(grid, p, [1000.0], nu, np.zeros(6), cfg, T=T)
    assert np.allclose(C.sum(axis=0), F, rtol=1e-12)
    assert np.all(C[22:] == 0.0)
    off = Fw.emission_contributions(grid, p, [1000.0], nu, np.zeros(6), _cfg(p_cloud=p[21]), T=T)
    assert np.max(np.abs(C.sum(axis=0) / off.sum(axis=0) - 1)) > 1e-3

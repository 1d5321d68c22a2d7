"""Pins of the oracle's emission contribution functions (post-processing of
Sec. 3): the decomposition adds up to the flux, a transparent atmosphere shows
only the bottom blackbody, an opaque first layer carries all the flux, and
for a constant opacity the contribution per unit ln P peaks where the optical
depth equals the ray's mu (the classic weighting-function maximum)."""
import numpy as np
import pytest

from oracle import radiation as R, forward as Fw

G = 2182.73


def _case(L=40, seed=2):
    rng = np.random.default_rng(seed)
    p = np.logspace(-6, 2, L)
    T = np.linspace(800.0, 2200.0, L)
    nu = np.linspace(1200.0, 5000.0, 9)
    chi = 10 ** rng.uniform(-4, 1, (L, nu.size))
    return p, T, nu, chi


@pytest.mark.parametrize("tau_max,thin", [(None, False), (2.0, False), (50.0, True)])
def test_contributions_add_up_to_the_flux(tau_max, thin):
    p, T, nu, chi = _case()
    if thin:                 # the limit is never reached and the bottom shows
        chi = chi * 1e-5
    C = R.emission_contributions(chi, p, T, nu, G, 8, tau_max=tau_max)
    F = R.emission_flux(chi, p, T, nu, G, 8, tau_max=tau_max)
    assert np.allclose(C.sum(axis=0), F, rtol=1e-12)
    assert np.all(C >= 0)
    if tau_max is not None:
        # below the level where the limit stops, nothing
        tau = R.optical_depth(chi.T, p, G)
        for r in range(nu.size):
            over = np.nonzero(tau[r, 1:] > tau_max)[0]
            kb = over[0] + 1 if over.size else len(p) - 1
            assert np.all(C[kb + 1:, r] == 0.0) and C[kb, r] > 0
            assert thin == (over.size == 0)


def test_contributions_stop_at_the_first_level_that_exceeds_the_limit():
    # tau_k = k exactly (g = 1e6, chi = 1, pressures 1, 2, 3, ... bar): with
    # tau_max = 3 the level with tau = 3 does not stop the sum, level 4 does.
    L = 10
    p = np.arange(1.0, L + 1.0)
    T = np.linspace(700.0, 1600.0, L)
    nu = np.linspace(1000, 3000, 5)
    chi = np.ones((L, 5))
    C = R.emission_contributions(chi, p, T, nu, 1e6, 4, tau_max=3.0)
    assert np.all(C[5:] == 0.0) and np.all(C[4] > 0)
    F = R.emission_flux(chi[:5], p[:5], T[:5], nu, 1e6, 4)
    assert np.allclose(C.sum(axis=0), F, rtol=1e-13)


def test_transparent_atmosphere_shows_only_the_bottom():
    p, T, nu, _ = _case()
    C = R.emission_contributions(np.zeros((40, nu.size)), p, T, nu, G, 4)
    assert np.all(C[:-1] == 0.0)
    assert np.allclose(C[-1], np.pi * R.planck(nu, T[-1]), rtol=1e-13)


def test_opaque_first_layer_carries_everything():
    p, T, nu, _ = _case()
    C = R.emission_contributions(np.full((40, nu.size), 1e9), p, T, nu, G, 4)
    assert np.allclose(C[0], 0.5 * np.pi * (R.planck(nu, T[0]) + R.planck(nu, T[1])), rtol=1e-13)
    assert np.all(C[1:] < 1e-300)


def test_weighting_function_peaks_at_tau_equal_mu():
    # one Gauss-Legendre angle: mu = 1/2.  Constant opacity, isothermal: the
    # contribution per unit ln P is B P chi / (g mu) exp(-tau / mu) in the
    # continuum limit, largest at tau = mu.
    L = 2000
    p = np.logspace(-6, 2, L)
    chi = np.full((L, 1), G / (0.5 * 1e6 * 0.03))      # tau = 1/2 near 0.03 bar
    C = R.emission_contributions(chi, p, np.full(L, 1500.0), np.array([2500.0]), G, 1)[:-1, 0]
    per_lnp = C / np.diff(np.log(p))
    k = int(np.argmax(per_lnp))
    tau_mid = chi[0, 0] * 0.5 * (p[k] + p[k + 1] - 2 * p[0]) * 1e6 / G
    assert abs(tau_mid / 0.5 - 1) < 0.01


def test_deck_ends_the_contributions():
    L = 30
    p = np.logspace(-6, 2, L)
    T = np.linspace(900.0, 2100.0, L)
    nu = np.linspace(1500.0, 6000.0, 5)
    cfg = dict(g=G, mu=2.3, n_angles=4, x0=[1e-4], p_cloud=float(p[12] * 0.98))
    C = Fw.emission_contributions(np.zeros((1, L, 1, nu.size)), p, [1000.0], nu, np.zeros(6), cfg, T=T)
    assert np.all(C[:12] == 0.0) and np.all(C[13:] == 0.0)
    assert np.allclose(C[12], np.pi * R.planck(nu, T[12]), rtol=1e-13)

"""Pins of the oracle's T(P) profile (Sec. 7, nine-parameter model), grid
interpolation and transit geometry (test f01oneline transit text, Sec. 6.1)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import profile as P
from oracle import transmission as Tr
from oracle import forward as Fw
from oracle.constants import K_BOLTZ, AMU
from scipy.special import expn

G = 2182.73


def _T(theta, p, t_int=100.0):
    return P.temperature(np.asarray(theta, float), p, G, t_int, 5000.0, 0.756 * 6.957e10,
                         0.0312 * 1.495978707e13)


def test_e2_matches_its_integral_definition():
    for x in (1e-3, 0.1, 1.0, 4.0, 20.0):
        val, _ = integrate.quad(lambda t: np.exp(-x * t) / t ** 2, 1, np.inf, epsrel=1e-12)
        assert abs(expn(2, x) / val - 1) < 1e-10


def test_no_irradiation_reduces_to_eddington():
    p = np.logspace(-8, 2, 50)
    th = [-1.0, 0.2, -0.4, 0.3, 0.0]                     # beta = 0 -> T_irr = 0
    tau = 0.1 * p * 1e6 / G
    assert np.allclose(_T(th, p), (0.75 * 100.0 ** 4 * (2 / 3 + tau)) ** 0.25, rtol=1e-14)


def test_top_of_atmosphere_closed_form():
    # tau -> 0: xi(g, 0) = 2/3 + 2g/3 (E2(0) = 1)
    th = [-2.0, 0.5, -1.0, 0.25, 1.1]
    t_irr = 1.1 * np.sqrt(0.756 * 6.957e10 / (2 * 0.0312 * 1.495978707e13)) * 5000.0
    g1, g2 = 10 ** 0.5, 10 ** -1.0
    T4 = 0.75 * 100.0 ** 4 * 2 / 3 + 0.75 * t_irr ** 4 * (0.75 * (2 / 3 + 2 * g1 / 3) + 0.25 * (2 / 3 + 2 * g2 / 3))
    assert abs(_T(th, np.array([1e-30]))[0] / T4 ** 0.25 - 1) < 1e-12


def test_channel_swap_symmetry():
    p = np.logspace(-8, 2, 40)
    a = _T([-1.5, 0.4, -0.9, 0.3, 1.0], p)
    b = _T([-1.5, -0.9, 0.4, 0.7, 1.0], p)
    assert np.allclose(a, b, rtol=1e-13)


def test_bracket_rule():
    ax = np.array([500.0, 1000.0, 1500.0])
    assert Fw.bracket(ax, 1000.0) == (1, 0.0)
    assert Fw.bracket(ax, 1500.0) == (1, 1.0)
    assert Fw.bracket(ax, 200.0) == (0, 0.0)
    assert Fw.bracket(ax, 9e9) == (1, 1.0)
    m, w = Fw.bracket(ax, 1250.0)
    assert m == 1 and abs(w - 0.5) < 1e-15


def test_interpolation_exact_on_linear_grids():
    rng = np.random.default_rng(1)
    t_ax = np.linspace(500, 3000, 6)
    p_ax = np.logspace(-8, 2, 5)
    a, b, c = rng.uniform(1, 2, (3, 2, 7))
    grid = (a[:, None, None, :] + b[:, None, None, :] * t_ax[None, None, :, None]
            + c[:, None, None, :] * np.log10(p_ax)[None, :, None, None])
    T = rng.uniform(500, 3000, 9)
    Pl = 10 ** rng.uniform(-8, 2, 9)
    got = Fw.level_opacity_bilinear(grid, p_ax, t_ax, Pl, T)
    exp = a[:, None, :] + b[:, None, :] * T[None, :, None] + c[:, None, :] * np.log10(Pl)[None, :, None]
    assert np.allclose(got, exp, rtol=1e-12)


@pytest.mark.parametrize("n_t,n_p", [(1, 5), (6, 1), (1, 1), (2, 2), (2, 5)])
def test_interpolation_on_degenerate_and_two_node_axes(n_t, n_p):
    # A grid with one node along an axis is constant along it; with two
    # nodes the bracket is the single interval.  Grids linear in the other
    # axis are reproduced exactly, in (log10 P, T) and, for layer_opacity, in T.
    rng = np.random.default_rng(n_t * 10 + n_p)
    t_ax = np.linspace(700, 2500, n_t)
    p_ax = np.logspace(-6, 1, n_p)
    a, b, c = rng.uniform(1, 2, (3, 2, 5))
    bt = b if n_t > 1 else 0 * b
    cp = c if n_p > 1 else 0 * c
    grid = (a[:, None, None, :] + bt[:, None, None, :] * t_ax[None, None, :, None]
            + cp[:, None, None, :] * np.log10(p_ax)[None, :, None, None])
    T = rng.uniform(700, 2500, 6)
    Pl = 10 ** rng.uniform(-6, 1, 6)
    got = Fw.level_opacity_bilinear(grid, p_ax, t_ax, Pl, T)
    exp = a[:, None, :] + bt[:, None, :] * T[None, :, None] + cp[:, None, :] * np.log10(Pl)[None, :, None]
    assert np.allclose(got, exp, rtol=1e-12)
    lay = Fw.layer_opacity(grid, t_ax, T[:n_p])
    exp_l = (a[:, None, :] + bt[:, None, :] * T[:n_p][None, :, None]
             + cp[:, None, :] * np.log10(p_ax)[None, :, None])
    assert np.allclose(lay, exp_l, rtol=1e-12)


def _iso_atm(L=200, T=1200.0, mu=2.3, g=G, rp=1.138 * 7.1492e9):
    p = np.logspace(-8, 2, L)
    return p, np.full(L, T), Tr.radii(p, np.full(L, T), rp, 0.1, g, mu)


def test_isothermal_radii_closed_form():
    p, T, r = _iso_atm()
    rp = 1.138 * 7.1492e9
    C = K_BOLTZ * 1200.0 / (2.3 * AMU * G * rp ** 2)
    assert np.allclose(r, 1.0 / (1.0 / rp + C * np.log(p / 0.1)), rtol=1e-13)


def test_transit_depth_limits():
    p, T, r = _iso_atm(L=80)
    rs = 0.756 * 6.957e10
    d0 = Tr.transit_depth(np.zeros((80, 3)), p, T, r, rs, 2.3)
    assert np.allclose(d0, r[-1] ** 2 / rs ** 2, rtol=1e-14)
    dinf = Tr.transit_depth(np.full((80, 3), 1e30), p, T, r, rs, 2.3)
    assert np.allclose(dinf, r[0] * r[1] / rs ** 2, rtol=1e-13)   # discrete closed form


def test_scale_height_law():
    # Constant cross-section, isothermal: R_eff(s2) - R_eff(s1) = H ln(s2/s1),
    # H = k T / (mu m_u g(R_eff)).
    p, T, r = _iso_atm(L=400)
    rs = 0.756 * 6.957e10
    d1 = Tr.transit_depth(np.full((400, 1), 1e-3), p, T, r, rs, 2.3)[0]
    d2 = Tr.transit_depth(np.full((400, 1), 1e-3 * np.e ** 2), p, T, r, rs, 2.3)[0]
    R1, R2 = np.sqrt(d1) * rs, np.sqrt(d2) * rs
    g_eff = G * (1.138 * 7.1492e9 / R1) ** 2
    H = K_BOLTZ * 1200.0 / (2.3 * AMU * g_eff)
    assert abs((R2 - R1) / (2 * H) - 1) < 0.02


@pytest.mark.parametrize("lk,lg1,lg2,alpha", [(-1.0, 0.6, -1.2, 0.3), (-2.5, -1.4, 0.9, 0.8), (0.0, 0.0, -0.5, 0.0)])
def test_irradiated_profile_is_gray_radiative_equilibrium(lk, lg1, lg2, alpha):
    """The profile is the gray two-stream solution in radiative equilibrium
    with an irradiating beam of isotropic incidence, attenuated exactly, in
    two visible channels.  In units where B = T^4:
      thermal field (Eddington closure): dJ/dtau = 3 H,  J(0) = 2 H(0);
      radiative equilibrium: J - B = -sum_c w_c gamma_c J_c;
      visible channel c: J_c = c0 E2(gamma_c tau), H_c = -c0 E3(gamma_c tau);
      flux conservation: H = H_int - sum_c w_c H_c,
    with w = (1 - alpha, alpha), H_int = T_int^4 / 4 and c0 = T_irr^4 / 2 (the
    absorbed stellar flux c0 E3(0) = T_irr^4 / 4 in the units of H_int).  The
    oracle's T is checked against these relations, E3 integrated by
    quadrature; a changed term of the profile breaks one of them."""
    beta, t_int = 1.05, 100.0
    th = [lk, lg1, lg2, alpha, beta]
    kappa = 10.0 ** lk
    gam = np.array([10.0 ** lg1, 10.0 ** lg2])
    w = np.array([1.0 - alpha, alpha])
    t_irr = beta * np.sqrt(0.756 * 6.957e10 / (2 * 0.0312 * 1.495978707e13)) * 5000.0
    c0, h_int = t_irr ** 4 / 2.0, t_int ** 4 / 4.0

    def tau_to_p(tau):
        return np.asarray(tau) * G / (kappa * 1e6)

    def J(tau):
        B = _T(th, tau_to_p(tau), t_int) ** 4
        return B - c0 * sum(w[c] * gam[c] * expn(2, gam[c] * np.asarray(tau)) for c in range(2))

    def H(t):
        return h_int + c0 * sum(w[c] * expn(3, gam[c] * t) for c in range(2))

    scale = _T(th, tau_to_p(np.array([1e3])), t_int)[0] ** 4
    j0 = J(np.array([1e-15]))[0]
    assert abs(j0 - 2.0 * H(0.0)) < 1e-12 * scale
    taus = np.concatenate([[1e-15], np.geomspace(1e-4, 60.0 / gam.min(), 25)])
    jt = J(taus)
    for a, b, ja, jb in zip(taus[:-1], taus[1:], jt[:-1], jt[1:]):
        flux, _ = integrate.quad(H, a, b, epsabs=0.0, epsrel=1e-13, limit=200)
        assert abs((jb - ja) - 3.0 * flux) < 1e-11 * scale


def test_radii_exact_for_temperature_linear_in_log_pressure():
    # Hydrostatic balance with g = g_ref (R_p / r)^2:
    #   d(1/r)/d ln P = k T / (mu m_u g_ref R_p^2),  r = R_p at P_ref;
    # for T = a + b ln P the solution is closed form (and the level trapezoid
    # with the reference pressure inserted as a node is exact).
    p = np.logspace(-7, 2, 37)
    a, b = 1400.0, 45.0
    T = a + b * np.log(p)
    rp = 1.21 * 7.1492e9
    r = Tr.radii(p, T, rp, 0.1, G, 2.3)
    C = K_BOLTZ / (2.3 * AMU * G * rp ** 2)
    lp, lr = np.log(p), np.log(0.1)
    exact = 1.0 / (1.0 / rp + C * (a * (lp - lr) + 0.5 * b * (lp ** 2 - lr ** 2)))
    assert np.max(np.abs(r / exact - 1)) < 1e-13


@pytest.mark.parametrize("alpha", [1e-11, 3e-10, 1e-8])
def test_transit_depth_constant_extinction(alpha):
    # Constant extinction alpha (cm^-1) in every shell: the chord through the
    # shells above impact parameter b telescopes to the chord through the top
    # sphere, tau(b) = 2 alpha sqrt(r_top^2 - b^2), at every level.  With the
    # levels' trapezoid in b the depth is then fixed in closed form; and with
    # many levels it converges (like h^1.5: the integrand has a square-root
    # edge at the top sphere) to the continuous integral
    #   R*^2 delta = r_bot^2 + U^2 - (1 - e^{-2 alpha U} (1 + 2 alpha U)) / (2 alpha^2),
    # U^2 = r_top^2 - r_bot^2.
    L = 3000
    p = np.logspace(-8, 2, L)
    T = np.linspace(900.0, 1700.0, L)
    rp, rs, mu = 1.138 * 7.1492e9, 0.756 * 6.957e10, 2.3
    r = Tr.radii(p, T, rp, 0.1, G, mu)
    rho = p * 1e6 * mu * AMU / (K_BOLTZ * T)
    chi = (alpha / rho)[:, None]
    got = Tr.transit_depth(chi, p, T, r, rs, mu)[0]
    f = -np.expm1(-2.0 * alpha * np.sqrt(np.maximum(r[0] ** 2 - r ** 2, 0.0)))
    trap = np.sum((f[:-1] * r[:-1] + f[1:] * r[1:]) * (r[:-1] - r[1:]))
    assert abs(got / ((r[-1] ** 2 + trap) / rs ** 2) - 1) < 1e-12
    U2 = r[0] ** 2 - r[-1] ** 2
    U = np.sqrt(U2)
    cont = (r[-1] ** 2 + U2 - (1 - np.exp(-2 * alpha * U) * (1 + 2 * alpha * U)) / (2 * alpha ** 2)) / rs ** 2
    assert abs(got / cont - 1) < 1e-5

"""Pins of the oracle's composed forward model: the steps between the opacity
grid and the radiative transfer -- temperature interpolation of the grid
(``forward.layer_opacity``), abundances X_s = X0_s 10^{a_s}
(``profile.abundances``) and the mass opacity chi = sum_s X_s sigma_s /
(mu m_u) (``forward.mass_opacity``) -- checked through the public oracle
entry points against closed forms whose constants are written here as
numbers, not taken from the oracle:

* f05abundance (Sec. 6.1.2, Eqs. 12-13): one absorbing layer of constant cross
  section over a hotter interior; its line depth and the ratio of depths at
  two abundances have closed forms in tau = X sigma dP / (mu m_u g);
* a transparent-to-opaque isothermal transit (Sec. 6.1, the f01oneline
  transit recipe): R_eff moves by H ln k when sigma or X is scaled by k, and
  sits where the slant optical depth is exp(-Euler gamma);
* layer_opacity is exact on grids linear in T and clamps outside the axis.
A missing m_u, mu instead of mu m_u, X0 a instead of X0 10^a or a wrong
interpolation weight fails at least one of these."""
import numpy as np

import workloads as W
from oracle import forward as Fw
from oracle import radiation as R

# CODATA 2018 values (cgs), typed here independently of oracle/constants.py
M_U = 1.66053906660e-24        # g
K_B = 1.380649e-16             # erg K^-1
EULER_GAMMA = 0.5772156649015329
G = 2182.73                    # cm s^-2 (Sec. 6.2)
SIG_ONE_LAYER = (2e-23, 7e-24)  # cm^2 per molecule of the two species


def _em_cfg(n_angles, x0, mu=2.3):
    return dict(g=G, t_int=100.0, t_star=5000.0, r_star_tp=0.756 * 6.957e10, a_orbit=0.0312 * 1.495978707e13,
                t_min=1.0, t_max=1e5, x0=list(x0), mu=mu, n_angles=n_angles)


def _one_layer_case(log_ab, n_angles=8):
    """Two levels (one layer, 0.01 -> 0.1 bar), T = 900 K above 1400 K;
    species 0 with sigma0, species 1 with sigma1 everywhere on a 3-T grid."""
    p = np.array([0.01, 0.1])
    t_axis = np.array([500.0, 1500.0, 3000.0])
    nu = np.array([1200.0, 2000.0, 2750.0])
    sig = np.array(SIG_ONE_LAYER)
    grid = np.empty((2, 2, 3, 3))
    grid[0], grid[1] = sig[0], sig[1]
    x0 = [1e-4, 3e-4]
    theta = np.array([-1.0, 0.0, 0.0, 0.5, 1.0] + list(log_ab))
    T = np.array([900.0, 1400.0])
    F = Fw.emission_spectrum(grid, p, t_axis, nu, theta, _em_cfg(n_angles, x0), T=T)
    # tau of the layer by hand: X_s = X0_s 10^a_s, chi = sum X sigma / (mu m_u),
    # dtau = chi (P1 - P0) / g with P in dyn cm^-2
    X = np.array(x0) * 10.0 ** np.asarray(log_ab, float)
    tau = float(np.dot(X, sig)) / (2.3 * M_U) * (0.1 - 0.01) * 1e6 / G
    return F, tau, nu, T


def test_f05_one_layer_depth_and_ratio_closed_form():
    """F0 - F = pi (B1 - B0) sum_i w_i mu_i (1 - exp(-tau/mu_i)) for one layer
    (layer-mean source, blackbody interior at the bottom level), with the
    Gauss-Legendre nodes from numpy; the depth ratio at abundance n over
    abundance 1 is f(n) = sum w mu (1 - e^{-n tau/mu}) / sum w mu (1 - e^{-tau/mu})."""
    x, w = np.polynomial.legendre.leggauss(8)
    mu, wq = 0.5 * (x + 1.0), 0.5 * w
    depth = {}
    for n in (1.0, 2.0, 5.0, 10.0):
        F, tau, nu, T = _one_layer_case([np.log10(n), 0.5])
        B0, B1 = R.planck(nu, T[0]), R.planck(nu, T[1])
        exp_depth = np.pi * (B1 - B0) * np.sum(wq * mu * -np.expm1(-tau / mu))
        got = np.pi * B1 - F
        assert np.allclose(got, exp_depth, rtol=1e-10), (n, got, exp_depth)
        depth[n] = got
    # the ratio depends on tau only through the X-weighted sum: scaling
    # species 0 by n scales its share of tau by n
    _, tau1, _, _ = _one_layer_case([0.0, 0.5])
    tau_s1 = 3e-4 * 10 ** 0.5 * SIG_ONE_LAYER[1] / (2.3 * M_U) * 0.09e6 / G
    tau_s0 = tau1 - tau_s1
    for n in (2.0, 5.0, 10.0):
        f = (np.sum(wq * mu * -np.expm1(-(n * tau_s0 + tau_s1) / mu))
             / np.sum(wq * mu * -np.expm1(-tau1 / mu)))
        assert np.allclose(depth[n] / depth[1.0], f, rtol=1e-10)
    # the case is optically thin-to-moderate, so the layer matters: tau ~ 0.1
    assert 0.01 < tau1 < 1.0


def test_abundance_scalings_are_powers_of_ten():
    """X_s = X0_s 10^{a_s}: a = 0, 1, -2, log10 3 multiply X0 by 1, 10, 0.01, 3."""
    from oracle import profile as P
    theta = np.array([0.0] * 5 + [0.0, 1.0, -2.0, np.log10(3.0)])
    x0 = [1e-4, 2e-4, 5e-5, 1e-3]
    assert np.allclose(P.abundances(theta, x0), [1e-4, 2e-3, 5e-7, 3e-3], rtol=1e-14)
    # only as many scalings as species are used
    assert np.allclose(P.abundances(theta, x0[:2]), [1e-4, 2e-3], rtol=1e-14)


def test_layer_opacity_exact_on_grids_linear_in_T():
    """grid = a + b T_m on every (species, layer, wavenumber): the layer
    opacity at T is a + b clip(T, T_0, T_last); M = 1 returns the one row."""
    rng = np.random.default_rng(11)
    S, L, M, N = 3, 7, 5, 4
    t_axis = np.sort(rng.uniform(400.0, 3200.0, M))
    a = rng.uniform(1.0, 2.0, (S, L, N))
    b = rng.uniform(-1e-4, 1e-4, (S, L, N))
    grid = a[:, :, None, :] + b[:, :, None, :] * t_axis[None, None, :, None]
    T = np.concatenate([rng.uniform(t_axis[0], t_axis[-1], L - 3), [t_axis[2], 100.0, 9000.0]])
    got = Fw.layer_opacity(grid, t_axis, T)
    Tc = np.clip(T, t_axis[0], t_axis[-1])
    exp = a + b * Tc[None, :, None]
    assert np.allclose(got, exp, rtol=1e-13, atol=0)
    one = Fw.layer_opacity(grid[:, :, :1, :], t_axis[:1], T)
    assert np.array_equal(one, grid[:, :, 0, :])


def test_mass_opacity_units():
    """chi = sum_s X_s sigma_s / (mu m_u) in cm^2 g^-1: 1e-4 of a 1e-20 cm^2
    absorber in a mu = 2 gas is 1e-24 / (2 m_u) = 0.3011070381... cm^2 g^-1."""
    sig = np.full((2, 1, 1), 1e-20)
    chi = Fw.mass_opacity(sig, [1e-4, 0.0], 2.0)
    assert abs(chi[0, 0] / 0.30110703810 - 1) < 1e-10


# ---- transit through the composed path (instance levels, T(P) clamp,
#      bilinear interpolation, abundances, mass opacity, radii, transit depth)

def _transit_case(sigma_per_nu, log_ab=0.0, n_levels=400, T0=1200.0):
    N = len(sigma_per_nu)
    p_axis = np.logspace(-8, 2, 5)
    t_axis = np.array([500.0, 3000.0])
    grid = np.empty((1, 5, 2, N))
    grid[:] = np.asarray(sigma_per_nu, float)[None, None, None, :]
    rp, rs = 1.138 * 7.1492e9, 0.756 * 6.957e10
    inst = W.Instances(n_levels=np.array([n_levels], np.int32), nu_lo=np.array([0], np.int64),
                       nu_hi=np.array([N], np.int64), r_planet=np.array([rp]), r_star=np.array([rs]),
                       theta=np.array([[-1.0, 0.0, 0.0, 0.5, 1.0, log_ab, 0.0, 0.0, 0.0]]))
    cfg = _em_cfg(1, [1e-4])
    cfg.update(t_min=T0, t_max=T0, p_ref=0.1, p_top=1e-8, p_bot=100.0)   # clamp: isothermal at T0
    d = Fw.transmission_spectrum(grid, p_axis, t_axis, 1000.0, 1.0, inst, 0, cfg)
    return np.sqrt(d) * rs, rp


def test_transit_radius_moves_by_scale_height_per_e_fold():
    """Isothermal, constant cross section: R_eff(k sigma) - R_eff(sigma) =
    H ln k, H = k_B T / (mu m_u g(R_eff)), both for sigma and for X (a = log10 k)."""
    s1 = 1e-25
    R, rp = _transit_case([s1, s1 * np.e, s1 * np.e ** 2])
    Ra, _ = _transit_case([s1], log_ab=np.log10(np.e ** 2))
    g_eff = G * (rp / R[1]) ** 2
    H = K_B * 1200.0 / (2.3 * M_U * g_eff)
    assert abs((R[1] - R[0]) / H - 1) < 0.02
    assert abs((R[2] - R[1]) / H - 1) < 0.02
    assert abs((Ra[0] - R[0]) / (2 * H) - 1) < 0.02


def test_transit_radius_absolute_closed_form():
    """The effective radius sits where the slant optical depth is
    exp(-Euler gamma) (Lecavelier des Etangs et al. 2008): for an isothermal
    column with g ~ r^-2 anchored at P_ref = 0.1 bar on R_p,
    P(r) = P_ref exp[(R_p / H_p)(R_p / r - 1)], H_p = k_B T / (mu m_u g),
    and tau(b) = X sigma P(b) / (k_B T) sqrt(2 pi b H(b)), H(b) = H_p (b/R_p)^2.
    Holds to a small fraction of H (terms of order H/R)."""
    T, mu, X = 1200.0, 2.3, 1e-4
    for s in (1e-25, 1e-24, 1e-23, 1e-21):
        R, rp = _transit_case([s], n_levels=600)
        Hp = K_B * T / (mu * M_U * G)

        def tau(b):
            P = 0.1e6 * np.exp(rp / Hp * (rp / b - 1.0))
            return X * s * P / (K_B * T) * np.sqrt(2 * np.pi * b * Hp * (b / rp) ** 2)
        lo, hi = rp - 40 * Hp, rp + 60 * Hp
        for _ in range(200):                     # tau falls with b: bisection
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if tau(mid) > np.exp(-EULER_GAMMA) else (lo, mid)
        b_star = 0.5 * (lo + hi)
        H_b = Hp * (b_star / rp) ** 2
        assert abs(R[0] - b_star) < 0.05 * H_b, (s, (R[0] - b_star) / H_b)

"""Per-proposal forward model on a precomputed opacity grid.

The retrieval interpolates the precomputed opacity table to the temperature of
each layer (Sec. 4 items 3 and Sec. 6.1.1, "it interpolates in the opacity
table ... to the temperature of each atmospheric layer"), scales by the
abundances from the profile generator (Sec. 3), and runs the emission or
transmission RT, then the spectrum integrator (Sec. 3).  Readings:

* interpolation is linear in T on the opacity: bracket m = max{m : T_m <= T}
  (limited to [0, M-2]), weight w = (T - T_m)/(T_{m+1} - T_m) limited to [0, 1];
  a node hits weight 0 on its upper neighbour;
* instances whose levels differ from the grid's layers interpolate bilinearly
  in (log10 P, T), with the same bracket rule in log10 P;
* chi = sum_s X_s sigma_s / (mu m_u) in cm^2 g^-1, plus the Rayleigh term and
  with the gray cloud deck of ``cloud_rayleigh`` when cfg sets rayleigh_coef
  or p_cloud.
"""
import numpy as np

from .constants import AMU
from . import profile, radiation, transmission
from .cloud_rayleigh import deck_levels, rayleigh_chi


def bracket(axis, v):
    """(index, weight) of linear interpolation with the rule above."""
    axis = np.asarray(axis, np.float64)
    M = axis.size
    if M == 1:
        return 0, 0.0
    m = int(np.searchsorted(axis, v, side="right")) - 1
    m = min(max(m, 0), M - 2)
    w = (v - axis[m]) / (axis[m + 1] - axis[m])
    return m, float(min(max(w, 0.0), 1.0))


def layer_opacity(grid, t_axis, T):
    """sigma[S][L][n_nu] at layer temperatures T[L] from grid[S][L][M][n_nu]."""
    S, L, M, N = grid.shape
    out = np.zeros((S, L, N))
    for k in range(L):
        m, w = bracket(t_axis, T[k])
        if M == 1:
            out[:, k] = grid[:, k, 0]
        else:
            out[:, k] = (1.0 - w) * grid[:, k, m] + w * grid[:, k, m + 1]
    return out


def level_opacity_bilinear(grid, p_axis, t_axis, P, T):
    """sigma[S][len(P)][n_nu] at (P, T) points, bilinear in (log10 P, T)."""
    S, L, M, N = grid.shape
    lp_axis = np.log10(np.asarray(p_axis, np.float64))
    out = np.zeros((S, len(P), N))
    for k in range(len(P)):
        a, u = bracket(lp_axis, np.log10(P[k]))
        m, w = bracket(t_axis, T[k])
        if L == 1:
            a, u = 0, 0.0
        g00 = grid[:, a, m]
        g01 = grid[:, a, m + 1] if M > 1 else g00
        if L > 1:
            g10 = grid[:, a + 1, m]
            g11 = grid[:, a + 1, m + 1] if M > 1 else g10
        else:
            g10, g11 = g00, g01
        out[:, k] = ((1 - u) * ((1 - w) * g00 + w * g01) + u * ((1 - w) * g10 + w * g11))
    return out


def mass_opacity(sigma, X, mu_amu):
    """chi[L][n_nu] = sum_s X_s sigma_s / (mu m_u)."""
    return np.tensordot(np.asarray(X, np.float64), sigma, axes=(0, 0)) / (mu_amu * AMU)


def tp_of(theta, p_bar, cfg):
    return profile.temperature(theta, p_bar, cfg["g"], cfg["t_int"], cfg["t_star"],
                               cfg["r_star_tp"], cfg["a_orbit"], cfg["t_min"], cfg["t_max"])


def emission_spectrum(grid, p_axis, t_axis, nu, theta, cfg, T=None):
    """F(nu) for one proposal; T given explicitly or from theta's T(P)."""
    if T is None:
        T = tp_of(theta, p_axis, cfg)
    X = profile.abundances(theta, cfg["x0"])
    sig = layer_opacity(grid, t_axis, T)
    chi = mass_opacity(sig, X, cfg["mu"]) + rayleigh_chi(nu, cfg.get("rayleigh_coef", 0.0), cfg["mu"])[None, :]
    Le = deck_levels(p_axis, cfg.get("p_cloud"))
    return radiation.emission_flux(chi[:Le], np.asarray(p_axis)[:Le], np.asarray(T)[:Le], nu, cfg["g"],
                                   cfg["n_angles"], tau_max=cfg.get("tau_max"))


def emission_contributions(grid, p_axis, t_axis, nu, theta, cfg, T=None):
    """Per-layer contributions C[L][n_nu] of one proposal's emission spectrum
    (``radiation.emission_contributions``), with the Rayleigh term and the
    gray cloud deck as in ``emission_spectrum``; levels below the deck are 0."""
    if T is None:
        T = tp_of(theta, p_axis, cfg)
    X = profile.abundances(theta, cfg["x0"])
    sig = layer_opacity(grid, t_axis, T)
    chi = mass_opacity(sig, X, cfg["mu"]) + rayleigh_chi(nu, cfg.get("rayleigh_coef", 0.0), cfg["mu"])[None, :]
    L = len(p_axis)
    Le = deck_levels(p_axis, cfg.get("p_cloud"))
    C = np.zeros((L, len(nu)))
    C[:Le] = radiation.emission_contributions(chi[:Le], np.asarray(p_axis)[:Le], np.asarray(T)[:Le], nu, cfg["g"],
                                              cfg["n_angles"], tau_max=cfg.get("tau_max"))
    return C


def instance_levels(n_levels, p_top, p_bot):
    return np.logspace(np.log10(p_top), np.log10(p_bot), int(n_levels))


def transmission_spectrum(grid, p_axis, t_axis, nu_start, dnu, inst, i, cfg):
    """delta(nu) over instance i's span (FP64)."""
    P = instance_levels(inst.n_levels[i], cfg["p_top"], cfg["p_bot"])
    th = inst.theta[i]
    T = tp_of(th, P, cfg)
    X = profile.abundances(th, cfg["x0"])
    lo, hi = int(inst.nu_lo[i]), int(inst.nu_hi[i])
    sub = grid[..., lo:hi]
    sig = level_opacity_bilinear(sub, p_axis, t_axis, P, T)
    nu = nu_start + np.arange(lo, hi, dtype=np.float64) * dnu
    chi = mass_opacity(sig, X, cfg["mu"])
    if cfg.get("rayleigh_coef", 0.0):
        chi = chi + rayleigh_chi(nu, cfg["rayleigh_coef"], cfg["mu"])[None, :]
    r = transmission.radii(P, T, float(inst.r_planet[i]), cfg["p_ref"], cfg["g"], cfg["mu"])
    Le = deck_levels(P, cfg.get("p_cloud"))
    return transmission.transit_depth(chi[:Le], P[:Le], T[:Le], r[:Le], float(inst.r_star[i]), cfg["mu"])

"""Transmission (transit) geometry.

The paper describes the transit calculation in words (test f01oneline,
Sec. 6.1): compute the slant path of rays at several altitudes through the
layers, the optical depth and transmission along each ray, multiply by 2 pi r
and integrate over altitude.  The details are in the companion paper; the
reading taken here:

* hydrostatic levels with g(r) = g_ref (R_p / r)^2 and r = R_p at P_ref:
  1/r(P) = 1/R_p + k_B / (mu m_u g_ref R_p^2) * integral_{ln P_ref}^{ln P} T dlnP,
  the integral by the trapezoid rule over the levels with P_ref inserted as a
  node (T(P_ref) linear in ln P); exact for an isothermal atmosphere;
* rays with impact parameter b_i = r_i; through the shell between levels k and
  k+1 (k < i) a ray's chord is ds = 2 (sqrt(r_k^2 - b^2) - sqrt(r_{k+1}^2 - b^2))
  and it sees the shell-mean extinction (alpha_k + alpha_{k+1}) / 2, with
  alpha = chi rho, rho = P mu m_u / (k_B T);
* the planet is opaque below the deepest level;
* transit depth delta = [r_bot^2 + 2 integral (1 - exp(-tau(b))) b db] / R_star^2,
  the integral by the trapezoid rule over b = r_{L-1} .. r_0.
"""
import numpy as np

from .constants import K_BOLTZ, AMU, BAR


def radii(p_bar, T, r_planet, p_ref_bar, g, mu_amu):
    """Level radii r_k (cm), levels ordered by increasing pressure."""
    lnp = np.log(np.asarray(p_bar, np.float64))
    T = np.asarray(T, np.float64)
    lnref = np.log(p_ref_bar)
    t_ref = np.interp(lnref, lnp, T)
    nodes = np.concatenate([lnp, [lnref]])
    temps = np.concatenate([T, [t_ref]])
    order = np.argsort(nodes, kind="stable")
    nodes, temps = nodes[order], temps[order]
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (temps[1:] + temps[:-1]) * np.diff(nodes))])
    iref = int(np.nonzero(order == len(lnp))[0][0])
    phi = cum - cum[iref]
    phi_levels = np.empty(len(lnp))
    for pos, orig in enumerate(order):
        if orig < len(lnp):
            phi_levels[orig] = phi[pos]
    C = K_BOLTZ / (mu_amu * AMU * g * r_planet ** 2)
    return 1.0 / (1.0 / r_planet + C * phi_levels)


def transit_depth(chi, p_bar, T, r, r_star, mu_amu):
    """delta(nu) for chi[L][n_nu] (cm^2 g^-1), T[L], radii r[L]; FP64 [n_nu]."""
    chi = np.asarray(chi, np.float64)
    p = np.asarray(p_bar, np.float64) * BAR
    rho = p * mu_amu * AMU / (K_BOLTZ * np.asarray(T, np.float64))
    alpha = chi * rho[:, None]                          # [L][n_nu] cm^-1
    L = len(r)
    abar = 0.5 * (alpha[:-1] + alpha[1:])              # shell k between k, k+1
    f = np.zeros((L, chi.shape[1]))
    for i in range(1, L):
        b = r[i]
        ds = 2.0 * (np.sqrt(r[:i] ** 2 - b * b) - np.sqrt(np.maximum(r[1:i + 1] ** 2 - b * b, 0.0)))
        tau = ds @ abar[:i]
        f[i] = -np.expm1(-tau)
    integ = np.zeros(chi.shape[1])
    for i in range(L - 1):
        integ += 0.5 * (f[i] * r[i] + f[i + 1] * r[i + 1]) * (r[i] - r[i + 1])
    return (r[-1] ** 2 + 2.0 * integ) / r_star ** 2

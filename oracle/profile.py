"""Temperature-pressure profile and abundances of a proposal.

The retrieval model has nine free parameters: five for the T(p) profile of
Line et al. (2013) and four log-abundance scalings (Sec. 7); the profile
generator scales each abundance profile by a constant factor (Sec. 3).  The
T(p) form is cited, not printed; the reading used is the two-stream
three-channel form

  T^4 = 3/4 T_int^4 (2/3 + tau)
      + 3/4 T_irr^4 (1 - alpha) xi(gamma1, tau) + 3/4 T_irr^4 alpha xi(gamma2, tau),
  xi(g, tau) = 2/3 + 2/(3g) [1 + (g tau / 2 - 1) exp(-g tau)]
             + (2g/3) (1 - tau^2 / 2) E2(g tau),
  tau = kappa P / g_surf,   T_irr = beta sqrt(R_star / (2 a)) T_star,

with theta = (log10 kappa, log10 gamma1, log10 gamma2, alpha, beta), T_int
fixed, and T clamped to the opacity grid's temperature range.  Abundances are
X_s = X0_s 10^{a_s}.
"""
import numpy as np
from scipy.special import expn

from .constants import BAR


def xi(gam, tau):
    gt = gam * tau
    return (2.0 / 3.0 + 2.0 / (3.0 * gam) * (1.0 + (gt / 2.0 - 1.0) * np.exp(-gt))
            + 2.0 * gam / 3.0 * (1.0 - tau ** 2 / 2.0) * expn(2, gt))


def temperature(theta, p_bar, g, t_int, t_star, r_star, a_orbit, t_min=None, t_max=None):
    """T at pressures p_bar for one proposal theta[0:5] (FP64)."""
    lk, lg1, lg2, alpha, beta = (float(v) for v in theta[:5])
    kappa, g1, g2 = 10.0 ** lk, 10.0 ** lg1, 10.0 ** lg2
    tau = kappa * np.asarray(p_bar, np.float64) * BAR / g
    t_irr = beta * np.sqrt(r_star / (2.0 * a_orbit)) * t_star
    T4 = (0.75 * t_int ** 4 * (2.0 / 3.0 + tau)
          + 0.75 * t_irr ** 4 * (1.0 - alpha) * xi(g1, tau)
          + 0.75 * t_irr ** 4 * alpha * xi(g2, tau))
    T = T4 ** 0.25
    if t_min is not None:
        T = np.clip(T, t_min, t_max)
    return T


def abundances(theta, x0):
    """X_s = X0_s 10^{a_s} for the log-abundance scalings theta[5:]."""
    a = np.asarray(theta[5:5 + len(x0)], np.float64)
    return np.asarray(x0, np.float64) * 10.0 ** a

"""Gray cloud deck and Rayleigh scattering opacity (FP64, test infrastructure).

Sec. 3 lists both among the transit code's capabilities without a formula; the
readings taken here are:

* gray cloud deck: an opaque surface at pressure p_cloud.  On a set of levels
  ordered by increasing pressure, the deck sits on the first level with
  P_k >= p_cloud (a deck between two levels moves down to the deeper one), and
  the atmosphere ends there: that level is the last one the integration sees.
  At least two levels remain (a deck above the second level acts at the
  second).  No level at or below p_cloud, or p_cloud <= 0: no deck.
  Emission then takes that level's blackbody as the bottom boundary;
  transmission takes the planet as opaque below it.  Altitudes are still
  those of the whole hydrostatic column (the deck does not move P_ref).
* Rayleigh scattering: extinction by the bulk gas with a cross-section per
  molecule sigma_R = a nu^4 (a in cm^2 (cm^-1)^-4, e.g. about 8.4e-45 for H2
  in the near infrared), i.e. a mass opacity chi_R = a nu^4 / (mu m_u) added
  at every level, treated as extinction (no scattered source), like the line
  opacity.  a = 0: off.
"""
import numpy as np

from .constants import AMU


def deck_levels(p_bar, p_cloud):
    """Number of levels the integration keeps with a deck at p_cloud (bar)."""
    p = np.asarray(p_bar, np.float64)
    L = p.size
    if p_cloud is None or not (p_cloud > 0):
        return L
    at = np.nonzero(p >= p_cloud)[0]
    if at.size == 0:
        return L
    return max(int(at[0]) + 1, 2)


def rayleigh_chi(nu, coef, mu_amu):
    """chi_R(nu) = a nu^4 / (mu m_u) in cm^2 g^-1."""
    nu = np.asarray(nu, np.float64)
    if not coef:
        return np.zeros(nu.shape)
    return coef * nu ** 4 / (mu_amu * AMU)

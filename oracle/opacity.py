"""Line-by-line opacity, point-sampled on the output wavenumber grid.

The paper's opacity grid (Sec. 3, the radiative-transfer module's table;
Sec. 4 items 3-4) holds, per molecule, the opacity on the
output wavenumber grid over the layer pressures and a grid of temperatures.
Lines are sampled at the grid wavenumbers, not bin-averaged (Sec. 4, text after
the list of optimisations).  The line-strength and width formulas live in the
companion paper and are not printed; the readings used here are:

* strength (HITRAN convention, T_ref = 296 K, Q(T)/Q(T_ref) = (T/T_ref)^1.5):
  S(T) = S_ref (T_ref/T)^1.5 exp(-c2 E'' (1/T - 1/T_ref))
         (1 - exp(-c2 nu0 / T)) / (1 - exp(-c2 nu0 / T_ref));
* Doppler width: the Gaussian standard deviation of Eq. 2,
  sigma = (nu0 / c) sqrt(k T / m);
* Lorentz half width: gamma = gamma_ref (P / 1 bar) (T_ref / T)^0.5;
* profile cutoff: hard and inclusive, |nu_j - nu0| <= cutoff, with
  nu_j = nu_start + j*dnu and nu_j - nu0 evaluated in FP64 in that order;
* no renormalisation of the truncated profile; by default no line-strength
  threshold.  With rel_threshold > 0 (Sec. 4 item 6) a line whose S(T) is
  below rel_threshold times the strongest line of the list at that T (and P)
  is left out.

The opacity of species s at grid point j is the plain sum
sigma_s(nu_j) = sum_i S_i V(nu_j - nu0_i; sigma_i, gamma_i)   [cm^2 molecule^-1],
added per point with math.fsum.
"""
import math
import numpy as np

from .constants import C2, C_LIGHT, K_BOLTZ, AMU, T_REF
from .voigt import voigt


def line_strength(log10_s296, nu0, elow, T):
    """S(T) in cm molecule^-1 (reading above)."""
    s_ref = 10.0 ** np.asarray(log10_s296, np.float64)
    nu0 = np.asarray(nu0, np.float64)
    elow = np.asarray(elow, np.float64)
    boltz = np.exp(-C2 * elow * (1.0 / T - 1.0 / T_REF))
    stim = (1.0 - np.exp(-C2 * nu0 / T)) / (1.0 - np.exp(-C2 * nu0 / T_REF))
    return s_ref * (T_REF / T) ** 1.5 * boltz * stim


def doppler_sigma(nu0, T, mass_amu):
    """Gaussian standard deviation in cm^-1."""
    return np.asarray(nu0, np.float64) / C_LIGHT * math.sqrt(K_BOLTZ * T / (mass_amu * AMU))


def lorentz_gamma(gamma_ref, p_bar, T):
    """Lorentz half width in cm^-1."""
    return np.asarray(gamma_ref, np.float64) * p_bar * math.sqrt(T_REF / T)


def opacity_cell(lines, p_bar, T, nu_start, dnu, n_nu, cutoff, j_lo=0, j_hi=None, rel_threshold=0.0):
    """Opacity of one species at one (P, T) on grid points j in [j_lo, j_hi).

    `lines` carries nu0, log10_s296, elow, gamma_ref, mass_amu.  For every grid
    point the contributions of all lines within the cutoff (and, with
    rel_threshold > 0, at or above the strength bound) are evaluated and added
    with math.fsum.  Returns an FP64 array of length j_hi - j_lo.
    """
    if j_hi is None:
        j_hi = n_nu
    n = j_hi - j_lo
    out = np.zeros(max(n, 0))
    if n <= 0:
        return out
    s_floor = 0.0
    if rel_threshold > 0 and len(lines.nu0):
        s_floor = rel_threshold * float(np.max(line_strength(lines.log10_s296, lines.nu0, lines.elow, T)))
    # Points are processed in chunks narrow against the cutoff so that the
    # (point x candidate line) matrix stays small.
    chunk = max(1, int(cutoff / (4.0 * dnu)))
    for c0 in range(j_lo, j_hi, chunk):
        c1 = min(c0 + chunk, j_hi)
        j = np.arange(c0, c1, dtype=np.int64)
        nu = nu_start + j.astype(np.float64) * dnu
        lo = np.searchsorted(lines.nu0, nu[0] - cutoff - dnu, side="left")
        hi = np.searchsorted(lines.nu0, nu[-1] + cutoff + dnu, side="right")
        if hi <= lo:
            continue
        nu0 = lines.nu0[lo:hi]
        S = line_strength(lines.log10_s296[lo:hi], nu0, lines.elow[lo:hi], T)
        sig = doppler_sigma(nu0, T, lines.mass_amu)
        gam = lorentz_gamma(lines.gamma_ref[lo:hi], p_bar, T)
        d = nu[:, None] - nu0[None, :]
        inside = (np.abs(d) <= cutoff) & (S[None, :] >= s_floor)
        v = S[None, :] * voigt(d, sig[None, :], gam[None, :])
        for r in range(j.size):
            out[c0 - j_lo + r] = math.fsum(v[r][inside[r]])
    return out


def opacity_cells(species, p_bar, t_K, nu_start, dnu, n_nu, cutoff, rel_threshold=0.0):
    """Direct opacity at each cell's own (P, T), computed for the cell (Sec. 3).

    Returns FP64 [n_species][n_cells][n_nu].
    """
    out = np.zeros((len(species), len(p_bar), n_nu))
    for s, ll in enumerate(species):
        for c in range(len(p_bar)):
            out[s, c] = opacity_cell(ll, p_bar[c], t_K[c], nu_start, dnu, n_nu, cutoff,
                                     rel_threshold=rel_threshold)
    return out


def opacity_grid(species, p_bar, t_K, nu_start, dnu, n_nu, cutoff):
    """Opacity grid [n_species][n_layers][n_temps][n_nu] (FP64)."""
    out = np.zeros((len(species), len(p_bar), len(t_K), n_nu))
    for s, ll in enumerate(species):
        for k, p in enumerate(p_bar):
            for m, T in enumerate(t_K):
                out[s, k, m] = opacity_cell(ll, p, T, nu_start, dnu, n_nu, cutoff)
    return out

"""The paper's own opacity scheme: a precomputed table of Voigt profiles (FP64,
test infrastructure).

Sec. 4 items 4-5 and the sampling text after the list, Sec. 6.1.1 (test
f04broadening): before the opacity grid is built, Voigt profiles are tabulated
for a grid of Doppler and Lorentz widths, each sampled finely (several samples
per output-grid interval) and aligned to the output grid.  A line then uses the
profile whose widths are closest to its own, shifted by a whole number of
samples so that its peak falls as close as possible to the line centre, and
the shifted profile is read at the output wavenumbers.  The paper gives the
size it uses (60 x 60 widths) but neither the spacing of the width grid nor
how closeness is measured; the readings here are:

* widths: n_sigma Doppler widths and n_gamma Lorentz widths, each log-spaced
  between the caller's bounds; the closest profile is the nearest node in
  ln sigma and in ln gamma separately (clamped to the bounds);
* position: the line centre is rounded to the nearest fine sample,
  s = round((nu0 - nu_start) * O / dnu), i.e. the profile's peak sits at
  nu_start + s dnu / O;
* the cutoff window and the point sampling are those of the direct sum
  (``oracle.opacity``): |nu_j - nu0| <= cutoff with the exact nu0.

The result at grid point j is sum_i S_i V(nu_j - nu0_i^q; sigma_i^q, gamma_i^q),
with nu0^q, sigma^q, gamma^q the quantised centre and widths, added per point
with math.fsum.  Written from that definition, not from a table: the table is
only a cache of these values.
"""
import math
import numpy as np

from .opacity import line_strength, doppler_sigma, lorentz_gamma
from .voigt import voigt


def width_nodes(lo, hi, n):
    """n log-spaced nodes from lo to hi (n = 1: lo)."""
    if n == 1:
        return np.array([lo], np.float64)
    return np.exp(np.linspace(math.log(lo), math.log(hi), n))


def nearest_node(v, lo, hi, n):
    """Index of the node nearest to v in ln v, clamped to [0, n - 1]."""
    if n == 1:
        return np.zeros(np.shape(v), np.int64)
    step = (math.log(hi) - math.log(lo)) / (n - 1)
    k = np.floor((np.log(np.asarray(v, np.float64)) - math.log(lo)) / step + 0.5)
    return np.clip(k, 0, n - 1).astype(np.int64)


def quantised_centre(nu0, nu_start, dnu, oversample):
    """Line centre rounded to the nearest of the oversample samples per grid interval."""
    s = np.floor((np.asarray(nu0, np.float64) - nu_start) * oversample / dnu + 0.5)
    return nu_start + s * dnu / oversample


def opacity_cell_table(lines, p_bar, T, nu_start, dnu, n_nu, cutoff, table):
    """Opacity of one species at one (P, T) with the table scheme.

    `table` holds n_sigma, sigma_lo, sigma_hi, n_gamma, gamma_lo, gamma_hi and
    oversample.  Returns FP64 [n_nu]."""
    nu = nu_start + np.arange(n_nu, dtype=np.float64) * dnu
    out = np.zeros(n_nu)
    if len(lines.nu0) == 0:
        return out
    S = line_strength(lines.log10_s296, lines.nu0, lines.elow, T)
    sig = doppler_sigma(lines.nu0, T, lines.mass_amu)
    gam = lorentz_gamma(lines.gamma_ref, p_bar, T)
    sn = width_nodes(table["sigma_lo"], table["sigma_hi"], table["n_sigma"])
    gn = width_nodes(table["gamma_lo"], table["gamma_hi"], table["n_gamma"])
    sq = sn[nearest_node(sig, table["sigma_lo"], table["sigma_hi"], table["n_sigma"])]
    gq = gn[nearest_node(gam, table["gamma_lo"], table["gamma_hi"], table["n_gamma"])]
    cq = quantised_centre(lines.nu0, nu_start, dnu, table["oversample"])
    terms = [[] for _ in range(n_nu)]
    for i in range(len(lines.nu0)):
        d_exact = nu - lines.nu0[i]
        inside = np.nonzero(np.abs(d_exact) <= cutoff)[0]
        if inside.size == 0:
            continue
        v = S[i] * voigt(nu[inside] - cq[i], sq[i], gq[i])
        for j, x in zip(inside, v):
            terms[j].append(x)
    for j in range(n_nu):
        out[j] = math.fsum(terms[j])
    return out


def opacity_cells_table(species, p_bar, t_K, nu_start, dnu, n_nu, cutoff, table):
    """FP64 [n_species][n_cells][n_nu] with the table scheme."""
    out = np.zeros((len(species), len(p_bar), n_nu))
    for s, ll in enumerate(species):
        for c in range(len(p_bar)):
            out[s, c] = opacity_cell_table(ll, p_bar[c], t_K[c], nu_start, dnu, n_nu, cutoff, table)
    return out

"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only draws random numbers and lays out arrays: line lists, pressure
and temperature axes, proposal parameters, filter transmission curves and
instance shapes.  It holds none of the method's arithmetic (no line strengths,
widths, profiles, optical depths or band integrals) so that neither side of a
parity test depends on the other through it.

Workloads (shapes follow the paper's retrieval setup, Sec. 7: 100 layers over
1e-8..100 bar, nine free parameters; line statistics are synthetic):

* ``emission_small``     2 species x 10,000 lines, 60 layers (1e-6..100 bar),
                         2,000 wavenumbers (1 cm^-1), 4 angles, 4 top-hat bands.
* ``opacity_grid``       3 species, 5e6 lines in total, 100 layers (1e-8..100 bar)
                         x 20 temperatures (500..3000 K) x 100,000 wavenumbers
                         (0.02 cm^-1 over 1000..3000 cm^-1), cutoff 25 cm^-1.
* ``emission_batch``     2,048 proposals on a 4-species grid of the same axes,
                         8 angles, 10 Gaussian filters.
* ``transmission_batch`` 1,024 instances with 40..150 levels and spans of
                         10,000..100,000 wavenumbers, 12 Gaussian filters.
* ``surrogate_demc``     16 chains, 9 parameters, MLP 9-256-256-256-10.

Seeds (numpy PCG64): line list of species s -> 1000+s; proposal draws of
generation g -> 2000+g; filters -> 3000; instance shapes -> 4000; MLP
initialisation -> 5000; DE-MC chain c -> 6000+c.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Physical inputs quoted by the paper for its HD 189733 b-like test planet
# (Sec. 6.2): stellar radius 0.756 R_sun, T_star 5000 K, planet radius
# 1.138 R_J, gravity 2182.73 cm s^-2, reference pressure 0.1 bar; orbit
# 0.0312 AU (Sec. 7).  IAU nominal radii.
R_SUN_CM = 6.957e10
R_JUP_CM = 7.1492e9
AU_CM = 1.495978707e13
HD189_RSTAR_CM = 0.756 * R_SUN_CM
HD189_TSTAR_K = 5000.0
HD189_RPLANET_CM = 1.138 * R_JUP_CM
HD189_GRAV_CGS = 2182.73
HD189_PREF_BAR = 0.1
HD189_A_CM = 0.0312 * AU_CM

SPECIES_MASS_AMU = (18.0, 28.0, 44.0, 16.0)   # H2O-, CO-, CO2-, CH4-like
BASE_VMR = 1e-4                                # X0_s, scaled by 10**a_s
MEAN_MOLECULAR_MASS_AMU = 2.3                  # H2/He background
T_INT_K = 100.0

# Prior box of the 5-parameter T(P) profile and the log-abundance scalings.
THETA_LO = np.array([-3.0, -1.5, -1.5, 0.0, 0.7, -3.0, -3.0, -3.0, -3.0])
THETA_HI = np.array([0.0, 1.0, 1.0, 1.0, 1.3, 3.0, 3.0, 3.0, 3.0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclasses.dataclass
class LineList:
    """One species' line list, sorted by line centre (structure of arrays)."""
    nu0: np.ndarray          # float64 [n] line centres, cm^-1
    log10_s296: np.ndarray   # float32 [n] log10 strength at 296 K, cm/molecule
    elow: np.ndarray         # float32 [n] lower-state energy, cm^-1
    gamma_ref: np.ndarray    # float32 [n] Lorentz HWHM at 1 bar and 296 K, cm^-1
    mass_amu: float

    @property
    def n(self) -> int:
        return int(self.nu0.shape[0])


# second radiation constant h c / k_B (cm K), for the lower-state population
# of the synthetic line strengths at 296 K
_C2_CM_K = 1.438776877


def line_list(species: int, n_lines: int, nu_lo: float = 1000.0, nu_hi: float = 3000.0) -> LineList:
    """Seeded synthetic line list, sorted by centre: centres U[nu_lo, nu_hi],
    E'' U[0, 5000] cm^-1, gamma_ref U[0.05, 0.1] cm^-1, and strengths at 296 K
    S = S_int exp(-c2 E'' / 296 K) with log10 S_int U[-25, -19]: a line from a
    highly excited lower state is weak at 296 K (its population), as in real
    line lists, so that hot layers are not made opaque by lines that are
    strong at every temperature."""
    g = _rng(1000 + species)
    nu0 = g.uniform(nu_lo, nu_hi, n_lines)
    logs = g.uniform(-25.0, -19.0, n_lines)
    elow = g.uniform(0.0, 5000.0, n_lines)
    logs = logs - _C2_CM_K * elow / (296.0 * np.log(10.0))
    gam = g.uniform(0.05, 0.1, n_lines)
    order = np.argsort(nu0, kind="stable")
    return LineList(nu0=nu0[order].astype(np.float64),
                    log10_s296=logs[order].astype(np.float32),
                    elow=elow[order].astype(np.float32),
                    gamma_ref=gam[order].astype(np.float32),
                    mass_amu=SPECIES_MASS_AMU[species])


def split_lines(total: int, n_species: int) -> list[int]:
    """Split a total line count over species as evenly as possible (first
    species get the remainder): 5e6 over 3 -> 1,666,667/1,666,667/1,666,666."""
    base, rem = divmod(total, n_species)
    return [base + (1 if s < rem else 0) for s in range(n_species)]


def log_pressures(n: int, p_top_bar: float, p_bot_bar: float) -> np.ndarray:
    """Levels evenly spaced in log pressure, index 0 at the top (lowest P)."""
    return np.logspace(np.log10(p_top_bar), np.log10(p_bot_bar), n)


def nu_axis(nu_start: float, dnu: float, n: int) -> np.ndarray:
    """Wavenumber grid nu_j = nu_start + j*dnu (evaluated in this order)."""
    return nu_start + np.arange(n, dtype=np.float64) * dnu


def inversion_profile(p_bar: np.ndarray) -> np.ndarray:
    """Fixed isothermal-plus-inversion profile: 1500 K aloft, 800 K deep,
    transition near 1 mbar."""
    return 800.0 + 700.0 * 0.5 * (1.0 - np.tanh((np.log10(p_bar) + 3.0) / 0.5))


def proposals(n: int, generation: int = 0, n_species: int = 4) -> np.ndarray:
    """[n][5+n_species] float32 draws uniform in the prior box."""
    g = _rng(2000 + generation)
    k = 5 + n_species
    u = g.uniform(0.0, 1.0, (n, 9))[:, :k]
    th = THETA_LO[:k] + u * (THETA_HI[:k] - THETA_LO[:k])
    return th.astype(np.float32)


def tophat_filters(nu: np.ndarray, edges) -> np.ndarray:
    """[n_bands][n_nu] float32, 1 inside [edge_b, edge_{b+1}), else 0."""
    w = np.zeros((len(edges) - 1, nu.size), np.float32)
    for b in range(len(edges) - 1):
        w[b] = ((nu >= edges[b]) & (nu < edges[b + 1])).astype(np.float32)
    return w


def gaussian_filters(nu: np.ndarray, n_bands: int, lo: float, hi: float,
                     fwhm_lo: float, fwhm_hi: float, seed: int = 3000) -> np.ndarray:
    """[n_bands][n_nu] float32 Gaussian transmission curves with seeded centres
    in [lo, hi] and FWHM in [fwhm_lo, fwhm_hi], truncated at +-3 sigma."""
    g = _rng(seed)
    cen = g.uniform(lo, hi, n_bands)
    fwhm = g.uniform(fwhm_lo, fwhm_hi, n_bands)
    sig = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    w = np.zeros((n_bands, nu.size), np.float32)
    for b in range(n_bands):
        d = (nu - cen[b]) / sig[b]
        w[b] = np.where(np.abs(d) <= 3.0, np.exp(-0.5 * d * d), 0.0).astype(np.float32)
    return w


@dataclasses.dataclass
class Instances:
    """Uneven transmission instances (one spherical-shell atmosphere each)."""
    n_levels: np.ndarray   # int32 [n]
    nu_lo: np.ndarray      # int64 [n] first grid index of the span
    nu_hi: np.ndarray      # int64 [n] one past the last grid index
    r_planet: np.ndarray   # float32 [n] cm, radius at the reference pressure
    r_star: np.ndarray     # float32 [n] cm
    theta: np.ndarray      # float32 [n][9]

    @property
    def offsets(self) -> np.ndarray:
        """int64 [n+1] packing offsets of the spectra."""
        return np.concatenate([[0], np.cumsum(self.nu_hi - self.nu_lo)]).astype(np.int64)


def instances(n: int, n_nu_grid: int, lmin: int = 40, lmax: int = 150,
              span_lo: int = 10_000, span_hi: int = 100_000, seed: int = 4000) -> Instances:
    g = _rng(seed)
    nl = g.integers(lmin, lmax + 1, n).astype(np.int32)
    span = g.integers(span_lo, min(span_hi, n_nu_grid) + 1, n).astype(np.int64)
    lo = np.array([g.integers(0, n_nu_grid - s + 1) for s in span], np.int64)
    rp = (g.uniform(1.0, 1.4, n) * R_JUP_CM).astype(np.float32)
    rs = (g.uniform(0.7, 1.2, n) * R_SUN_CM).astype(np.float32)
    u = g.uniform(0.0, 1.0, (n, 9))
    th = (THETA_LO + u * (THETA_HI - THETA_LO)).astype(np.float32)
    return Instances(nl, lo, lo + span, rp, rs, th)


# ---------------------------------------------------------------- workloads
@dataclasses.dataclass
class EmissionSmall:
    species: list
    p_bar: np.ndarray
    t_K: np.ndarray
    nu_start: float
    dnu: float
    n_nu: int
    cutoff: float
    n_angles: int
    filters: np.ndarray
    log_ab: np.ndarray      # [n_species] log10 abundance scalings (0 = X0)


def emission_small() -> EmissionSmall:
    p = log_pressures(60, 1e-6, 100.0)
    nu = nu_axis(1000.0, 1.0, 2000)
    return EmissionSmall(species=[line_list(s, 10_000) for s in range(2)],
                         p_bar=p, t_K=inversion_profile(p), nu_start=1000.0, dnu=1.0,
                         n_nu=2000, cutoff=25.0, n_angles=4,
                         filters=tophat_filters(nu, [1000.0, 1500.0, 2000.0, 2500.0, 3000.0]),
                         log_ab=np.zeros(2, np.float32))


@dataclasses.dataclass
class GridAxes:
    p_bar: np.ndarray
    t_K: np.ndarray
    nu_start: float
    dnu: float
    n_nu: int
    cutoff: float


def grid_axes(n_layers: int = 100, n_temps: int = 20, n_nu: int = 100_000,
              dnu: float = 0.02) -> GridAxes:
    return GridAxes(p_bar=log_pressures(n_layers, 1e-8, 100.0),
                    t_K=np.linspace(500.0, 3000.0, n_temps),
                    nu_start=1000.0, dnu=dnu, n_nu=n_nu, cutoff=25.0)


def opacity_grid_species(n_species: int = 3, total_lines: int = 5_000_000) -> list:
    """Line lists of the opacity-grid workload (the 4-species variant adds a
    fourth species with the same per-species count)."""
    counts = split_lines(total_lines, 3)
    if n_species == 4:
        counts = counts + [counts[0]]
    return [line_list(s, counts[s]) for s in range(n_species)]


def opacity_field(n_species: int, p_bar: np.ndarray, t_K: np.ndarray, n_nu: int,
                  seed: int = 3500) -> np.ndarray:
    """Seeded stand-in for an opacity grid, float32 [S][L][M][n_nu] in cm^2 per
    molecule, for tests of the per-proposal forward model at full layer and
    temperature counts without building a grid from lines.  Random numbers
    only: per species a base level U[-23.5, -21.5] (log10), a random walk over
    wavenumber detrended and scaled to +-2.5 decades, sparse spikes of up to
    +3 decades that fall off by a random factor per point, a random slope in
    log10 P per (species, layer) and a random temperature trend per
    (species, wavenumber), clipped to [1e-30, 1e-16].  Optical depths of
    1 then fall anywhere from 1e-4 to 1e4 bar in the 9-parameter prior."""
    g = _rng(seed)
    L, M = len(p_bar), len(t_K)
    lp = (np.log10(np.asarray(p_bar, np.float64)) + 3.0)[:, None]        # [L, 1]
    tt = ((np.asarray(t_K, np.float64) - 1750.0) / 1250.0)[:, None]       # [M, 1]
    out = np.empty((n_species, L, M, n_nu), np.float32)
    j = np.arange(n_nu)
    for s in range(n_species):
        walk = np.cumsum(g.normal(0.0, 0.2, n_nu))
        walk -= np.polyval(np.polyfit(j, walk, 1), j)
        walk *= 2.5 / max(np.max(np.abs(walk)), 1e-12)
        spikes = np.zeros(n_nu)
        for c in g.integers(0, n_nu, max(1, n_nu // 50)):
            h, q = g.uniform(0.5, 3.0), g.uniform(0.5, 0.9)
            spikes = np.maximum(spikes, h * q ** np.abs(j - c))
        row = g.uniform(-23.5, -21.5) + walk + spikes                        # [n_nu]
        pslope = g.uniform(-0.3, 0.3, (L, 1))
        tslope = g.uniform(-1.0, 1.0, (1, n_nu))
        for k in range(L):
            lg = row[None, :] + pslope[k] * lp[k] + tslope * tt + g.normal(0.0, 0.05, (M, n_nu))
            out[s, k] = (10.0 ** np.clip(lg, -30.0, -16.0)).astype(np.float32)
    return out


SURROGATE_WIDTHS = (9, 256, 256, 256, 10)


def mlp_init(widths=SURROGATE_WIDTHS, seed: int = 5000) -> np.ndarray:
    """Flat FP32 initial parameters: per layer W [out][in] ~ N(0, 2/in) then
    b = 0 (the layout of the surrogate network)."""
    g = _rng(seed)
    parts = []
    for l in range(len(widths) - 1):
        n_in, n_out = widths[l], widths[l + 1]
        parts.append(g.normal(0.0, np.sqrt(2.0 / n_in), n_out * n_in))
        parts.append(np.zeros(n_out))
    return np.concatenate(parts).astype(np.float32)

"""Pins of the oracle's version of the paper's Voigt-table opacity scheme
(Sec. 4 items 4-5 and the sampling text; Sec. 6.1.1, test f04broadening)."""
import dataclasses
import math

import numpy as np

from oracle import opacity as O
from oracle import voigt_table as VT


@dataclasses.dataclass
class Lines:
    nu0: np.ndarray
    log10_s296: np.ndarray
    elow: np.ndarray
    gamma_ref: np.ndarray
    mass_amu: float


def _lines(nu0, logs, elow, gam, mass=18.0):
    return Lines(np.asarray(nu0, np.float64), np.asarray(logs, np.float32),
                 np.asarray(elow, np.float32), np.asarray(gam, np.float32), mass)


def _exact_table(ll, p, T, oversample):
    # one node per width axis, placed at the line's own widths
    s = float(O.doppler_sigma(ll.nu0[0], T, ll.mass_amu))
    g = float(O.lorentz_gamma(ll.gamma_ref[0], p, T))
    return dict(n_sigma=1, sigma_lo=s, sigma_hi=s, n_gamma=1, gamma_lo=g, gamma_hi=g, oversample=oversample)


def test_reduces_to_the_direct_sum_on_nodes():
    # Widths on nodes and the centre on a fine sample: no quantisation at all.
    dnu, O_s = 0.01, 16
    ll = _lines([1500.0 + 37 * dnu + 5 * dnu / O_s], [-20.0], [700.0], [0.07])
    tab = _exact_table(ll, 0.2, 1100.0, O_s)
    got = VT.opacity_cell_table(ll, 0.2, 1100.0, 1499.0, dnu, 400, 1.5, tab)
    exp = O.opacity_cell(ll, 0.2, 1100.0, 1499.0, dnu, 400, 1.5)
    # the centre is on a fine sample up to the FP64 rounding of nu0 (~1e-13 cm^-1)
    assert np.max(np.abs(got - exp)) <= 1e-10 * np.max(exp)


def test_the_shift_is_the_only_change():
    # Widths on nodes: the table result is the direct sum of the same line moved
    # to its quantised centre (cutoff wider than the grid, so the windows agree).
    dnu = 0.01
    for nu0 in (1500.3337, 1500.30001, 1500.1249):
        ll = _lines([nu0], [-20.0], [700.0], [0.07])
        for O_s in (4, 16, 64):
            cq = float(VT.quantised_centre(ll.nu0, 1499.0, dnu, O_s)[0])
            moved = _lines([cq], [-20.0], [700.0], [0.07])
            got = VT.opacity_cell_table(ll, 1e-3, 1100.0, 1499.0, dnu, 300, 10.0,
                                        _exact_table(ll, 1e-3, 1100.0, O_s))
            exp = O.opacity_cell(moved, 1e-3, 1100.0, 1499.0, dnu, 300, 10.0)
            # the moved line's own strength and Doppler width differ from the
            # original's by O((cq - nu0)/nu0) < 1e-6, which steep parts of the
            # profile turn into up to ~1e-5
            assert np.max(np.abs(got / exp - 1)) < 2e-5


def test_nearest_node_by_brute_force():
    rng = np.random.default_rng(7)
    lo, hi = 0.003, 0.05
    for n in (1, 2, 3, 60):
        nodes = VT.width_nodes(lo, hi, n)
        assert len(nodes) == n
        assert abs(nodes[0] - lo) < 1e-15 and (n == 1 or abs(nodes[-1] / hi - 1) < 1e-14)
        v = np.exp(rng.uniform(math.log(lo) - 0.5, math.log(hi) + 0.5, 2000))
        k = VT.nearest_node(v, lo, hi, n)
        brute = np.argmin(np.abs(np.log(v)[:, None] - np.log(nodes)[None, :]), axis=1)
        assert np.array_equal(k, brute)


def test_window_of_a_single_point_and_the_inclusive_cutoff():
    # A cutoff shorter than the grid step leaves each line at most one point,
    # or two at exactly one cutoff on either side (|d| <= cutoff); the grid
    # step and offsets are exact binary fractions.
    dnu = 0.25
    ll = _lines([1500.0 + 40 * dnu, 1500.0 + 120.5 * dnu], [-20.0, -20.5], [700.0, 100.0], [0.07, 0.07])
    tab = _exact_table(ll, 0.2, 1100.0, 2)
    got = VT.opacity_cell_table(ll, 0.2, 1100.0, 1500.0, dnu, 200, 0.5 * dnu, tab)
    assert list(np.nonzero(got)[0]) == [40, 120, 121]
    S = O.line_strength(ll.log10_s296, ll.nu0, ll.elow, 1100.0)
    v0 = S[0] * O.voigt(0.0, tab["sigma_lo"], tab["gamma_lo"])
    assert abs(got[40] / v0 - 1) < 1e-12


def test_quantised_centre_is_within_half_a_sample():
    rng = np.random.default_rng(8)
    nu0 = rng.uniform(1000, 1010, 500)
    for O_s in (1, 8, 64):
        c = VT.quantised_centre(nu0, 1000.0, 0.02, O_s)
        assert np.all(np.abs(c - nu0) <= 0.5 * 0.02 / O_s + 1e-12)
        # on the fine grid
        k = (c - 1000.0) * O_s / 0.02
        assert np.all(np.abs(k - np.round(k)) < 1e-6)


def test_width_quantisation_error_converges_to_the_papers_bound():
    # f04broadening-like layer (Sec. 6.1.1): 0.33516 bar and 1442.58 K, a table
    # spanning the list's widths at that layer, sampled 1,000 times per grid
    # interval (the paper samples its profiles thousands of times per
    # interval).  The error comes from the nearest-width choice and falls as
    # the width nodes get denser; with dense nodes it is below the paper's
    # 0.1% (with 60 x 60 nodes over this list's factor-2 range of Lorentz
    # widths it is ~0.4%).
    rng = np.random.default_rng(9)
    n = 60
    ll = _lines(np.sort(rng.uniform(1500.0, 1520.0, n)), rng.uniform(-22, -20, n), rng.uniform(0, 3000, n),
                rng.uniform(0.05, 0.1, n))
    p, T = 0.33516, 1442.58
    sig = O.doppler_sigma(ll.nu0, T, ll.mass_amu)
    gam = O.lorentz_gamma(ll.gamma_ref, p, T)
    exp = O.opacity_cell(ll, p, T, 1495.0, 0.01, 3000, 5.0)
    big = exp > 1e-3 * exp.max()
    errs = []
    for nodes in (60, 600, 6000):
        tab = dict(n_sigma=nodes, sigma_lo=float(sig.min()), sigma_hi=float(sig.max()), n_gamma=nodes,
                   gamma_lo=float(gam.min()), gamma_hi=float(gam.max()), oversample=1000)
        got = VT.opacity_cell_table(ll, p, T, 1495.0, 0.01, 3000, 5.0, tab)
        errs.append(np.max(np.abs(got[big] / exp[big] - 1)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3
    assert errs[0] < 1e-2

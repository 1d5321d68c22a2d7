"""Pins of the oracle's line strengths, widths and point-sampled opacity
(Sec. 4 items 3-4 and the sampling text after them; tests f01-f03 ideas,
Sec. 6.1 Table 1)."""
import dataclasses
import numpy as np

from oracle import opacity as O
from oracle import voigt as V


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


def test_strength_at_reference_temperature():
    s = O.line_strength(np.float32(-20.0), 2000.0, np.float32(1234.0), 296.0)
    assert abs(s / 10.0 ** np.float64(np.float32(-20.0)) - 1.0) < 1e-14


def test_strength_ground_state_limit():
    # E'' = 0 and c2 nu0 / T >> 1: only the partition-function ratio remains.
    for T in (500.0, 1500.0):
        s = O.line_strength(0.0, 40000.0, 0.0, T)
        assert abs(s - (296.0 / T) ** 1.5) < 1e-12


def test_strength_boltzmann_slope():
    # log S vs E'' at fixed nu0 is linear with slope -c2 (1/T - 1/296) / ln 10,
    # with c2 = 1.4387769 cm K (textbook second radiation constant).
    E = np.linspace(0, 5000, 11)
    T = 1200.0
    ls = np.log10(O.line_strength(np.zeros(11), np.full(11, 2000.0), E, T))
    slope = np.polyfit(E, ls, 1)[0]
    assert abs(slope / (-1.4387769 * (1 / T - 1 / 296.0) / np.log(10)) - 1) < 1e-6


def test_doppler_width_textbook_constant():
    # Doppler FWHM = 7.1623e-7 nu0 sqrt(T / M[amu]) (textbook constant)
    fwhm = 2 * np.sqrt(2 * np.log(2)) * O.doppler_sigma(2000.0, 1500.0, 18.0)
    assert abs(fwhm / (7.1623e-7 * 2000.0 * np.sqrt(1500.0 / 18.0)) - 1) < 2e-5


def test_lorentz_width_scaling():
    assert abs(O.lorentz_gamma(0.07, 1.0, 296.0) - 0.07) < 1e-16
    assert abs(O.lorentz_gamma(0.07, 3.0, 4 * 296.0) - 0.07 * 3 / 2) < 1e-15


def test_single_line_brute_force():
    # f01oneline idea: one line gives S V at every point within the cutoff, 0 outside.
    ll = _lines([1500.3], [-20.0], [800.0], [0.07])
    p, T = 0.5, 1100.0
    out = O.opacity_cell(ll, p, T, 1400.0, 0.1, 2000, 25.0)
    nu = 1400.0 + np.arange(2000) * 0.1
    S = O.line_strength(ll.log10_s296, ll.nu0, ll.elow, T)[0]
    sig = O.doppler_sigma(1500.3, T, 18.0)
    gam = O.lorentz_gamma(np.float32(0.07), p, T)
    d = nu - 1500.3
    exp = np.where(np.abs(d) <= 25.0, S * V.voigt(d, sig, gam), 0.0)
    assert np.max(np.abs(out - exp)) <= 1e-14 * np.max(exp)
    assert np.count_nonzero(out) == np.count_nonzero(np.abs(d) <= 25.0)


def test_cutoff_is_inclusive_on_exact_points():
    ll = _lines([1025.0], [-20.0], [0.0], [0.07])      # nu_0 - 25 is exactly grid point 0
    out = O.opacity_cell(ll, 1.0, 1000.0, 1000.0, 1.0, 60, 25.0)
    assert out[0] > 0 and out[50] > 0 and out[51] == 0.0


def test_additivity_over_line_lists():
    # f02/f03 idea: the opacity of a union of lists is the sum of their opacities.
    rng = np.random.default_rng(7)
    a = _lines(np.sort(rng.uniform(1000, 1100, 30)), rng.uniform(-24, -19, 30),
               rng.uniform(0, 3000, 30), rng.uniform(0.05, 0.1, 30))
    b = _lines(np.sort(rng.uniform(1000, 1100, 20)), rng.uniform(-24, -19, 20),
               rng.uniform(0, 3000, 20), rng.uniform(0.05, 0.1, 20))
    order = np.argsort(np.concatenate([a.nu0, b.nu0]))
    u = _lines(np.concatenate([a.nu0, b.nu0])[order], np.concatenate([a.log10_s296, b.log10_s296])[order],
               np.concatenate([a.elow, b.elow])[order], np.concatenate([a.gamma_ref, b.gamma_ref])[order])
    args = (0.01, 900.0, 990.0, 0.05, 2400, 25.0)
    oa, ob, ou = (O.opacity_cell(x, *args) for x in (a, b, u))
    assert np.max(np.abs(ou - (oa + ob))) <= 1e-13 * np.max(ou)


def test_linear_in_strength():
    ll = _lines([1050.0, 1052.5], [-21.0, -22.0], [100.0, 200.0], [0.06, 0.08])
    l2 = _lines([1050.0, 1052.5], [-21.0 + np.log10(3.0), -22.0 + np.log10(3.0)],
                [100.0, 200.0], [0.06, 0.08])
    o1 = O.opacity_cell(ll, 0.1, 700.0, 1000.0, 0.05, 2000, 25.0)
    o3 = O.opacity_cell(l2, 0.1, 700.0, 1000.0, 0.05, 2000, 25.0)
    assert np.max(np.abs(o3 - 3 * o1)) <= 1e-6 * np.max(o3)   # float32 log10 S rounding


def test_translation_by_grid_steps():
    # Shifting a line by k grid steps shifts its profile by k points.  S and
    # the Doppler width depend on nu0, so compare S-normalised profiles in a
    # Lorentz-dominated regime (50 bar), where the width change is negligible.
    k = 7
    T = 1000.0
    ll = _lines([1030.0], [-20.0], [0.0], [0.07])
    sh = _lines([1030.0 + k * 0.25], [-20.0], [0.0], [0.07])
    o = O.opacity_cell(ll, 50.0, T, 1000.0, 0.25, 400, 25.0)
    s = O.opacity_cell(sh, 50.0, T, 1000.0, 0.25, 400, 25.0)
    S0 = O.line_strength(ll.log10_s296, ll.nu0, ll.elow, T)[0]
    S1 = O.line_strength(sh.log10_s296, sh.nu0, sh.elow, T)[0]
    assert np.max(np.abs(s[k:] / S1 - o[:-k] / S0)) <= 1e-8 * np.max(o / S0)


# ---- line-strength bound (Sec. 4 item 6)

def _random_lines(n, seed, lo=1500.0, hi=1510.0):
    rng = np.random.default_rng(seed)
    return _lines(np.sort(rng.uniform(lo, hi, n)), rng.uniform(-25, -19, n), rng.uniform(0, 4000, n),
                  rng.uniform(0.05, 0.1, n))


def test_threshold_zero_or_tiny_changes_nothing():
    ll = _random_lines(40, 31)
    args = (ll, 0.01, 900.0, 1499.0, 0.01, 1200, 2.0)
    ref = O.opacity_cell(*args)
    assert np.array_equal(O.opacity_cell(*args, rel_threshold=0.0), ref)
    assert np.array_equal(O.opacity_cell(*args, rel_threshold=1e-30), ref)


def test_threshold_above_one_leaves_nothing():
    ll = _random_lines(40, 32)
    assert np.all(O.opacity_cell(ll, 0.01, 900.0, 1499.0, 0.01, 1200, 2.0, rel_threshold=1.0001) == 0.0)


def test_threshold_near_one_keeps_only_the_strongest_line():
    # The strongest line at this T, found independently of the oracle's own
    # selection: one-line list through the same point-sampled sum.
    ll = _random_lines(40, 33)
    T = 1300.0
    S = [O.line_strength(ll.log10_s296[i], ll.nu0[i], ll.elow[i], T) for i in range(40)]
    i = int(np.argmax(S))
    one = _lines(ll.nu0[i:i + 1], ll.log10_s296[i:i + 1], ll.elow[i:i + 1], ll.gamma_ref[i:i + 1])
    got = O.opacity_cell(ll, 0.3, T, 1499.0, 0.01, 1200, 2.0, rel_threshold=0.999)
    exp = O.opacity_cell(one, 0.3, T, 1499.0, 0.01, 1200, 2.0)
    assert np.array_equal(got, exp)


def test_threshold_is_relative_to_each_temperature():
    # Scaling every strength by the same factor leaves the selection (and the
    # shape) unchanged: the bound is relative.
    ll = _random_lines(40, 34)
    scaled = _lines(ll.nu0, ll.log10_s296 + np.float32(2.0), ll.elow, ll.gamma_ref)
    a = O.opacity_cell(ll, 0.1, 800.0, 1499.0, 0.01, 1200, 2.0, rel_threshold=1e-3)
    b = O.opacity_cell(scaled, 0.1, 800.0, 1499.0, 0.01, 1200, 2.0, rel_threshold=1e-3)
    ok = a > 0
    assert np.array_equal(ok, b > 0)
    assert np.allclose(b[ok] / a[ok], 100.0, rtol=1e-12)


def test_strength_follows_the_population_difference():
    # Absorption minus stimulated emission: S(T) Q(T) is proportional to the
    # Boltzmann population difference of the lower and upper levels,
    # exp(-c2 E'' / T) - exp(-c2 (E'' + nu0) / T), with Q ~ T^1.5 and the
    # textbook c2 = 1.438776877 cm K.  Low nu0 makes the stimulated term large.
    c2 = 1.438776877
    for nu0, E in ((150.0, 0.0), (420.0, 900.0), (2500.0, 3000.0)):
        for T in (500.0, 1600.0, 3000.0):
            ratio = O.line_strength(0.0, nu0, E, T) / O.line_strength(0.0, nu0, E, 296.0)
            pop = lambda t: (np.exp(-c2 * E / t) - np.exp(-c2 * (E + nu0) / t)) / t ** 1.5
            assert abs(ratio / (pop(T) / pop(296.0)) - 1) < 1e-8


def _brute_force(lines, p, T, nu_start, dnu, n_nu, cutoff, rel_threshold=0.0):
    # The point-sampled sum written out: every line against every point.
    nu = nu_start + np.arange(n_nu) * dnu
    S = O.line_strength(lines.log10_s296, lines.nu0, lines.elow, T)
    floor = rel_threshold * S.max() if rel_threshold > 0 else 0.0
    out = np.zeros(n_nu)
    for j in range(n_nu):
        terms = []
        for i in range(len(lines.nu0)):
            d = nu[j] - lines.nu0[i]
            if abs(d) <= cutoff and S[i] >= floor:
                sig = O.doppler_sigma(lines.nu0[i], T, lines.mass_amu)
                gam = O.lorentz_gamma(lines.gamma_ref[i], p, T)
                terms.append(S[i] * V.voigt(d, sig, gam))
        out[j] = sum(sorted(terms))
    return out


def test_dense_list_against_every_line_at_every_point():
    # Lines inside the grid, beyond both ends and exactly one cutoff (plus or
    # minus one grid step) from grid points; binary-exact grid and offsets, a
    # sub-range starting inside the grid.
    rng = np.random.default_rng(12)
    dnu, cut, n = 0.25, 3.0, 160
    edge = 1000.0 + np.array([-cut - dnu, -cut, -cut + dnu, 17 * dnu - cut, 40 * dnu + cut,
                              (n - 1) * dnu + cut, (n - 1) * dnu + cut + dnu])
    nu0 = np.sort(np.concatenate([edge, rng.uniform(995.0, 1045.0, 45)]))
    ll = _lines(nu0, rng.uniform(-23, -19, nu0.size), rng.uniform(0, 3000, nu0.size),
                rng.uniform(0.05, 0.1, nu0.size))
    for p, T in ((1e-4, 800.0), (3.0, 2100.0)):
        exp = _brute_force(ll, p, T, 1000.0, dnu, n, cut)
        got = O.opacity_cell(ll, p, T, 1000.0, dnu, n, cut)
        assert np.max(np.abs(got - exp)) <= 1e-14 * np.max(exp)
        assert np.array_equal(got > 0, exp > 0)
        part = O.opacity_cell(ll, p, T, 1000.0, dnu, n, cut, j_lo=37, j_hi=121)
        assert np.array_equal(part, got[37:121])
        one = O.opacity_cell(ll, p, T, 1000.0, dnu, n, cut, j_lo=59, j_hi=60)
        assert np.array_equal(one, got[59:60])
        assert O.opacity_cell(ll, p, T, 1000.0, dnu, n, cut, j_lo=70, j_hi=70).size == 0


def test_threshold_at_exactly_one_keeps_the_strongest_line():
    # The bound keeps lines at or above rel_threshold x the strongest: at
    # exactly 1 the strongest line alone survives.
    ll = _random_lines(30, 35)
    T = 1250.0
    exp = _brute_force(ll, 0.2, T, 1499.0, 0.01, 1200, 2.0, rel_threshold=1.0)
    got = O.opacity_cell(ll, 0.2, T, 1499.0, 0.01, 1200, 2.0, rel_threshold=1.0)
    assert np.count_nonzero(got) > 0
    assert np.max(np.abs(got - exp)) <= 1e-14 * np.max(exp)


def test_cells_keep_lines_of_any_strength_by_default():
    # No bound unless asked: a line 1e-8 times weaker than its neighbour
    # still adds its own opacity.
    strong = _lines([1500.0], [-19.0], [300.0], [0.07])
    weak = _lines([1500.5], [-27.0], [300.0], [0.07])
    both = _lines([1500.0, 1500.5], [-19.0, -27.0], [300.0, 300.0], [0.07, 0.07])
    args = ([0.05], [1000.0], 1495.0, 0.01, 1000, 5.0)
    o_s, o_w, o_b = (O.opacity_cells([x], *args)[0, 0] for x in (strong, weak, both))
    assert np.max(np.abs(o_b - (o_s + o_w))) <= 1e-14 * np.max(o_b)
    assert np.max(np.abs(o_b - o_s)) > 0.5 * np.max(o_w)

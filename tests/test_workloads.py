"""The seeded synthetic inputs: deterministic, sorted, and with line strengths
that carry the lower-state population at 296 K (a line from an excited state
is weak at 296 K), so that hot layers are not opaque to every line."""
import numpy as np

import workloads as W


def test_line_lists_are_seeded_and_sorted():
    a, b = W.line_list(1, 5000), W.line_list(1, 5000)
    assert np.array_equal(a.nu0, b.nu0) and np.array_equal(a.log10_s296, b.log10_s296)
    assert np.all(np.diff(a.nu0) >= 0)
    assert not np.array_equal(W.line_list(2, 5000).nu0, a.nu0)


def test_strengths_carry_the_296K_population():
    ll = W.line_list(0, 200_000)
    c2 = 1.438776877
    # log10 S_int = log10 S + c2 E'' / (296 ln 10) is uniform on [-25, -19]
    s_int = ll.log10_s296.astype(np.float64) + c2 * ll.elow.astype(np.float64) / (296.0 * np.log(10.0))
    assert s_int.min() >= -25.0 - 1e-4 and s_int.max() <= -19.0 + 1e-4
    assert abs(np.mean(s_int) + 22.0) < 0.02
    # and is independent of E'' (the population factor is the only link)
    assert abs(np.corrcoef(s_int, ll.elow)[0, 1]) < 0.01
    # corr(log10 S, E'') = -sd_pop / sqrt(sd_pop^2 + sd_int^2) with sd_pop =
    # (c2 5000 / (296 ln 10)) / sqrt(12) = 3.05 and sd_int = 6 / sqrt(12) = 1.73
    assert abs(np.corrcoef(ll.log10_s296, ll.elow)[0, 1] + 0.870) < 0.01


def test_grid_axes_and_split():
    ax = W.grid_axes()
    assert len(ax.p_bar) == 100 and len(ax.t_K) == 20 and ax.n_nu == 100_000
    assert np.isclose(ax.p_bar[0], 1e-8) and np.isclose(ax.p_bar[-1], 100.0)
    assert W.split_lines(5_000_000, 3) == [1_666_667, 1_666_667, 1_666_666]


def test_line_list_ranges_and_masses():
    for s, mass in enumerate((18.0, 28.0, 44.0, 16.0)):
        ll = W.line_list(s, 20_000)
        assert ll.mass_amu == mass and ll.nu0.dtype == np.float64
        assert 1000.0 <= ll.nu0.min() and ll.nu0.max() <= 3000.0
        assert 0.0 <= ll.elow.min() and ll.elow.max() <= 5000.0
        assert 0.05 <= ll.gamma_ref.min() and ll.gamma_ref.max() <= 0.1
        # uniform centres: about a tenth of the lines in each tenth of the range
        counts = np.histogram(ll.nu0, bins=10, range=(1000.0, 3000.0))[0]
        assert np.all(np.abs(counts - 2000) < 6 * np.sqrt(2000))


def test_grid_axes_recipe():
    ax = W.grid_axes()
    assert np.allclose(np.diff(np.log10(ax.p_bar)), 10.0 / 99.0, rtol=1e-12)   # 100 levels over 10 decades
    assert np.allclose(ax.t_K, np.linspace(500.0, 3000.0, 20))
    assert ax.nu_start == 1000.0 and ax.dnu == 0.02 and ax.cutoff == 25.0
    nu = W.nu_axis(ax.nu_start, ax.dnu, ax.n_nu)
    assert abs(nu[-1] - 2999.98) < 1e-9


def test_proposals_fill_the_prior_box():
    th = W.proposals(2048, generation=5)
    assert th.shape == (2048, 9) and th.dtype == np.float32
    lo, hi = W.THETA_LO.astype(np.float32), W.THETA_HI.astype(np.float32)
    assert np.all(th >= lo) and np.all(th <= hi)
    u = (th - lo) / (hi - lo)
    assert np.all(np.abs(u.mean(axis=0) - 0.5) < 0.03)
    assert np.array_equal(W.proposals(16, generation=5), W.proposals(16, generation=5))
    assert not np.array_equal(W.proposals(16, generation=5), W.proposals(16, generation=6))
    # log10 kappa [-3, 0], log10 gamma1,2 [-1.5, 1], alpha [0, 1], beta [0.7, 1.3], a_s [-3, 3]
    assert np.array_equal(W.THETA_LO, [-3.0, -1.5, -1.5, 0.0, 0.7, -3.0, -3.0, -3.0, -3.0])
    assert np.array_equal(W.THETA_HI, [0.0, 1.0, 1.0, 1.0, 1.3, 3.0, 3.0, 3.0, 3.0])


def test_gaussian_filters_recipe():
    nu = W.nu_axis(1000.0, 0.5, 4000)
    w = W.gaussian_filters(nu, 10, 1100.0, 2900.0, 20.0, 200.0)
    assert w.shape == (10, 4000) and np.all(w >= 0) and np.all(w <= 1)
    for b in range(10):
        on = nu[w[b] > 0]
        cen = nu[np.argmax(w[b])]
        assert 1100.0 - 0.5 <= cen <= 2900.0 + 0.5
        # truncated at 3 sigma: the support spans 6 sigma = 6 FWHM / 2.3548
        fwhm = (on[-1] - on[0]) / 6.0 * 2.0 * np.sqrt(2.0 * np.log(2.0))
        assert 20.0 - 1.0 <= fwhm <= 200.0 + 1.0


def test_transit_instances_recipe():
    inst = W.instances(1024, 100_000)
    assert np.all((inst.n_levels >= 40) & (inst.n_levels <= 150))
    span = inst.nu_hi - inst.nu_lo
    assert np.all((span >= 10_000) & (span <= 100_000))
    assert np.all(inst.nu_lo >= 0) and np.all(inst.nu_hi <= 100_000)
    assert np.all((inst.r_planet >= np.float32(1.0 * W.R_JUP_CM)) & (inst.r_planet <= np.float32(1.4 * W.R_JUP_CM)))
    assert np.all((inst.r_star >= np.float32(0.7 * W.R_SUN_CM)) & (inst.r_star <= np.float32(1.2 * W.R_SUN_CM)))
    assert inst.offsets[-1] == span.sum() and inst.offsets[0] == 0


def test_opacity_field_recipe():
    # seeded random numbers only: a grid [S][L][M][n_nu] of cross sections in
    # [1e-30, 1e-16] cm^2, reproducible by seed, varying over every axis
    ax = W.grid_axes(n_layers=20, n_temps=5, n_nu=3000)
    f = W.opacity_field(4, ax.p_bar, ax.t_K, ax.n_nu, seed=3600)
    assert f.shape == (4, 20, 5, 3000) and np.all(np.isfinite(f))
    assert f.min() >= 1e-30 and f.max() <= 1e-16
    assert np.array_equal(f, W.opacity_field(4, ax.p_bar, ax.t_K, ax.n_nu, seed=3600))
    assert not np.array_equal(f, W.opacity_field(4, ax.p_bar, ax.t_K, ax.n_nu, seed=3601))
    lf = np.log10(f)
    for axis in range(4):
        assert np.ptp(lf.mean(axis=tuple(a for a in range(4) if a != axis))) > 0.0
    assert np.ptp(lf) > 3.0                      # several decades of dynamic range

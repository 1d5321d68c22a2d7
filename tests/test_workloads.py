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

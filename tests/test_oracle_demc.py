"""Pins of the oracle sampler: from an overdispersed start it recovers a
correlated Gaussian's mean, variances and 68.27% credible-region content
within the App. C standard errors, with and without a (deliberately wrong)
surrogate screen; at stationarity its acceptance rates equal those of its
proposals computed by plain Monte Carlo from independent draws of the
target."""
import numpy as np
import pytest
from scipy.stats import chi2

from oracle import demc as D
from demc_target import target


def _check(hist, mu, cov, burn):
    s = hist[burn:]
    n, C, d = s.shape
    flat = s.reshape(-1, d)
    e = D.ess(s)
    sd = np.sqrt(np.diag(cov))
    z = np.abs(flat.mean(0) - mu) / (sd / np.sqrt(e))
    assert np.all(z < 4.5), z
    var_ratio = flat.var(0) / sd ** 2
    assert np.all(np.abs(var_ratio - 1) < 4.5 * np.sqrt(2.0 / e)), var_ratio
    inv = np.linalg.inv(cov)
    m2 = np.einsum("ij,jk,ik->i", flat - mu, inv, flat - mu)
    c = float(np.mean(m2 <= chi2.ppf(0.6827, d)))
    assert abs(c - 0.6827) < 4.5 * D.credible_content_se(0.6827, e), c
    return e


@pytest.mark.parametrize("screened,beta,margin", [(False, 1.0, 0.0), (True, 1.0, 0.0), (True, 0.5, 2.0)])
def test_recovers_gaussian(screened, beta, margin):
    mu, cov, lo, hi = target()
    inv = np.linalg.inv(cov)
    L = lambda v: -0.5 * (v - mu) @ inv @ (v - mu)
    # a surrogate with the wrong scale: delayed acceptance keeps the exact target
    Ls = (lambda v: -0.5 * 0.7 * (v - mu) @ inv @ (v - mu)) if screened else None
    rng = np.random.default_rng(6000)
    # overdispersed start: a sampler that does not move fails the check
    x0 = mu + rng.normal(size=(16, 9)) * np.sqrt(np.diag(cov)) * 3.0
    hist, acc = D.run(L, x0, lo, hi, 3000, rng, surrogate=Ls, beta=beta, margin=margin)
    e = _check(hist, mu, cov, burn=500)
    assert e > 300
    assert np.all(D.gelman_rubin(hist[500:]) < 1.05)


def test_speis_of_white_noise_and_ar1():
    rng = np.random.default_rng(1)
    assert abs(D.speis(rng.normal(size=20000)) - 1.0) < 0.05
    phi = 0.9
    x = np.zeros(200000)
    for t in range(1, x.size):
        x[t] = phi * x[t - 1] + rng.normal()
    # integrated autocorrelation time of AR(1): (1 + phi) / (1 - phi) = 19
    assert abs(D.speis(x) - 19.0) < 2.0


# ---- DEMCzs (Sec. 4) and the Gelman-Rubin statistic (Sec. 5)

def test_demczs_recovers_gaussian_with_three_chains():
    mu, cov, lo, hi = target()
    inv = np.linalg.inv(cov)
    L = lambda v: -0.5 * (v - mu) @ inv @ (v - mu)
    rng = np.random.default_rng(6010)
    sd = np.sqrt(np.diag(cov))
    z0 = mu + rng.normal(size=(90, 9)) * sd * 2.0
    x0 = mu + rng.normal(size=(3, 9)) * sd * 3.0
    hist, acc, Z = D.run_zs(L, x0, z0, lo, hi, 12000, rng, thin=10)
    e = _check(hist, mu, cov, burn=2000)
    assert e > 150
    assert len(Z) == 90 + 3 * (12000 // 10)


def test_demczs_snooker_only_keeps_the_target():
    # all moves snooker: the (|y - z|/|x - z|)^(d-1) factor is what keeps the
    # target; without it the sampler would not pass _check
    mu, cov, lo, hi = target()
    inv = np.linalg.inv(cov)
    L = lambda v: -0.5 * (v - mu) @ inv @ (v - mu)
    rng = np.random.default_rng(6011)
    sd = np.sqrt(np.diag(cov))
    z0 = mu + rng.normal(size=(90, 9)) * sd
    x0 = mu + rng.normal(size=(4, 9)) * sd * 3.0
    hist, acc, _ = D.run_zs(L, x0, z0, lo, hi, 12000, rng, thin=10, p_snooker=1.0)
    _check(hist, mu, cov, burn=2000)


def test_gelman_rubin_limits():
    rng = np.random.default_rng(12)
    same = rng.normal(size=(4000, 4, 3))
    assert np.all(np.abs(D.gelman_rubin(same) - 1.0) < 0.01)
    apart = same + np.array([0.0, 0.0, 5.0, 5.0])[None, :, None]
    assert np.all(D.gelman_rubin(apart) > 2.0)
    # closed form for two chains of constant-variance noise with means +-a:
    # W = 1, B = n * 2 a^2, V = (n - 1)/n + 2 a^2, R = sqrt(V)
    # and for within-chain variance s^2 = 4: V = (n - 1)/n s^2 + 2 a^2, R = sqrt(V / s^2)
    n, a = 4000, 0.5
    two = np.stack([rng.normal(size=n), rng.normal(size=n)], axis=1)[:, :, None]
    two = (two - two.mean(0)) / two.std(0, ddof=1)
    assert abs(D.gelman_rubin(two + np.array([a, -a])[None, :, None])[0] - np.sqrt((n - 1) / n + 2 * a * a)) < 1e-12
    wide = 2.0 * two + np.array([a, -a])[None, :, None]
    assert abs(D.gelman_rubin(wide)[0] - np.sqrt(((n - 1) / n * 4.0 + 2 * a * a) / 4.0)) < 1e-12


# ---- acceptance rates at stationarity
#
# With every chain (and archive state) distributed as the target pi and
# mutually independent, one proposal is accepted with probability
# E[min(1, pi(y) q(y -> x) / (pi(x) q(x -> y)))], an expectation over
# independent draws of pi that plain Monte Carlo estimates without the
# sampler.  A wrong jump scale, direction or Jacobian changes that number.

def _gauss():
    mu, cov, lo, hi = target()
    inv = np.linalg.inv(cov)
    Lc = np.linalg.cholesky(cov)
    L = lambda v: -0.5 * (v - mu) @ inv @ (v - mu)
    draw = lambda rng, n: mu + rng.normal(size=(n, 9)) @ Lc.T
    Lv = lambda v: -0.5 * np.einsum("ij,jk,ik->i", v - mu, inv, v - mu)
    return mu, cov, lo, hi, L, draw, Lv


def test_de_acceptance_rate_matches_its_proposal():
    # parallel DE move y = x + gamma (x_r1 - x_r2), gamma = 2.38 / sqrt(2 d)
    mu, cov, lo, hi, L, draw, Lv = _gauss()
    rng = np.random.default_rng(21)
    n_gen, C = 1500, 16
    x0 = draw(rng, C)
    _, acc = D.run(L, x0, lo, hi, n_gen, rng, jump_every=0, eps=1e-9)
    rate = acc / (n_gen * C)
    m = np.random.default_rng(22)
    x, a, b = draw(m, 400000), draw(m, 400000), draw(m, 400000)
    g = 2.38 / np.sqrt(18.0)
    mc = np.mean(np.minimum(1.0, np.exp(Lv(x + g * (a - b)) - Lv(x))))
    assert abs(rate - mc) < 0.015, (rate, mc)


def test_snooker_acceptance_rate_matches_its_proposal():
    # snooker move about z with z1, z2 from a frozen archive of target draws:
    # y = x + g_s ((z1 - z2) . e) e, e = (x - z) / |x - z|, g_s ~ U[1.2, 2.2],
    # accepted with the extra factor (|y - z| / |x - z|)^(d - 1)
    mu, cov, lo, hi, L, draw, Lv = _gauss()
    rng = np.random.default_rng(23)
    z0 = draw(rng, 3000)
    C, n_steps = 8, 2500
    _, acc, Z = D.run_zs(L, draw(rng, C), z0, lo, hi, n_steps, rng, capacity=len(z0), p_snooker=1.0)
    assert len(Z) == len(z0)
    rate = acc / (n_steps * C)
    m = np.random.default_rng(24)
    n = 400000
    x, z, z1, z2 = (draw(m, n) for _ in range(4))
    e = x - z
    nn = np.sum(e * e, axis=1)
    gs = 1.2 + m.uniform(size=n)
    y = x + (gs * np.sum((z1 - z2) * e, axis=1) / nn)[:, None] * e
    logq = 8 * 0.5 * (np.log(np.sum((y - z) ** 2, axis=1)) - np.log(nn))
    mc = np.mean(np.minimum(1.0, np.exp(Lv(y) - Lv(x) + logq)))
    assert abs(rate - mc) < 0.015, (rate, mc)


def test_de_acceptance_rate_with_unit_jumps_every_tenth_generation():
    # With jump_every = 10 one generation in ten uses gamma = 1: the rate is
    # the 9:1 mixture of the two proposals' stationary acceptance.
    mu, cov, lo, hi, L, draw, Lv = _gauss()
    rng = np.random.default_rng(25)
    n_gen, C = 3000, 16
    _, acc = D.run(L, draw(rng, C), lo, hi, n_gen, rng, jump_every=10, eps=1e-9)
    rate = acc / (n_gen * C)
    m = np.random.default_rng(26)
    x, a, b = draw(m, 400000), draw(m, 400000), draw(m, 400000)
    mc = [np.mean(np.minimum(1.0, np.exp(Lv(x + g * (a - b)) - Lv(x)))) for g in (2.38 / np.sqrt(18.0), 1.0)]
    assert abs(rate - (0.9 * mc[0] + 0.1 * mc[1])) < 0.008, (rate, mc)


def test_delayed_acceptance_snooker_rate_matches_its_two_stages():
    # Two-stage acceptance with a surrogate (Christen & Fox 2005) of a
    # snooker move: the move is accepted with probability
    #   min(a1(x -> y), exp(L_y - L_x) q a1(y -> x)),
    #   a1(x -> y) = min(1, exp(beta (ls_y - ls_x) + margin) q),
    #   a1(y -> x) = min(1, exp(beta (ls_x - ls_y) + margin) / q),
    # q = (|y - z| / |x - z|)^(d - 1), here with a surrogate of the wrong
    # scale and a shifted centre.
    mu, cov, lo, hi, L, draw, Lv = _gauss()
    inv = np.linalg.inv(cov)
    off = 0.2 * np.sqrt(np.diag(cov))
    Ls = lambda v: -0.5 * 0.6 * (v - mu - off) @ inv @ (v - mu - off)
    Lsv = lambda v: -0.5 * 0.6 * np.einsum("ij,jk,ik->i", v - mu - off, inv, v - mu - off)
    beta, margin = 0.5, 0.7
    rng = np.random.default_rng(27)
    z0 = draw(rng, 3000)
    C, n_steps = 8, 2500
    _, acc, _ = D.run_zs(L, draw(rng, C), z0, lo, hi, n_steps, rng, capacity=len(z0), p_snooker=1.0,
                         surrogate=Ls, beta=beta, margin=margin)
    rate = acc / (n_steps * C)
    m = np.random.default_rng(28)
    n = 400000
    x, z, z1, z2 = (draw(m, n) for _ in range(4))
    e = x - z
    nn = np.sum(e * e, axis=1)
    y = x + ((1.2 + m.uniform(size=n)) * np.sum((z1 - z2) * e, axis=1) / nn)[:, None] * e
    logq = 8 * 0.5 * (np.log(np.sum((y - z) ** 2, axis=1)) - np.log(nn))
    dls = Lsv(y) - Lsv(x)
    a1xy = np.minimum(1.0, np.exp(beta * dls + margin + logq))
    a1yx = np.minimum(1.0, np.exp(-beta * dls + margin - logq))
    mc = np.mean(np.minimum(a1xy, np.exp(Lv(y) - Lv(x) + logq) * a1yx))
    assert abs(rate - mc) < 0.015, (rate, mc)


@pytest.mark.parametrize("p_snooker", [0.1, 1.0])
def test_screened_demczs_recovers_gaussian(p_snooker):
    # delayed acceptance with a wrong-scale surrogate keeps the exact target
    mu, cov, lo, hi = target()
    inv = np.linalg.inv(cov)
    L = lambda v: -0.5 * (v - mu) @ inv @ (v - mu)
    Ls = lambda v: -0.5 * 0.7 * (v - mu) @ inv @ (v - mu)
    rng = np.random.default_rng(6020)
    sd = np.sqrt(np.diag(cov))
    z0 = mu + rng.normal(size=(90, 9)) * sd * 2.0
    x0 = mu + rng.normal(size=(4, 9)) * sd * 3.0
    hist, _, _ = D.run_zs(L, x0, z0, lo, hi, 10000, rng, thin=10, p_snooker=p_snooker, surrogate=Ls,
                          beta=0.5, margin=1.0)
    _check(hist, mu, cov, burn=2000)


@pytest.mark.parametrize("d", [2, 3])
def test_snooker_keeps_a_low_dimensional_target(d):
    # In few dimensions the (|y - z| / |x - z|)^(d - 1) factor decides the
    # radial law: snooker moves about archive draws of N(0, I) must keep
    # E |x|^2 = d (without the factor, or with d - 2, it falls by ~30%).
    L = lambda v: -0.5 * v @ v
    rng = np.random.default_rng(40 + d)
    z0 = rng.normal(size=(4000, d))
    hist, _, _ = D.run_zs(L, rng.normal(size=(8, d)), z0, np.full(d, -12.0), np.full(d, 12.0), 6000, rng,
                          capacity=len(z0), p_snooker=1.0)
    s = hist[500:].reshape(-1, d)
    assert abs(np.mean(np.sum(s * s, axis=1)) / d - 1) < 0.05


def test_archive_grows_by_the_population_every_thin_steps():
    # Every `thin` steps the chains' current states are appended to Z, until
    # Z holds `capacity` states (by default, room for every append).
    mu, cov, lo, hi, L, draw, Lv = _gauss()
    rng = np.random.default_rng(29)
    z0 = draw(rng, 50)
    C, thin = 3, 7
    hist, _, Z = D.run_zs(L, draw(rng, C), z0, lo, hi, 40, rng, thin=thin, capacity=len(z0) + 4 * C)
    assert len(Z) == len(z0) + 4 * C
    assert np.array_equal(Z[:len(z0)], z0)
    for k in range(4):
        assert np.array_equal(Z[len(z0) + k * C:len(z0) + (k + 1) * C], hist[(k + 1) * thin])
    _, _, Z = D.run_zs(L, draw(rng, 4), z0, lo, hi, 70, rng, thin=thin)
    assert len(Z) == len(z0) + 4 * (70 // thin)


def test_demczs_acceptance_rate_with_unit_jumps():
    # Parallel moves from a frozen archive of target draws, gamma = 1 every
    # tenth step: the 9:1 mixture of the two proposals' acceptance.
    mu, cov, lo, hi, L, draw, Lv = _gauss()
    rng = np.random.default_rng(31)
    z0 = draw(rng, 3000)
    C, n_steps = 8, 4000
    _, acc, _ = D.run_zs(L, draw(rng, C), z0, lo, hi, n_steps, rng, capacity=len(z0), p_snooker=0.0,
                         jump_every=10, eps=1e-9)
    rate = acc / (n_steps * C)
    m = np.random.default_rng(32)
    x, a, b = draw(m, 400000), draw(m, 400000), draw(m, 400000)
    mc = [np.mean(np.minimum(1.0, np.exp(Lv(x + g * (a - b)) - Lv(x)))) for g in (2.38 / np.sqrt(18.0), 1.0)]
    assert abs(rate - (0.9 * mc[0] + 0.1 * mc[1])) < 0.008, (rate, mc)


def test_credible_content_error_is_the_binomial_spread():
    # For N independent samples the estimated content of a region of
    # probability C scatters over repeated experiments with standard
    # deviation sqrt(C (1 - C) / N), which App. C's posterior standard
    # deviation sqrt(C (1 - C) / (N + 3)) matches to O(1/N): replicate
    # experiments by plain sampling.
    rng = np.random.default_rng(30)
    N, reps, C = 400, 4000, 0.6827
    inside = rng.uniform(size=(reps, N)) < C
    spread = inside.mean(axis=1).std(ddof=1)
    assert abs(spread / D.credible_content_se(C, N) - 1) < 0.05


def test_rejected_proposals_leave_the_chains_and_the_count_alone():
    # A likelihood that is -inf everywhere except at the starting states:
    # nothing is accepted and every chain stays where it started.
    mu, cov, lo, hi, _, draw, _ = _gauss()
    rng = np.random.default_rng(33)
    x0 = draw(rng, 6)
    L = lambda v: 0.0 if any(np.array_equal(v, s) for s in x0) else -np.inf
    hist, acc = D.run(L, x0, lo, hi, 30, rng)
    assert acc == 0 and np.all(hist == x0[None])
    hist, acc, _ = D.run_zs(L, x0, draw(rng, 40), lo, hi, 30, rng)
    assert acc == 0 and np.all(hist == x0[None])


def test_credible_content_error_reproduces_the_papers_retrieval_table():
    # Sec. 6.3 prints, for thirteen retrievals, the ESS and the uncertainty of
    # the 68.27%, 95.45% and 99.73% regions' content to 0.01%: App. C's
    # s_C = sqrt(C (1 - C) / (ESS + 3)) reproduces every entry to its last
    # digit (without the 3, the low-ESS rows are off by up to 0.08%).
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "retrieval_posterior_accuracy.json")) as fh:
        table = json.load(fh)
    for name, _, ess, *printed in table["rows"]:
        for C, pct in zip((0.6827, 0.9545, 0.9973), printed):
            assert abs(100.0 * D.credible_content_se(C, ess) - pct) <= 0.005 + 1e-9, (name, C)


def test_credible_content_error_meets_the_sizing_examples():
    # App. C (and Sec. 5) size runs by ESS ~ C (1 - C) / s_C^2: 68.27% to 2%
    # needs ~500, 95.45% to 0.5% ~1700, 99.73% to 0.1% ~2700 samples.
    for C, s, n in ((0.6827, 0.02, 500), (0.9545, 0.005, 1700), (0.9973, 0.001, 2700)):
        assert abs(D.credible_content_se(C, n) / s - 1) < 0.05


def test_speis_and_ess_of_a_square_wave_in_closed_form():
    # A chain of +1, +1, +1, +1, -1, -1, -1, -1, ... of length n = 8m has mean
    # 0 and variance 1; counting sign changes, the lag-1 sum of products is
    # n/2 + 1 (rho_1 = 1/2 + 1/n) and the lag-2 sum is 2 (rho_2 = 2/n, below
    # the 0.01 threshold), so SPEIS = 1 + 2 rho_1 = 2 + 2/n exactly.
    for n in (800, 8000):
        c = np.tile([1.0, 1.0, 1.0, 1.0, -1.0, -1.0, -1.0, -1.0], n // 8)
        assert abs(D.speis(c) - (2.0 + 2.0 / n)) < 1e-12
        chains = np.stack([c, -c, c], axis=1)[:, :, None]          # [n][3 chains][1 parameter]
        assert abs(D.ess(chains) - n * 3 / (2.0 + 2.0 / n)) < 1e-9

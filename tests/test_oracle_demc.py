"""Pins of the oracle sampler: it recovers a correlated Gaussian's mean,
variances and 68.27% credible-region content within the App. C standard
errors, with and without a (deliberately wrong) surrogate screen."""
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
    x0 = mu + rng.normal(size=(16, 9)) * np.sqrt(np.diag(cov))
    hist, acc = D.run(L, x0, lo, hi, 3000, rng, surrogate=Ls, beta=beta, margin=margin)
    e = _check(hist, mu, cov, burn=500)
    assert e > 300


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
    x0 = mu + rng.normal(size=(3, 9)) * sd
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
    x0 = mu + rng.normal(size=(4, 9)) * sd
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
    n, a = 4000, 0.5
    two = np.stack([rng.normal(size=n), rng.normal(size=n)], axis=1)[:, :, None]
    two = (two - two.mean(0)) / two.std(0, ddof=1) + np.array([a, -a])[None, :, None]
    assert abs(D.gelman_rubin(two)[0] - np.sqrt((n - 1) / n + 2 * a * a)) < 1e-12

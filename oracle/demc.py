"""Differential-evolution MCMC and its convergence statistics, in FP64 (test
infrastructure).

Sampler (Sec. 3-4: the paper's DEMC of ter Braak 2006): chains split into two
halves; a half-step moves every chain i of one half to
y_i = x_i + gamma (x_r1 - x_r2) + e_i with r1 != r2 drawn from the other half,
e_i ~ N(0, (eps * width)^2), gamma = 2.38/sqrt(2 d) (1 on every jump_every-th
generation), uniform prior on a box.  With a surrogate log-likelihood the
move is delayed acceptance (two-stage Metropolis-Hastings, Christen & Fox
2005): stage 1 with probability a1(x -> y) = min(1, exp(beta (ls_y - ls_x) +
margin)), stage 2 with min(1, exp(L_y - L_x) a1(y -> x) / a1(x -> y)); for
beta = 1, margin = 0 the stage-2 ratio is exp((L_y - L_x) - (ls_y - ls_x)).  Random numbers come from numpy, so
parity with the GPU sampler is distributional.

DEMCzs (Sec. 4, the snooker DE-MC of ter Braak & Vrugt 2008, cited there as
converging with as few as three chains): every chain proposes from an archive
Z of past states instead of from the other chains, so all chains move in one
step.  With probability p_snooker the move is a snooker update: z, z1, z2
drawn from Z, the proposal x + g_s ((z1 - z2) . e) e with e the unit vector
from z to x and g_s ~ U[1.2, 2.2], accepted with the extra factor
(|y - z| / |x - z|)^(d - 1); otherwise a parallel-direction update
x + gamma (z1 - z2) + noise.  Every `thin` steps all chains' states are
appended to Z (until it holds `capacity` states).  With a surrogate, the
delayed acceptance carries the proposal factor q in both stages:
a1(x -> y) = min(1, exp(beta (ls_y - ls_x) + margin) q) and the stage-2
ratio exp(L_y - L_x) q a1(y -> x) / a1(x -> y).

Statistics (Sec. 5 "Bayesian samplers and convergence", App. C):
* SPEIS by summing the autocorrelation from lag 0 until it first falls below a
  small positive threshold: SPEIS = 1 + 2 sum_{k>=1} rho_k; ESS = N / SPEIS;
* standard error of a mean, s = sigma / sqrt(ESS) (App. C, Eq. C3 reading);
* accuracy of a credible region's probability content,
  s_C = sqrt(C (1 - C) / (ESS + 3)) (App. C: the standard deviation of the
  Beta posterior of a binomial proportion under a flat prior, with the ESS
  as the number of trials; Sec. 5 drops the 3 when sizing a run);
* the Gelman-Rubin statistic (Sec. 5, GR 1992) of m chains of length n:
  W = mean within-chain variance, B = n x variance of the chain means,
  V = (n - 1)/n W + B/n, R = sqrt(V / W).
"""
import math

import numpy as np


def run(loglike, x0, lo, hi, n_gen, rng, gamma=None, jump_every=10, eps=1e-4, surrogate=None, beta=1.0,
        margin=0.0):
    """Returns the chain history [n_gen+1][C][d] and acceptance counts."""
    x = np.array(x0, np.float64)
    C, d = x.shape
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    g0 = 2.38 / np.sqrt(2.0 * d) if gamma is None else gamma
    L = np.array([loglike(v) for v in x])
    Ls = np.array([surrogate(v) for v in x]) if surrogate else np.zeros(C)
    hist = [x.copy()]
    acc = 0
    halves = (np.arange(0, C // 2), np.arange(C // 2, C))
    for gen in range(n_gen):
        gm = 1.0 if (jump_every and gen % jump_every == jump_every - 1) else g0
        for h in (0, 1):
            own, other = halves[h], halves[1 - h]
            for i in own:
                r1, r2 = rng.choice(other, 2, replace=False)
                y = x[i] + gm * (x[r1] - x[r2]) + eps * (hi - lo) * rng.normal(size=d)
                if np.any(y < lo) or np.any(y > hi):
                    continue
                ly_s = surrogate(y) if surrogate else 0.0
                dl = ly_s - Ls[i]
                if surrogate and np.log(rng.uniform()) >= min(0.0, beta * dl + margin):
                    continue
                ly = loglike(y)
                r = ly - L[i]
                if surrogate:
                    r += min(0.0, -beta * dl + margin) - min(0.0, beta * dl + margin)
                if r >= 0 or np.log(rng.uniform()) < r:
                    x[i], L[i], Ls[i] = y, ly, ly_s
                    acc += 1
        hist.append(x.copy())
    return np.array(hist), acc


def speis(chain, threshold=0.01):
    """Steps per effectively independent sample of a 1-D chain.  A chain of
    zero variance (it never moved) has no autocorrelation to sum; it gets 1,
    the same convention as the GPU statistics kernel, so a stuck chain must be
    caught by its acceptance count, not by its ESS."""
    c = np.asarray(chain, np.float64) - np.mean(chain)
    n = c.size
    var = np.dot(c, c) / n
    if var == 0:
        return 1.0
    s = 1.0
    for k in range(1, n // 2):
        rho = np.dot(c[:-k], c[k:]) / (n * var)
        if rho < threshold:
            break
        s += 2.0 * rho
    return s


def ess(samples_per_chain):
    """Effective sample size of samples [n][C][d]: total samples divided by
    the largest SPEIS over parameters (mean over chains)."""
    n, C, d = samples_per_chain.shape
    sp = max(np.mean([speis(samples_per_chain[:, c, q]) for c in range(C)]) for q in range(d))
    return n * C / sp


def credible_content_se(c_hat, ess_value):
    return np.sqrt(c_hat * (1.0 - c_hat) / (ess_value + 3.0))


def run_zs(loglike, x0, z0, lo, hi, n_steps, rng, thin=10, capacity=None, p_snooker=0.1, gamma=None,
           jump_every=10, eps=1e-4, surrogate=None, beta=1.0, margin=0.0):
    """DEMCzs; returns the chain history [n_steps+1][C][d], acceptance count
    and the final archive."""
    x = np.array(x0, np.float64)
    C, d = x.shape
    Z = [np.asarray(v, np.float64) for v in z0]
    cap = capacity if capacity is not None else len(Z) + n_steps * C
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    g0 = 2.38 / np.sqrt(2.0 * d) if gamma is None else gamma
    L = np.array([loglike(v) for v in x])
    Ls = np.array([surrogate(v) for v in x]) if surrogate else np.zeros(C)
    hist = [x.copy()]
    acc = 0
    for step in range(n_steps):
        gm = 1.0 if (jump_every and step % jump_every == jump_every - 1) else g0
        m = len(Z)
        new = x.copy()
        for i in range(C):
            a, b = rng.choice(m, 2, replace=False)
            logq = 0.0
            if rng.uniform() < p_snooker:
                c = rng.integers(m)
                dirv = x[i] - Z[c]
                nn = float(dirv @ dirv)
                if nn == 0.0:
                    continue
                gs = 1.2 + rng.uniform()
                y = x[i] + gs * (float((Z[a] - Z[b]) @ dirv) / nn) * dirv
                logq = (d - 1) * (0.5 * math.log(float((y - Z[c]) @ (y - Z[c]))) - 0.5 * math.log(nn))
            else:
                y = x[i] + gm * (Z[a] - Z[b]) + eps * (hi - lo) * rng.normal(size=d)
            if np.any(y < lo) or np.any(y > hi):
                continue
            ly_s = surrogate(y) if surrogate else 0.0
            dl = ly_s - Ls[i]
            if surrogate and np.log(rng.uniform()) >= min(0.0, beta * dl + margin + logq):
                continue
            ly = loglike(y)
            r = ly - L[i] + logq
            if surrogate:
                r += min(0.0, -beta * dl + margin - logq) - min(0.0, beta * dl + margin + logq)
            if r >= 0 or np.log(rng.uniform()) < r:
                new[i], L[i], Ls[i] = y, ly, ly_s
                acc += 1
        x = new
        hist.append(x.copy())
        if (step + 1) % thin == 0 and len(Z) + C <= cap:
            Z.extend(v.copy() for v in x)
    return np.array(hist), acc, np.array(Z)


def gelman_rubin(samples):
    """R for each parameter of samples [n][m][d] (m chains of length n)."""
    s = np.asarray(samples, np.float64)
    n = s.shape[0]
    means = s.mean(axis=0)                       # [m][d]
    W = s.var(axis=0, ddof=1).mean(axis=0)       # [d]
    B = n * means.var(axis=0, ddof=1)            # [d]
    V = (n - 1) / n * W + B / n
    return np.sqrt(V / W)

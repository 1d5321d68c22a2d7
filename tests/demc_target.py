"""A correlated 9-D Gaussian target shared by the sampler tests (test data:
mean, covariance and prior box; no sampler arithmetic)."""
import numpy as np

D = 9


def target(seed=6100):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(D, D))
    cov = A @ A.T / D + 0.05 * np.eye(D)
    sd = np.sqrt(np.diag(cov))
    cov = cov / np.outer(sd, sd) * np.outer(np.linspace(0.2, 1.0, D), np.linspace(0.2, 1.0, D))
    mu = rng.uniform(-1, 1, D)
    lo, hi = mu - 8.0, mu + 8.0
    return mu, cov, lo, hi

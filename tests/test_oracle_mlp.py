"""Pins of the oracle's surrogate network: GELU limits, central finite
differences of the loss gradient, BF16 rounding and one Adam step."""
import numpy as np

from oracle import mlp as N

WIDTHS = [9, 16, 16, 16, 10]


def _params(seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.3, N.n_params(WIDTHS))


def test_gelu_limits_and_derivative():
    assert N.gelu(0.0) == 0.0
    assert abs(N.gelu(10.0) - 10.0) < 1e-12 and abs(N.gelu(-10.0)) < 1e-12
    assert abs(N.gelu(1.0) - 0.8413447460685429) < 1e-15      # 1 * Phi(1)
    x = np.linspace(-4, 4, 81)
    h = 1e-6
    fd = (N.gelu(x + h) - N.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - N.gelu_grad(x))) < 1e-9


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = _params()
    x = rng.uniform(-1, 1, (7, 9))
    t = rng.normal(0, 1, (7, 10))
    _, g = N.loss_and_grad(p, WIDTHS, x, t)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (N.loss_and_grad(pp, WIDTHS, x, t)[0] - N.loss_and_grad(pm, WIDTHS, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159265, 0.0], np.float32)
    r = N.round_bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                         # tie rounds to even
    assert r[2] == np.float32(1.0 + 2 ** -7)   # above the tie rounds up
    assert abs(r[3] + 3.140625) < 1e-7
    assert r[4] == 0.0
    # a weight-rounded parameter vector keeps its biases
    p = _params(2).astype(np.float32)
    q = N.weights_bf16(p, WIDTHS)
    nW = WIDTHS[1] * WIDTHS[0]
    assert np.array_equal(q[nW:nW + WIDTHS[1]], p[nW:nW + WIDTHS[1]])


def test_adam_first_step_is_sign_times_lr():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -1e-3, 2.0])
    p1, m, v = N.adam_step(p, g, np.zeros(3), np.zeros(3), 1, 0.01, eps=0.0)
    assert np.allclose(p1, p - 0.01 * np.sign(g), rtol=0, atol=1e-15)


def test_training_reduces_loss():
    rng = np.random.default_rng(3)
    p = _params(4)
    x = rng.uniform(-1, 1, (64, 9))
    t = np.sin(x @ rng.normal(size=(9, 10)))
    m, v = np.zeros_like(p), np.zeros_like(p)
    l0 = N.loss_and_grad(p, WIDTHS, x, t)[0]
    for s in range(1, 201):
        _, g = N.loss_and_grad(p, WIDTHS, x, t)
        p, m, v = N.adam_step(p, g, m, v, s, 1e-2)
    assert N.loss_and_grad(p, WIDTHS, x, t)[0] < 0.2 * l0

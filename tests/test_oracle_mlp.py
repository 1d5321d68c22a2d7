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


def _nearest_bf16_brute(v):
    # The two BF16 neighbours of a positive normal float32 (truncation and
    # one BF16 ulp above), the nearer one in FP64, ties to the even pattern.
    out = np.empty_like(v)
    for i, x in enumerate(v):
        bits = int(np.float32(x).view(np.uint32))
        lo_bits = bits & 0xFFFF0000
        hi_bits = lo_bits + 0x10000
        lo = float(np.uint32(lo_bits).view(np.float32))
        hi = float(np.uint32(hi_bits).view(np.float32))
        dl, dh = float(x) - lo, hi - float(x)
        if dl < dh or (dl == dh and ((lo_bits >> 16) & 1) == 0):
            out[i] = lo
        else:
            out[i] = hi
    return out


def test_bf16_rounding_by_brute_force_and_odd_ties():
    rng = np.random.default_rng(5)
    v = (rng.uniform(0.5, 2.0, 3000) * 2.0 ** rng.integers(-20, 20, 3000)).astype(np.float32)
    assert np.array_equal(N.round_bf16(v), _nearest_bf16_brute(v))
    assert np.array_equal(N.round_bf16(-v), -_nearest_bf16_brute(v))
    # ties between an odd and an even neighbour go to the even one, upwards
    odd_tie = np.float32(1.0 + 2 ** -7 + 2 ** -8)
    assert N.round_bf16(np.array([odd_tie]))[0] == np.float32(1.0 + 2 ** -6)
    assert N.round_bf16(np.array([np.float32(3.0 + 3 * 2 ** -7)]))[0] == np.float32(3.0 + 2 ** -5)


def test_weights_bf16_rounds_every_weight_and_no_bias():
    p = _params(6).astype(np.float32)
    q = N.weights_bf16(p, WIDTHS)
    o = 0
    for l in range(len(WIDTHS) - 1):
        n = WIDTHS[l + 1] * WIDTHS[l]
        assert np.array_equal(q[o:o + n], N.round_bf16(p[o:o + n]))
        assert np.all((q[o:o + n].view(np.uint32) & 0xFFFF) == 0)
        o += n
        assert np.array_equal(q[o:o + WIDTHS[l + 1]], p[o:o + WIDTHS[l + 1]])
        o += WIDTHS[l + 1]
    assert o == p.size


def test_standardise_closed_form():
    shift, scale = np.array([4.0, -2.0]), np.array([2.0, 0.5])
    k = np.array([[0.0, 0.0], [1.0, -3.0], [-0.25, 2.0]])
    t = 10.0 ** (shift + k / scale)
    assert np.allclose(N.standardise(t, shift, scale, True), k, rtol=0, atol=1e-13)
    assert np.allclose(N.standardise(shift + k / scale, shift, scale, False), k, rtol=0, atol=1e-13)


def test_loss_value_and_output_bias_gradient():
    # Targets offset from the prediction by +1/2 everywhere: the loss is 1/4
    # and the last layer's bias gradient is 2 (-1/2) B / (B n_out) = -1/n_out.
    rng = np.random.default_rng(8)
    p = _params(7)
    x = rng.uniform(-1, 1, (11, 9))
    y, _ = N.forward(p, WIDTHS, x)
    assert N.loss_and_grad(p, WIDTHS, x, y)[0] == 0.0
    loss, g = N.loss_and_grad(p, WIDTHS, x, y + 0.5)
    assert abs(loss - 0.25) < 1e-15
    assert np.allclose(g[-WIDTHS[-1]:], -1.0 / WIDTHS[-1], rtol=1e-13)


def test_adam_two_steps_and_epsilon():
    # After gradients g1, g2 the bias-corrected moments are the normalised
    # exponential averages (b1 g1 + g2) / (1 + b1) and (b2 g1^2 + g2^2) / (1 + b2),
    # with Kingma & Ba's defaults b1 = 0.9, b2 = 0.999.
    p0 = np.array([0.3, -1.0, 2.0])
    g1 = np.array([0.4, -0.2, 1.5])
    g2 = np.array([-0.1, -0.6, 0.5])
    z = np.zeros(3)
    p1, m, v = N.adam_step(p0, g1, z, z, 1, 0.01, eps=0.0)
    p2, _, _ = N.adam_step(p1, g2, m, v, 2, 0.01, eps=0.0)
    mh = (0.9 * g1 + g2) / 1.9
    vh = (0.999 * g1 ** 2 + g2 ** 2) / 1.999
    assert np.allclose(p2, p1 - 0.01 * mh / np.sqrt(vh), rtol=0, atol=1e-15)
    # a gradient equal to the default eps = 1e-8 moves half a step
    q1, _, _ = N.adam_step(p0, np.full(3, 1e-8), z, z, 1, 0.01)
    assert np.allclose(q1, p0 - 0.005, rtol=0, atol=1e-12)

"""The surrogate GEMMs' handling of FP32 operands on BF16 tensor cores: an
FP32 value enters as a pair of BF16 numbers x = hi + lo, hi = bf16(x),
lo = bf16(x - hi), and a product of two such operands is taken as
hi_a hi_b + lo_a hi_b + hi_a lo_b (the lo_a lo_b term, ~2^-16 of the product,
is dropped); products of BF16 numbers are exact in FP32 and the sums are FP32.
Emulated here in numpy on 256-term dot products (the layers' width), against
FP64: a BF16 weight times an FP32 activation keeps the activation to about
2^-16, two FP32 operands lose about 2^-15 of each product, i.e. the GEMMs
match FP32 operands to ~1e-5 relative to sum |a b|, as the forward (1.3e-5)
and gradient (3.9e-6) parity of the kernels shows."""
import numpy as np

from oracle.mlp import round_bf16


def _split(x):
    x = np.asarray(x, np.float32)
    hi = round_bf16(x)
    lo = round_bf16(x - hi)
    return hi, lo


def _dot_f32(terms):
    # FP32 accumulation of FP32-exact products, in order
    acc = np.zeros(terms[0].shape[:-1], np.float32)
    for t in terms:
        for k in range(t.shape[-1]):
            acc = np.float32(acc + t[..., k].astype(np.float32))
    return acc


def test_split_keeps_sixteen_bits():
    rng = np.random.default_rng(4)
    x = (rng.normal(size=20000) * 10.0 ** rng.uniform(-3, 3, 20000)).astype(np.float32)
    hi, lo = _split(x)
    assert np.all((hi.view(np.uint32) & 0xFFFF) == 0) and np.all((lo.view(np.uint32) & 0xFFFF) == 0)
    rel = np.abs((hi.astype(np.float64) + lo) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -16


def test_weight_times_activation_and_activation_times_gradient():
    rng = np.random.default_rng(5)
    n, K = 64, 256
    W = round_bf16(rng.normal(0, 0.06, (n, K)).astype(np.float32))       # BF16 weights
    x = rng.normal(0, 1.0, (n, K)).astype(np.float32)                    # FP32 activations
    g = (rng.normal(0, 1e-3, (n, K))).astype(np.float32)                 # FP32 output gradients
    # BF16 weight x FP32 activation: W hi_x + W lo_x (W has no lo part)
    xh, xl = _split(x)
    y = _dot_f32([W * xh, W * xl])
    exact = np.sum(W.astype(np.float64) * x, axis=1)
    scale = np.sum(np.abs(W.astype(np.float64) * x), axis=1)
    assert np.max(np.abs(y - exact) / scale) <= 2.0 ** -15      # 2^-17 per product + FP32 sums
    assert np.max(np.abs(_dot_f32([W * xh]) - exact) / scale) > 2.0 ** -12   # the lo part is needed
    # FP32 x FP32: hi hi + lo hi + hi lo
    gh, gl = _split(g)
    z = _dot_f32([xh * gh, xl * gh, xh * gl])
    exact = np.sum(x.astype(np.float64) * g, axis=1)
    scale = np.sum(np.abs(x.astype(np.float64) * g), axis=1)
    err = np.max(np.abs(z - exact) / scale)
    assert err <= 2.0 ** -14
    # dropping a cross term instead costs ~2^-9: the three terms are needed
    z2 = _dot_f32([xh * gh, xh * gl])
    assert np.max(np.abs(z2 - exact) / scale) > 30 * err

"""Surrogate network of the screened sampler, in FP64 (test infrastructure).

The paper has no learned component (ML surrogates appear only as related work,
Sec. 1); the library's surrogate is a multilayer perceptron
theta (9) -> 256 -> 256 -> 256 -> band values (10), GELU activations, trained
by Adam on spectra produced by the forward model.  This module writes out the
plain definitions the GPU kernels must reproduce:

* layer l: z_l = W_l h_{l-1} + b_l; h_l = GELU(z_l) except on the last layer;
  GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2;
* inputs are affinely rescaled, x = (theta - in_shift) * in_scale, and the
  network predicts standardised targets, (log10(t) - out_shift) * out_scale
  when log_outputs is set, else (t - out_shift) * out_scale;
* loss = mean over the batch and outputs of the squared error of the
  standardised prediction;
* Adam (Kingma & Ba 2015) with bias correction:
  m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parameters are a flat vector: for each layer W_l (row-major [out][in]) then b_l.
When the forward pass uses BF16 weights, `weights_bf16` rounds every W_l to the
nearest BF16 value (ties to even) before use, exactly as the kernels do; biases
and the master copy stay FP32/FP64.
"""
import math

import numpy as np
from scipy.special import erf


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def n_params(widths):
    return sum(widths[l + 1] * widths[l] + widths[l + 1] for l in range(len(widths) - 1))


def unpack(flat, widths):
    out, o = [], 0
    for l in range(len(widths) - 1):
        n_in, n_out = widths[l], widths[l + 1]
        W = np.asarray(flat[o:o + n_out * n_in], np.float64).reshape(n_out, n_in)
        o += n_out * n_in
        b = np.asarray(flat[o:o + n_out], np.float64)
        o += n_out
        out.append((W, b))
    return out


def round_bf16(a):
    """Nearest BF16 value (round to nearest, ties to even) of float32 values."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def weights_bf16(flat, widths):
    """Copy of the flat parameters with every weight matrix rounded to BF16."""
    flat = np.asarray(flat, np.float32).copy()
    o = 0
    for l in range(len(widths) - 1):
        n = widths[l + 1] * widths[l]
        flat[o:o + n] = round_bf16(flat[o:o + n])
        o += n + widths[l + 1]
    return flat


def forward(flat, widths, x):
    """Returns (y, cache) for inputs x [B][in] (already rescaled)."""
    layers = unpack(flat, widths)
    h = np.asarray(x, np.float64)
    cache = [h]
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append(z)
        h = gelu(z) if l < len(layers) - 1 else z
    return h, cache


def standardise(t, out_shift, out_scale, log_outputs):
    t = np.asarray(t, np.float64)
    if log_outputs:
        t = np.log10(t)
    return (t - np.asarray(out_shift)) * np.asarray(out_scale)


def loss_and_grad(flat, widths, x, t_std):
    """Mean squared error against standardised targets and its gradient."""
    layers = unpack(flat, widths)
    y, cache = forward(flat, widths, x)
    B, n_out = y.shape
    r = y - t_std
    loss = float(np.mean(r * r))
    dh = 2.0 * r / (B * n_out)
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        z = cache[l + 1]
        dz = dh if l == len(layers) - 1 else dh * gelu_grad(z)
        h_prev = gelu(cache[l]) if l > 0 else cache[0]
        grads.append((dz.T @ h_prev, dz.sum(axis=0)))
        dh = dz @ W
    grads.reverse()
    flat_g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat_g


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v

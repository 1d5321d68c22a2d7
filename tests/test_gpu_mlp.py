"""GPU parity of the surrogate network's forward, backward and Adam kernels
against the FP64 oracle network (same BF16-rounded weights)."""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as N
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu

WIDTHS = list(W.SURROGATE_WIDTHS)


@pytest.fixture(scope="module")
def ctx():
    return make_ctx()


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _data(B, seed=0):
    rng = np.random.default_rng(seed)
    th = (W.THETA_LO + rng.uniform(size=(B, 9)) * (W.THETA_HI - W.THETA_LO)).astype(np.float32)
    t = (10 ** rng.uniform(3.5, 4.5, (B, 10))).astype(np.float32)
    return th, t


def _scaling():
    in_shift = (0.5 * (W.THETA_LO + W.THETA_HI)).astype(np.float32)
    in_scale = (2.0 / (W.THETA_HI - W.THETA_LO)).astype(np.float32)
    out_shift = np.full(10, 4.0, np.float32)
    out_scale = np.full(10, 2.0, np.float32)
    return in_shift, in_scale, out_shift, out_scale


def _net(ctx, torch, bf16, params):
    import paper_2104_12522_gb300 as bart
    net = bart.Mlp(ctx, WIDTHS, bf16_weights=bf16, log_outputs=True, max_batch=2048)
    net.set_scaling(*_scaling())
    net.set_params(torch.tensor(params, device="cuda"))
    return net


def _oracle_inputs(th, t):
    a, b, c, d = _scaling()
    return (th.astype(np.float64) - a) * b, N.standardise(t, c, d, True)


@pytest.mark.parametrize("bf16", [True, False])
def test_forward_and_gradient_match_oracle(ctx, torch, bf16):
    p = W.mlp_init(WIDTHS)
    th, t = _data(300)
    net = _net(ctx, torch, bf16, p)
    x_dev, t_dev = torch.tensor(th, device="cuda"), torch.tensor(t, device="cuda")
    y = net.forward(x_dev).cpu().numpy().astype(np.float64)
    g, loss = net.gradient(x_dev, t_dev)
    g, loss = g.cpu().numpy().astype(np.float64), float(loss.cpu())
    pw = N.weights_bf16(p, WIDTHS) if bf16 else p
    x, ts = _oracle_inputs(th, t)
    y_std, _ = N.forward(pw, WIDTHS, x)
    a, b, c, d = _scaling()
    y_o = 10 ** (y_std / d + c)
    lo, go = N.loss_and_grad(pw, WIDTHS, x, ts)
    ey = np.max(np.abs(y - y_o) / y_o)
    # per-tensor relative L2 error of the gradient
    eg, o = 0.0, 0
    for l in range(len(WIDTHS) - 1):
        for n in (WIDTHS[l + 1] * WIDTHS[l], WIDTHS[l + 1]):
            ref = go[o:o + n]
            eg = max(eg, np.linalg.norm(g[o:o + n] - ref) / np.linalg.norm(ref))
            o += n
    print(f"MLP ({'bf16' if bf16 else 'fp32'} weights): forward {ey:.2e}, loss {abs(loss - lo) / lo:.2e}, "
          f"gradient {eg:.2e}")
    assert ey < 1e-4 and abs(loss - lo) / lo < 1e-4
    assert eg < (1e-3 if bf16 else 1e-5)


def test_adam_steps_match_oracle(ctx, torch):
    p = W.mlp_init(WIDTHS)
    th, t = _data(256, seed=1)
    net = _net(ctx, torch, False, p)
    x_dev, t_dev = torch.tensor(th, device="cuda"), torch.tensor(t, device="cuda")
    x, ts = _oracle_inputs(th, t)
    po, m, v = p.astype(np.float64), np.zeros(p.size), np.zeros(p.size)
    for s in range(1, 4):
        net.train_step(x_dev, t_dev, 1e-3)
        _, go = N.loss_and_grad(po, WIDTHS, x, ts)
        po, m, v = N.adam_step(po, go, m, v, s, 1e-3)
    got = net.get_params().cpu().numpy().astype(np.float64)
    # Adam normalises each step to ~lr, so compare the displacement
    err = np.linalg.norm((got - p) - (po - p)) / np.linalg.norm(po - p)
    print(f"Adam (3 steps, fp32 weights): displacement rel error {err:.2e}")
    assert err < 1e-3


def test_training_reduces_loss(ctx, torch):
    th, t = _data(2048, seed=2)
    # a smooth target the network can learn
    t = (10 ** (4.0 + 0.2 * np.sin(th @ np.linspace(0.1, 0.9, 90).reshape(9, 10)))).astype(np.float32)
    net = _net(ctx, torch, True, W.mlp_init(WIDTHS))
    x_dev, t_dev = torch.tensor(th, device="cuda"), torch.tensor(t, device="cuda")
    loss = torch.empty(1, device="cuda")
    net.train_step(x_dev, t_dev, 1e-3, loss)
    l0 = float(loss.cpu())
    for _ in range(300):
        net.train_step(x_dev, t_dev, 1e-3, loss)
    l1 = float(loss.cpu())
    print(f"training: loss {l0:.3e} -> {l1:.3e}")
    assert l1 < 0.05 * l0


def test_train_steps_equal_single_steps(ctx, torch):
    """bart_mlp_train_steps (the step loop in the library, batches gathered
    on the device) gives the parameters of the same sequence of single
    bart_mlp_train_step calls, bit for bit."""
    th, t = _data(600, seed=3)
    x_dev, t_dev = torch.tensor(th, device="cuda"), torch.tensor(t, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(11)
    rows = torch.randint(0, 600, (5, 128), device="cuda", generator=g, dtype=torch.int32)
    lrs = [1e-3, 8e-4, 6e-4, 4e-4, 2e-4]
    a = _net(ctx, torch, True, W.mlp_init(WIDTHS))
    loss = torch.empty(5, device="cuda")
    a.train_steps(x_dev, t_dev, rows, lrs, loss)
    b = _net(ctx, torch, True, W.mlp_init(WIDTHS))
    for k in range(5):
        r = rows[k].long()
        b.train_step(x_dev[r].contiguous(), t_dev[r].contiguous(), lrs[k])
    ctx.sync()
    assert torch.equal(a.get_params(), b.get_params())
    assert torch.isfinite(loss).all()

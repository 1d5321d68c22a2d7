"""A DE-MC run checkpointed to a file and resumed in a fresh sampler continues
exactly: random numbers are keyed by (seed, half-step, chain, draw), so after
the resumed half-steps the chains and log-likelihoods equal those of the
uninterrupted run bit for bit (the paper's sampler saves its state at
intervals during a run, Sec. 5)."""
import numpy as np
import pytest

from gpu_common import make_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return make_ctx()


def test_resumed_run_continues_exactly(ctx, tmp_path):
    import torch
    import paper_2104_12522_gb300 as bart
    C, d = 10, 3
    lo, hi = np.zeros(d, np.float32), np.ones(d, np.float32)
    mu = torch.full((d,), 0.5, dtype=torch.float64, device="cuda")

    def L(y):          # the target density is test data, evaluated with torch
        r = y.double() - mu
        return (-0.5 * (r * r).sum(dim=1) / 0.01).contiguous()

    s = bart.Demc(ctx, C, lo, hi, jump_every=10, eps=1e-4, seed=6301)
    x0 = torch.tensor(np.random.default_rng(0).uniform(0.3, 0.7, (C, d)).astype(np.float32), device="cuda")
    s.set_state(x0, L(x0))
    y = torch.empty((C, d), dtype=torch.float32, device="cuda")
    inbox = torch.empty(C, dtype=torch.int32, device="cuda")
    passed = torch.empty(C, dtype=torch.int32, device="cuda")

    def half_step(smp, h):
        smp.propose(h, y, inbox)
        ly = L(y)
        smp.screen(h, inbox, None, passed)
        smp.accept(h, y, passed, ly)

    for h in range(40):
        half_step(s, h)
    path = str(tmp_path / "demc.npz")
    bart.save_checkpoint(path, s.checkpoint(40))
    ck = bart.load_checkpoint(path)
    assert ck["next_half_step"] == 40
    r = bart.Demc.from_checkpoint(ctx, ck)
    for h in range(40, 100):
        half_step(s, h)
        half_step(r, h)
    a, b = s.checkpoint(100), r.checkpoint(100)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["loglike"], b["loglike"])
    assert not np.array_equal(a["x"], x0.cpu().numpy())          # the chains moved

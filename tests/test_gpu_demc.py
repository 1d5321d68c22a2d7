"""GPU DE-MC sampler (two-halves proposals, delayed-acceptance screen): it
samples a correlated 9-D Gaussian with the moments and credible-region
content the App. C standard errors allow, like the oracle sampler; and the
band log-likelihood kernel matches its FP64 definition."""
import numpy as np
import pytest
from scipy.stats import chi2

from oracle import demc as D
from demc_target import target
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return make_ctx()


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _run_gpu(ctx, torch, n_gen, screened, seed=6000, beta=1.0, margin=0.0):
    import paper_2104_12522_gb300 as bart
    mu, cov, lo, hi = target()
    C, d = 16, 9
    inv = torch.tensor(np.linalg.inv(cov), device="cuda")
    mu_t = torch.tensor(mu, device="cuda")
    # the target density is test data: evaluated here with torch
    def L(y):
        r = y.double() - mu_t
        return -0.5 * torch.einsum("ij,jk,ik->i", r, inv, r)
    s = bart.Demc(ctx, C, lo.astype(np.float32), hi.astype(np.float32), jump_every=10, eps=1e-4, seed=seed)
    s.set_screen(beta, margin)
    rng = np.random.default_rng(seed)
    x0 = torch.tensor((mu + rng.normal(size=(C, d)) * np.sqrt(np.diag(cov))).astype(np.float32), device="cuda")
    ls0 = 0.7 * L(x0) if screened else None
    s.set_state(x0, L(x0).contiguous(), ls0.contiguous() if screened else None)
    y = torch.empty((C, d), dtype=torch.float32, device="cuda")
    inbox = torch.empty(C, dtype=torch.int32, device="cuda")
    passed = torch.empty(C, dtype=torch.int32, device="cuda")
    acc = torch.zeros(C, dtype=torch.int32, device="cuda")
    hist = []
    x = torch.empty((C, d), dtype=torch.float32, device="cuda")
    n_acc = 0
    for g in range(n_gen):
        for h in (0, 1):
            hs = 2 * g + h
            s.propose(hs, y, inbox)
            ly = L(y).contiguous()
            ls = (0.7 * ly).contiguous() if screened else None
            s.screen(hs, inbox, ls, passed)
            s.accept(hs, y, passed, ly, ls, acc)
            n_acc += int(acc.sum())
        s.get_state(x)
        hist.append(x.cpu().numpy().astype(np.float64))
    return np.array(hist), n_acc, mu, cov


@pytest.mark.parametrize("screened,beta,margin", [(False, 1.0, 0.0), (True, 1.0, 0.0), (True, 0.5, 2.0)])
def test_gpu_sampler_recovers_gaussian(ctx, torch, screened, beta, margin):
    hist, n_acc, mu, cov = _run_gpu(ctx, torch, 3000, screened, beta=beta, margin=margin)
    s = hist[500:]
    n, C, d = s.shape
    flat = s.reshape(-1, d)
    e = D.ess(s)
    sd = np.sqrt(np.diag(cov))
    z = np.abs(flat.mean(0) - mu) / (sd / np.sqrt(e))
    var_ratio = flat.var(0) / sd ** 2
    inv = np.linalg.inv(cov)
    m2 = np.einsum("ij,jk,ik->i", flat - mu, inv, flat - mu)
    c = float(np.mean(m2 <= chi2.ppf(0.6827, d)))
    print(f"GPU DE-MC ({'screened' if screened else 'plain'}): ESS {e:.0f}, max |z| mean {z.max():.2f}, "
          f"var ratio {var_ratio.min():.3f}..{var_ratio.max():.3f}, C68 {c:.4f}, accepted {n_acc}")
    assert e > 300
    assert np.all(z < 4.5)
    assert np.all(np.abs(var_ratio - 1) < 4.5 * np.sqrt(2.0 / e))
    assert abs(c - 0.6827) < 4.5 * D.credible_content_se(0.6827, e)


def test_proposals_respect_halves_and_box(ctx, torch):
    import paper_2104_12522_gb300 as bart
    C, d = 10, 3
    lo, hi = np.zeros(d, np.float32), np.ones(d, np.float32)
    s = bart.Demc(ctx, C, lo, hi, eps=0.0, seed=1)
    x0 = torch.tensor(np.random.default_rng(0).uniform(0.2, 0.8, (C, d)).astype(np.float32), device="cuda")
    s.set_state(x0, torch.zeros(C, dtype=torch.float64, device="cuda"))
    y = torch.empty((C, d), dtype=torch.float32, device="cuda")
    inbox = torch.empty(C, dtype=torch.int32, device="cuda")
    for hs in range(6):
        s.propose(hs, y, inbox)
        own = slice(0, C // 2) if hs % 2 == 0 else slice(C // 2, C)
        other = slice(C // 2, C) if hs % 2 == 0 else slice(0, C // 2)
        yy, ib, xx = y.cpu().numpy(), inbox.cpu().numpy(), x0.cpu().numpy()
        assert np.all(ib[other] == 0) and np.array_equal(yy[other], xx[other])
        inside = np.all((yy[own] >= 0) & (yy[own] <= 1), axis=1)
        assert np.array_equal(ib[own] == 1, inside)
        # eps = 0: every move is gamma times a difference of two other-half chains
        diffs = xx[other][:, None, :] - xx[other][None, :, :]
        gam = 2.38 / np.sqrt(2 * d) if (hs // 2) % 10 != 9 else 1.0
        for i in range(*own.indices(C)):
            step = (yy[i] - xx[i]) / gam
            assert np.min(np.max(np.abs(diffs - step), axis=2)) < 1e-5


def test_loglike_bands(ctx, torch):
    rng = np.random.default_rng(3)
    m = rng.uniform(1, 2, (33, 10)).astype(np.float32)
    dat = rng.uniform(1, 2, 10).astype(np.float32)
    sig = rng.uniform(0.01, 0.1, 10).astype(np.float32)
    mask = (rng.uniform(size=33) > 0.3).astype(np.int32)
    dev = lambda a: torch.tensor(a, device="cuda")
    out = torch.empty(33, dtype=torch.float64, device="cuda")
    ctx.loglike_bands(dev(m), dev(dat), dev(sig), out, mask=dev(mask))
    ref = -0.5 * np.sum(((m.astype(np.float64) - dat) / sig.astype(np.float64)) ** 2, axis=1)
    got = out.cpu().numpy()
    assert np.all(np.isneginf(got[mask == 0]))
    assert np.allclose(got[mask == 1], ref[mask == 1], rtol=1e-12)


# ---- DEMCzs (Sec. 4) and the chain statistics (Sec. 5, App. C)

def _run_zs(ctx, torch, n_steps, C, p_snooker, screened=False, seed=6020):
    import paper_2104_12522_gb300 as bart
    mu, cov, lo, hi = target()
    d = 9
    sd = np.sqrt(np.diag(cov))
    inv = torch.tensor(np.linalg.inv(cov), device="cuda")
    mu_t = torch.tensor(mu, device="cuda")
    def L(y):
        r = y.double() - mu_t
        return -0.5 * torch.einsum("ij,jk,ik->i", r, inv, r)
    s = bart.Demc(ctx, C, lo.astype(np.float32), hi.astype(np.float32), jump_every=10, eps=1e-4, seed=seed)
    rng = np.random.default_rng(seed)
    z0 = torch.tensor((mu + rng.normal(size=(90, d)) * sd * 2.0).astype(np.float32), device="cuda")
    s.set_archive(z0, capacity=90 + C * (n_steps // 10), thin=10, p_snooker=p_snooker)
    x0 = torch.tensor((mu + rng.normal(size=(C, d)) * sd).astype(np.float32), device="cuda")
    ls0 = 0.7 * L(x0) if screened else None
    s.set_state(x0, L(x0).contiguous(), ls0.contiguous() if screened else None)
    y = torch.empty((C, d), dtype=torch.float32, device="cuda")
    inbox = torch.empty(C, dtype=torch.int32, device="cuda")
    passed = torch.empty(C, dtype=torch.int32, device="cuda")
    hist = torch.empty((n_steps, C, d), dtype=torch.float32, device="cuda")
    for st in range(n_steps):
        s.propose(st, y, inbox)
        ly = L(y).contiguous()
        ls = (0.7 * ly).contiguous() if screened else None
        s.screen(st, inbox, ls, passed)
        s.accept(st, y, passed, ly, ls)
        s.get_state(hist[st])
    return s, hist, mu, cov


@pytest.mark.parametrize("C,p_snooker,screened", [(3, 0.1, False), (4, 1.0, False), (4, 0.1, True)])
def test_gpu_demczs_recovers_gaussian(ctx, torch, C, p_snooker, screened):
    n = 12000
    s, hist, mu, cov = _run_zs(ctx, torch, n, C, p_snooker, screened)
    assert s.archive_size() == 90 + C * (n // 10)
    sm = hist.cpu().numpy().astype(np.float64)[2000:]
    flat = sm.reshape(-1, 9)
    e = D.ess(sm)
    sd = np.sqrt(np.diag(cov))
    z = np.abs(flat.mean(0) - mu) / (sd / np.sqrt(e))
    var_ratio = flat.var(0) / sd ** 2
    print(f"GPU DEMCzs (C={C}, p_snooker={p_snooker}, screened={screened}): ESS {e:.0f}, "
          f"max |z| {z.max():.2f}, var ratio {var_ratio.min():.3f}..{var_ratio.max():.3f}")
    assert e > 100
    assert np.all(z < 4.5)
    assert np.all(np.abs(var_ratio - 1) < 4.5 * np.sqrt(2.0 / e))


def test_chain_stats_match_the_oracle(ctx, torch):
    rng = np.random.default_rng(21)
    n, C, d = 3000, 4, 3
    x = np.zeros((n, C, d))
    phi = np.array([0.0, 0.5, 0.9])
    for t in range(1, n):
        x[t] = phi * x[t - 1] + rng.normal(size=(C, d))
    x += np.array([0.0, 0.1, 0.0, -0.1])[None, :, None]
    x32 = x.astype(np.float32)
    sp, gr, ess = ctx.chain_stats(torch.tensor(x32, device="cuda"))
    sp, gr = sp.cpu().numpy(), gr.cpu().numpy()
    ref_sp = np.array([[D.speis(x32[:, c, q].astype(np.float64)) for q in range(d)] for c in range(C)])
    ref_gr = D.gelman_rubin(x32.astype(np.float64))
    print(f"SPEIS GPU vs oracle: max rel {np.max(np.abs(sp / ref_sp - 1)):.2e}; GR {gr} vs {ref_gr}")
    assert np.allclose(sp, ref_sp, rtol=1e-9)
    assert np.allclose(gr, ref_gr, rtol=1e-9)
    assert abs(ess - D.ess(x32.astype(np.float64))) < 1e-6 * ess

"""The native retrieval loop (DE-MC + emission forward model + bands, with and
without the surrogate screen): graph replay equals eager execution, the
screen cuts exact evaluations, and screened and plain runs sample the same
posterior.  The surrogate is trained by the library's own kernels on spectra
the forward model produces."""
import numpy as np
import pytest

import workloads as W
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu

S, L, M, N, DNU = 4, 24, 6, 700, 0.05
NB = 10


@pytest.fixture(scope="module")
def ctx():
    return make_ctx()


@pytest.fixture(scope="module")
def setup(ctx):
    import torch
    import paper_2104_12522_gb300 as bart
    species = [W.line_list(s, 400, 1000.0, 1000.0 + N * DNU) for s in range(S)]
    species[3].mass_amu = 16.0
    p = W.log_pressures(L, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    nu = bart.NuGrid(1000.0, DNU, N)
    grid = ctx.build_opacity_grid([bart.device_lines(s) for s in species], p, t, nu, 25.0)
    filt = torch.tensor(W.gaussian_filters(W.nu_axis(1000.0, DNU, N), NB, 1002.0, 1033.0, 2.0, 12.0),
                        device="cuda")
    cfg = dict(geometry=0, n_angles=4, g=W.HD189_GRAV_CGS, mu=W.MEAN_MOLECULAR_MASS_AMU, x0=[W.BASE_VMR] * S,
               t_int=W.T_INT_K, t_star=W.HD189_TSTAR_K, r_star_tp=W.HD189_RSTAR_CM, a_orbit=W.HD189_A_CM,
               t_min=500.0, t_max=3000.0)

    def bands_of(theta):
        out = torch.empty((theta.shape[0], NB), dtype=torch.float32, device="cuda")
        ctx.forward_spectra_batch(grid, p, t, nu, cfg, theta=theta, filters=filt, bands=out)
        return out

    # synthetic data: the model at a seeded true theta plus noise at S/N = 50
    rng = np.random.default_rng(6500)
    truth = (W.THETA_LO + rng.uniform(0.3, 0.7, 9) * (W.THETA_HI - W.THETA_LO)).astype(np.float32)
    b_true = bands_of(torch.tensor(truth[None], device="cuda")).cpu().numpy()[0]
    sigma = (b_true / 50.0).astype(np.float32)
    data = (b_true + rng.normal(size=NB) * sigma).astype(np.float32)

    # surrogate: trained on forward-model spectra with the library's kernels
    th_train = torch.tensor(W.proposals(8192, generation=11, n_species=S), device="cuda")
    y_train = torch.cat([bands_of(th_train[i:i + 2048]) for i in range(0, 8192, 2048)])
    net = bart.Mlp(ctx, W.SURROGATE_WIDTHS, bf16_weights=True, log_outputs=True, max_batch=2048)
    lo, hi = W.THETA_LO.astype(np.float32), W.THETA_HI.astype(np.float32)
    logy = np.log10(y_train.cpu().numpy().astype(np.float64))
    net.set_scaling(0.5 * (lo + hi), 2.0 / (hi - lo), logy.mean(0).astype(np.float32),
                    (1.0 / logy.std(0)).astype(np.float32))
    net.set_params(torch.tensor(W.mlp_init(), device="cuda"))
    g = torch.Generator(device="cuda").manual_seed(5000)
    for step in range(600):
        idx = torch.randint(0, 8192, (1024,), device="cuda", generator=g)
        net.train_step(th_train[idx].contiguous(), y_train[idx].contiguous(), 1e-3)
    return dict(grid=grid, p=p, t=t, nu=nu, filt=filt, cfg=cfg, data=torch.tensor(data, device="cuda"),
                sigma=torch.tensor(sigma, device="cuda"), net=net, bands_of=bands_of, truth=truth)


def _sampler(ctx, su, seed, screened):
    import torch
    import paper_2104_12522_gb300 as bart
    lo, hi = W.THETA_LO.astype(np.float32), W.THETA_HI.astype(np.float32)
    s = bart.Demc(ctx, 16, lo, hi, jump_every=10, eps=1e-4, seed=seed)
    rng = np.random.default_rng(seed)
    x0 = torch.tensor((lo + rng.uniform(size=(16, 9)) * (hi - lo)).astype(np.float32), device="cuda")
    L0 = torch.empty(16, dtype=torch.float64, device="cuda")
    ctx.loglike_bands(su["bands_of"](x0), su["data"], su["sigma"], L0)
    Ls0 = None
    if screened:
        Ls0 = torch.empty(16, dtype=torch.float64, device="cuda")
        ctx.loglike_bands(su["net"].forward(x0), su["data"], su["sigma"], Ls0)
    s.set_state(x0, L0, Ls0)
    return s


def _run(ctx, su, seed, screened, n_gen, graph):
    import torch
    s = _sampler(ctx, su, seed, screened)
    chain = torch.empty((n_gen, 16, 9), dtype=torch.float32, device="cuda")
    st = ctx.retrieval_run(s, su["net"] if screened else None, su["grid"], su["p"], su["t"], su["nu"], su["cfg"],
                           su["filt"], su["data"], su["sigma"], n_gen, use_graph=graph, chain=chain)
    return chain.cpu().numpy(), st


def test_surrogate_accuracy(ctx, setup):
    import torch
    th = torch.tensor(W.proposals(512, generation=12, n_species=S), device="cuda")
    exact = setup["bands_of"](th).cpu().numpy()
    pred = setup["net"].forward(th).cpu().numpy()
    err = np.abs(pred / exact - 1)
    print(f"surrogate band error on held-out proposals: median {np.median(err):.2e}, p99 "
          f"{np.percentile(err, 99):.2e}")
    assert np.median(err) < 0.05


@pytest.mark.parametrize("screened", [False, True])
def test_graph_replay_equals_eager(ctx, setup, screened):
    a, sa = _run(ctx, setup, 6001, screened, 40, graph=False)
    b, sb = _run(ctx, setup, 6001, screened, 40, graph=True)
    assert np.array_equal(a, b)
    assert sa == sb


def test_screen_cuts_exact_evaluations_and_keeps_posterior(ctx, setup):
    n_gen = 1500
    plain, sp = _run(ctx, setup, 6002, False, n_gen, graph=True)
    scr, ss = _run(ctx, setup, 6002, True, n_gen, graph=True)
    print(f"plain: {sp}\nscreened: {ss}")
    assert sp["exact_evals"] == sp["proposals"] and sp["screened_out"] == 0
    assert ss["exact_evals"] + ss["screened_out"] == ss["proposals"]
    assert ss["exact_evals"] < 0.8 * ss["proposals"]
    assert ss["accepted"] > 0
    # posterior means of the two runs agree within their combined spread
    burn = n_gen // 2
    mp, ms = plain[burn:].reshape(-1, 9), scr[burn:].reshape(-1, 9)
    width = W.THETA_HI - W.THETA_LO
    diff = np.abs(mp.mean(0) - ms.mean(0)) / width
    spread = np.sqrt(mp.var(0) + ms.var(0)) / width
    print("posterior mean difference / box width:", np.round(diff, 4))
    assert np.all(diff < 3 * spread + 0.02)


def test_screen_gains_ess_per_exact_evaluation_at_equal_posterior(ctx, setup):
    """What the surrogate buys: after a shared exact-model burn-in, the
    screened DE-MC sampler reaches the plain sampler's posterior within the
    App. C standard errors (means: s = sigma / sqrt(ESS); central 68% interval
    content: s_C = sqrt(C (1 - C) / ESS), the large-ESS form) while spending fewer exact
    forward-model evaluations per effective sample (Sec. 5 ESS and SPEIS).
    The data here are the model at the seeded truth with noise at S/N = 10 per
    band, so that 16 chains mix within the run and the ESS estimates hold."""
    import torch
    import paper_2104_12522_gb300 as bart
    lo, hi = W.THETA_LO.astype(np.float32), W.THETA_HI.astype(np.float32)
    su = setup
    b_true = su["bands_of"](torch.tensor(su["truth"][None], device="cuda")).cpu().numpy()[0]
    sig = (b_true / 10.0).astype(np.float32)
    rng = np.random.default_rng(6600)
    data = torch.tensor((b_true + rng.normal(size=NB) * sig).astype(np.float32), device="cuda")
    sigma = torch.tensor(sig, device="cuda")
    x0 = torch.tensor((lo + rng.uniform(size=(16, 9)) * (hi - lo)).astype(np.float32), device="cuda")
    L0 = torch.empty(16, dtype=torch.float64, device="cuda")
    ctx.loglike_bands(su["bands_of"](x0), data, sigma, L0)
    s0 = bart.Demc(ctx, 16, lo, hi, jump_every=10, eps=1e-4, seed=6100)
    s0.set_state(x0, L0)
    ctx.retrieval_run(s0, None, su["grid"], su["p"], su["t"], su["nu"], su["cfg"], su["filt"], data, sigma, 3000,
                      use_graph=True)
    x_b = torch.empty((16, 9), dtype=torch.float32, device="cuda")
    L_b = torch.empty(16, dtype=torch.float64, device="cuda")
    s0.get_state(x_b, L_b)
    n_gen = 6000
    out = {}
    for mode in ("plain", "screened"):
        s = bart.Demc(ctx, 16, lo, hi, jump_every=10, eps=1e-4, seed=6200)
        Ls = None
        if mode == "screened":
            s.set_screen(1.0, 1.0)
            Ls = torch.empty(16, dtype=torch.float64, device="cuda")
            ctx.loglike_bands(su["net"].forward(x_b), data, sigma, Ls)
        s.set_state(x_b.clone(), L_b.clone(), Ls)
        chain = torch.empty((n_gen, 16, 9), dtype=torch.float32, device="cuda")
        st = ctx.retrieval_run(s, su["net"] if mode == "screened" else None, su["grid"], su["p"], su["t"], su["nu"],
                               su["cfg"], su["filt"], data, sigma, n_gen, use_graph=True, chain=chain)
        sp, gr, ess = ctx.chain_stats(chain)
        out[mode] = dict(x=chain.reshape(-1, 9).double().cpu().numpy(),
                         ess_j=(n_gen * 16 / sp.mean(0)).cpu().numpy(), ess=ess, st=st,
                         ess_per_eval=ess / st["exact_evals"], gr=float(gr.max()))
    p, s = out["plain"], out["screened"]
    print(f"ESS per exact evaluation: plain {p['ess_per_eval']:.3e} ({p['ess']:.0f} / {p['st']['exact_evals']}), "
          f"screened {s['ess_per_eval']:.3e} ({s['ess']:.0f} / {s['st']['exact_evals']}); R max {p['gr']:.3f} / "
          f"{s['gr']:.3f}")
    assert s["ess_per_eval"] > 2.0 * p["ess_per_eval"]
    z_mean, z_c = [], []
    for j in range(9):
        sp_ = p["x"][:, j].std() / np.sqrt(p["ess_j"][j])
        ss_ = s["x"][:, j].std() / np.sqrt(s["ess_j"][j])
        z_mean.append(abs(p["x"][:, j].mean() - s["x"][:, j].mean()) / np.hypot(sp_, ss_))
        q16, q84 = np.percentile(p["x"][:, j], [16, 84])
        c = np.mean((s["x"][:, j] >= q16) & (s["x"][:, j] <= q84))
        z_c.append(abs(c - 0.68) / np.sqrt(0.68 * 0.32 * (1 / p["ess_j"][j] + 1 / s["ess_j"][j])))
    print("posterior agreement z (means):", np.round(z_mean, 2), " (68% content):", np.round(z_c, 2))
    # nine parameters, two statistics each: 4 standard errors leaves room for chance
    assert max(z_mean) < 4.0 and max(z_c) < 4.0

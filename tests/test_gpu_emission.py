"""GPU parity of the emission forward model and the spectrum integrator
against the FP64 oracle (Sec. 3; f08isothermal Sec. 6.1.3)."""
import numpy as np
import pytest

import workloads as W
from oracle import opacity as O, forward as Fw, radiation as R
from gpu_common import make_ctx, max_rel

pytestmark = pytest.mark.gpu

RTOL = 1e-4      # spectra and band values, relative (FP32 path vs FP64 oracle)


@pytest.fixture(scope="module")
def ctx():
    return make_ctx()


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _cfg(n_angles, x0):
    return dict(geometry=0, n_angles=n_angles, g=W.HD189_GRAV_CGS, mu=W.MEAN_MOLECULAR_MASS_AMU, x0=list(x0),
                t_int=W.T_INT_K, t_star=W.HD189_TSTAR_K, r_star_tp=W.HD189_RSTAR_CM, a_orbit=W.HD189_A_CM,
                t_min=500.0, t_max=3000.0)


def test_small_emission_workload_end_to_end(ctx, torch):
    """2 species x 10,000 lines, 60 layers, 2,000 wavenumbers, 4 angles, 4
    top-hat bands: opacity on the spot, emission, band integration."""
    import paper_2104_12522_gb300 as bart
    w = W.emission_small()
    x0 = [W.BASE_VMR] * 2
    nu = bart.NuGrid(w.nu_start, w.dnu, w.n_nu)
    sig = ctx.opacity_cells([bart.device_lines(s) for s in w.species], w.p_bar, w.t_K, nu, w.cutoff)
    tprof = torch.tensor(w.t_K, dtype=torch.float32, device="cuda")[None].contiguous()
    spec = torch.empty((1, w.n_nu), dtype=torch.float32, device="cuda")
    filt = torch.tensor(w.filters, device="cuda")
    bands = torch.empty((1, 4), dtype=torch.float32, device="cuda")
    cfg = _cfg(4, x0)
    cfg.update(t_min=1.0, t_max=1e5)
    ctx.forward_spectra_batch(sig[:, :, None, :].contiguous(), w.p_bar, [1000.0], nu, cfg, t_profile=tprof,
                              spectra=spec, filters=filt, bands=bands, n=1)
    ctx.sync()
    sig_o = O.opacity_cells(w.species, w.p_bar, w.t_K, w.nu_start, w.dnu, w.n_nu, w.cutoff)
    chi = Fw.mass_opacity(sig_o, np.asarray(x0), W.MEAN_MOLECULAR_MASS_AMU)
    nu_ax = W.nu_axis(w.nu_start, w.dnu, w.n_nu)
    F = R.emission_flux(chi, w.p_bar, w.t_K, nu_ax, W.HD189_GRAV_CGS, 4)
    Bo = R.band_integrate(F, w.filters)
    e_spec, e_band = max_rel(spec.cpu().numpy()[0], F), max_rel(bands.cpu().numpy()[0], Bo)
    print(f"emission (small workload) FP32 vs FP64: spectrum {e_spec:.2e}, bands {e_band:.2e}")
    assert e_spec < RTOL and e_band < RTOL


def test_isothermal_gives_planck(ctx, torch):
    import paper_2104_12522_gb300 as bart
    rng = np.random.default_rng(5)
    S, L, N = 2, 40, 777
    p = W.log_pressures(L, 1e-6, 100.0)
    grid = torch.tensor(10 ** rng.uniform(-26, -18, (S, L, 1, N)), dtype=torch.float32, device="cuda")
    nu = bart.NuGrid(1000.0, 2.5, N)
    T = torch.full((3, L), 1234.5, dtype=torch.float32, device="cuda")
    spec = torch.empty((3, N), dtype=torch.float32, device="cuda")
    for na in (1, 8, 16):
        cfg = _cfg(na, [1e-4, 3e-4])
        cfg.update(t_min=1.0, t_max=1e5)
        ctx.forward_spectra_batch(grid, p, [1000.0], nu, cfg, t_profile=T, spectra=spec, n=3)
        exp = np.pi * R.planck(W.nu_axis(1000.0, 2.5, N), 1234.5)
        assert max_rel(spec.cpu().numpy(), exp[None]) < 1e-5


def _grid_case(S=2, L=24, M=6, N=700, dnu=0.05, n_lines=400):
    species = [W.line_list(s, n_lines, 1000.0, 1000.0 + N * dnu) for s in range(S)]
    p = W.log_pressures(L, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    return species, p, t, N, dnu


@pytest.fixture(scope="module")
def grid_case(ctx, torch):
    import paper_2104_12522_gb300 as bart
    species, p, t, N, dnu = _grid_case()
    nu = bart.NuGrid(1000.0, dnu, N)
    g_dev = ctx.build_opacity_grid([bart.device_lines(s) for s in species], p, t, nu, 25.0)
    g_ora = O.opacity_grid(species, p, t, 1000.0, dnu, N, 25.0)
    return species, p, t, N, dnu, nu, g_dev, g_ora


@pytest.mark.parametrize("n_angles", [4, 8])
def test_batched_emission_from_grid(ctx, torch, grid_case, n_angles):
    """Proposals with the five-parameter T(P) profile and log-abundance
    scalings, interpolated in T on a GPU-built grid; the oracle uses its own
    grid.  Includes spans that end inside a CTA tile."""
    species, p, t, N, dnu, nu, g_dev, g_ora = grid_case
    n = 37
    theta = W.proposals(n, generation=7, n_species=2)
    lo = np.array([0, 5, 129] + [0] * (n - 3), np.int64)
    hi = np.array([N, N - 3, 400] + [N] * (n - 3), np.int64)
    offs = np.concatenate([[0], np.cumsum(hi - lo)]).astype(np.int64)
    filt = W.gaussian_filters(W.nu_axis(1000.0, dnu, N), 5, 1002.0, 1033.0, 2.0, 12.0)
    x0 = [W.BASE_VMR] * 2
    cfg = _cfg(n_angles, x0)
    dev = lambda a: torch.tensor(a, device="cuda")
    spec = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    bands = torch.empty((n, 5), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, theta=dev(theta), nu_lo=dev(lo), nu_hi=dev(hi),
                              spec_offsets=dev(offs), spectra=spec, filters=dev(filt), bands=bands)
    ctx.sync()
    spec, bands = spec.cpu().numpy(), bands.cpu().numpy()
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0, x0=x0, mu=cfg["mu"], n_angles=n_angles)
    nu_ax = W.nu_axis(1000.0, dnu, N)
    es, eb = 0.0, 0.0
    for i in range(n):
        F = Fw.emission_spectrum(g_ora[..., lo[i]:hi[i]], p, t, nu_ax[lo[i]:hi[i]], theta[i], ocfg)
        es = max(es, max_rel(spec[offs[i]:offs[i + 1]], F))
        Bo = R.band_integrate(F, filt, nu_lo=lo[i])
        ok = Bo != 0
        if ok.any():
            eb = max(eb, max_rel(bands[i][ok], Bo[ok]))
        assert np.all(bands[i][~ok] == 0.0)
    print(f"batched emission ({n_angles} angles) FP32 vs FP64: spectra {es:.2e}, bands {eb:.2e}")
    assert es < RTOL and eb < RTOL


@pytest.mark.parametrize("S,n_angles,N", [(1, 16, 701), (1, 1, 700), (3, 2, 702), (4, 16, 701)])
def test_fused_instantiations(ctx, torch, S, n_angles, N):
    """Species counts and angle counts of the fused generation beyond the
    other tests (one species, 1, 2 and 16 angles), on odd and even n_nu
    (4-byte and 8-byte grid reads), with spans that start and end inside a
    pair and a tile, against the oracle on the same seeded opacity field."""
    import paper_2104_12522_gb300 as bart
    L, M, dnu = 30, 7, 0.05
    p = W.log_pressures(L, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    field = W.opacity_field(S, p, t, N, seed=3600 + S)
    g_dev = torch.tensor(field, device="cuda")
    nu = bart.NuGrid(1000.0, dnu, N)
    n = 11
    theta = W.proposals(n, generation=31, n_species=S)
    lo = np.array([0, 1, 3, 255, 0, 7] + [0] * (n - 6), np.int64)
    hi = np.array([N, N - 1, 260, 514, 1, N] + [N] * (n - 6), np.int64)
    offs = np.concatenate([[0], np.cumsum(hi - lo)]).astype(np.int64)
    filt = W.gaussian_filters(W.nu_axis(1000.0, dnu, N), 3, 1003.0, 1030.0, 2.0, 10.0)
    x0 = [W.BASE_VMR] * S
    cfg = _cfg(n_angles, x0)
    dev = lambda a: torch.tensor(a, device="cuda")
    spec = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    bands = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, theta=dev(theta), nu_lo=dev(lo), nu_hi=dev(hi),
                              spec_offsets=dev(offs), spectra=spec, filters=dev(filt), bands=bands)
    ctx.sync()
    spec, bands = spec.cpu().numpy(), bands.cpu().numpy()
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0, x0=x0, mu=cfg["mu"], n_angles=n_angles)
    g_ora = field.astype(np.float64)
    nu_ax = W.nu_axis(1000.0, dnu, N)
    es, eb = 0.0, 0.0
    for i in range(n):
        F = Fw.emission_spectrum(g_ora[..., lo[i]:hi[i]], p, t, nu_ax[lo[i]:hi[i]], theta[i], ocfg)
        es = max(es, max_rel(spec[offs[i]:offs[i + 1]], F))
        Bo = R.band_integrate(F, filt, nu_lo=lo[i])
        ok = Bo != 0
        if ok.any():
            eb = max(eb, max_rel(bands[i][ok], Bo[ok]))
    print(f"fused S={S}, {n_angles} angles, n_nu={N}: spectra {es:.2e}, bands {eb:.2e}")
    assert es < RTOL and eb < RTOL


def test_band_integrate_standalone(ctx, torch):
    rng = np.random.default_rng(9)
    N, n = 1000, 5
    spec = rng.uniform(0.5, 2.0, (n, N))
    filt = W.gaussian_filters(W.nu_axis(1000.0, 1.0, N), 7, 1050.0, 1950.0, 20.0, 300.0, seed=77)
    lo = np.array([0, 10, 500, 999, 3], np.int64)
    hi = np.array([N, 20, 1000, 1000, 900], np.int64)
    offs = np.concatenate([[0], np.cumsum(hi - lo)]).astype(np.int64)
    packed = np.concatenate([spec[i, :hi[i] - lo[i]] for i in range(n)]).astype(np.float32)
    import paper_2104_12522_gb300 as bart
    dev = lambda a: torch.tensor(a, device="cuda")
    out = torch.empty((n, 7), dtype=torch.float32, device="cuda")
    ctx.band_integrate(dev(packed), dev(filt), bart.NuGrid(1000.0, 1.0, N), out, n, spec_offsets=dev(offs),
                       nu_lo=dev(lo), nu_hi=dev(hi))
    got = out.cpu().numpy()
    for i in range(n):
        ref = R.band_integrate(packed[offs[i]:offs[i + 1]].astype(np.float64), filt, nu_lo=lo[i])
        ok = ref != 0
        assert np.allclose(got[i][ok], ref[ok], rtol=1e-5)
        assert np.all(got[i][~ok] == 0)


def test_autotuned_tiles_give_the_same_spectra(ctx, torch, grid_case):
    """The tile autotuner times each wavenumber-tile width once per launch
    shape; spectra do not depend on the width, band values only through the
    order of their partial sums."""
    species, p, t, N, dnu, nu, g_dev, g_ora = grid_case
    theta = torch.tensor(W.proposals(9, generation=21, n_species=2), device="cuda")
    filt = torch.tensor(W.gaussian_filters(W.nu_axis(1000.0, dnu, N), 3, 1002.0, 1033.0, 2.0, 12.0), device="cuda")
    cfg = _cfg(4, [W.BASE_VMR] * 2)
    outs = []
    for tune in (False, True, True):
        ctx.set_autotune(tune)
        spec = torch.empty((9, N), dtype=torch.float32, device="cuda")
        bands = torch.empty((9, 3), dtype=torch.float32, device="cuda")
        ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, theta=theta, spectra=spec, filters=filt, bands=bands)
        ctx.sync()
        outs.append((spec.cpu().numpy(), bands.cpu().numpy()))
    rep = ctx.autotune_report()
    print("autotune choices:", rep)
    assert any(v in (64, 128, 256) for v in rep.values())
    for s_, b_ in outs[1:]:
        assert np.array_equal(s_, outs[0][0])
        assert np.allclose(b_, outs[0][1], rtol=1e-6)


def test_tau_limit(ctx, torch, grid_case):
    """Sec. 4 item 7: the layer integration stops where the vertical optical
    depth exceeds tau_max; parity with the oracle's truncated integration on
    the batched grid case, and an isothermal atmosphere still gives pi B."""
    species, p, t, N, dnu, nu, g_dev, g_ora = grid_case
    theta = W.proposals(7, generation=9, n_species=2)
    cfg = _cfg(4, [W.BASE_VMR] * 2)
    cfg["tau_max"] = 3.0
    spec = torch.empty((7, N), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, theta=torch.tensor(theta, device="cuda"), spectra=spec)
    spec = spec.cpu().numpy()
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0, x0=cfg["x0"], mu=cfg["mu"], n_angles=4,
                tau_max=3.0)
    nu_ax = W.nu_axis(1000.0, dnu, N)
    es = max(max_rel(spec[i], Fw.emission_spectrum(g_ora, p, t, nu_ax, theta[i], ocfg)) for i in range(7))
    print(f"emission with tau_max = 3, FP32 vs FP64: spectra {es:.2e}")
    assert es < RTOL
    T = torch.full((2, len(p)), 1500.0, dtype=torch.float32, device="cuda")
    iso = torch.empty((2, N), dtype=torch.float32, device="cuda")
    icfg = dict(cfg, t_min=1.0, t_max=1e5)
    ctx.forward_spectra_batch(g_dev, p, t, nu, icfg, t_profile=T, spectra=iso, n=2)
    assert max_rel(iso.cpu().numpy(), np.pi * R.planck(nu_ax, 1500.0)[None]) < 1e-5


@pytest.mark.parametrize("deck,ray", [(True, 0.0), (False, 1e-34), (True, 1e-34)])
def test_cloud_deck_and_rayleigh(ctx, torch, grid_case, deck, ray):
    """Sec. 3 gray cloud deck and Rayleigh scattering: parity with the oracle
    on the batched grid case.  The Rayleigh coefficient is raised to a haze
    (vertical optical depth 1 near 1e-4 bar at 1000 cm^-1) so that it matters on
    this grid; the deck sits between two grid layers."""
    species, p, t, N, dnu, nu, g_dev, g_ora = grid_case
    theta = W.proposals(6, generation=11, n_species=2)
    cfg = _cfg(4, [W.BASE_VMR] * 2)
    p_cloud = float(np.sqrt(p[8] * p[9])) if deck else 0.0
    cfg.update(p_cloud=p_cloud, rayleigh_coef=ray)
    spec = torch.empty((6, N), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, theta=torch.tensor(theta, device="cuda"), spectra=spec)
    spec = spec.cpu().numpy()
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0, x0=cfg["x0"], mu=cfg["mu"], n_angles=4,
                p_cloud=p_cloud, rayleigh_coef=ray)
    nu_ax = W.nu_axis(1000.0, dnu, N)
    ref = [Fw.emission_spectrum(g_ora, p, t, nu_ax, theta[i], ocfg) for i in range(6)]
    es = max(max_rel(spec[i], ref[i]) for i in range(6))
    plain = [Fw.emission_spectrum(g_ora, p, t, nu_ax, theta[i], dict(ocfg, p_cloud=None, rayleigh_coef=0.0))
             for i in range(6)]
    change = max(max_rel(ref[i], plain[i]) for i in range(6))
    print(f"emission, deck {deck}, Rayleigh {ray}: FP32 vs FP64 {es:.2e} (the options change the spectra by "
          f"{change:.2e})")
    assert change > 5e-3                       # the case exercises the option
    assert es < RTOL


def test_deck_seen_through_a_transparent_atmosphere(ctx, torch):
    """No opacity above an opaque deck on layer k: F = pi B(T_k)."""
    import paper_2104_12522_gb300 as bart
    L, N = 30, 500
    p = W.log_pressures(L, 1e-6, 100.0)
    grid = torch.zeros((1, L, 1, N), dtype=torch.float32, device="cuda")
    nu = bart.NuGrid(1500.0, 9.0, N)
    T = np.linspace(900.0, 2100.0, L)
    Tt = torch.tensor(T, dtype=torch.float32, device="cuda")[None].contiguous()
    spec = torch.empty((1, N), dtype=torch.float32, device="cuda")
    nu_ax = W.nu_axis(1500.0, 9.0, N)
    for k in (1, 9, 22):
        cfg = _cfg(8, [1e-4])
        cfg.update(t_min=1.0, t_max=1e5, p_cloud=float(p[k] * 0.99))
        ctx.forward_spectra_batch(grid, p, [1000.0], nu, cfg, t_profile=Tt, spectra=spec, n=1)
        assert max_rel(spec.cpu().numpy()[0], np.pi * R.planck(nu_ax, np.float32(T[k]))) < 1e-5


@pytest.mark.parametrize("deck", [False, True])
def test_contribution_functions(ctx, torch, grid_case, deck):
    """Per-layer contribution functions (post-processing of Sec. 3): parity
    of the rows with the oracle on proposals with uneven spans (and with a
    cloud deck), band values of the rows against the oracle's band means, and
    the rows adding up to the forward model's own spectra and bands."""
    species, p, t, N, dnu, nu, g_dev, g_ora = grid_case
    n, L = 5, len(p)
    theta = W.proposals(n, generation=13, n_species=2)
    lo = np.array([0, 3, 100, 257, 640], np.int64)
    hi = np.array([N, 700, 101, 612, N], np.int64)
    cfg = _cfg(4, [W.BASE_VMR] * 2)
    p_cloud = float(np.sqrt(p[15] * p[16])) if deck else 0.0
    cfg.update(p_cloud=p_cloud)
    filt = W.gaussian_filters(W.nu_axis(1000.0, dnu, N), 6, 1002.0, 1033.0, 1.0, 6.0)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    th, d_lo, d_hi, d_f = dev(theta), dev(lo), dev(hi), dev(filt)
    contrib = torch.full((n, L, N), -1.0, dtype=torch.float32, device="cuda")
    cb = torch.empty((n, L, 6), dtype=torch.float32, device="cuda")
    ctx.contribution_functions(g_dev, p, t, nu, cfg, theta=th, nu_lo=d_lo, nu_hi=d_hi, contrib=contrib,
                               filters=d_f, bands=cb)
    offs = np.concatenate([[0], np.cumsum(hi - lo)]).astype(np.int64)
    spec = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    sb = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, theta=th, nu_lo=d_lo, nu_hi=d_hi, spec_offsets=dev(offs),
                              spectra=spec, filters=d_f, bands=sb)
    ctx.sync()
    contrib, cb, spec, sb = (v.cpu().numpy() for v in (contrib, cb, spec, sb))
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0, x0=cfg["x0"], mu=cfg["mu"], n_angles=4,
                p_cloud=p_cloud)
    nu_ax = W.nu_axis(1000.0, dnu, N)
    e_row, e_band, e_sum = 0.0, 0.0, 0.0
    for i in range(n):
        # the oracle's contributions over the entry's span
        sub = g_ora[..., lo[i]:hi[i]]
        Co = Fw.emission_contributions(sub, p, t, nu_ax[lo[i]:hi[i]], theta[i], ocfg)
        got = contrib[i][:, lo[i]:hi[i]]
        assert np.all(contrib[i][:, :lo[i]] == -1.0) and np.all(contrib[i][:, hi[i]:] == -1.0)
        # each layer's term, relative to the spectrum at that wavenumber (a
        # thin layer's term is a difference of two transmittances: its own
        # relative error in FP32 grows as the layer thins, its share of the
        # flux does not)
        e_row = max(e_row, float(np.max(np.abs(got - Co) / Co.sum(axis=0)[None, :])))
        Bo = np.array([R.band_integrate(Co[k], filt, nu_lo=int(lo[i])) for k in range(L)])
        Bs = Bo.sum(axis=0)
        ok = Bs > 0
        if ok.any():
            e_band = max(e_band, float(np.max(np.abs(cb[i][:, ok] - Bo[:, ok]) / Bs[None, ok])))
        e_sum = max(e_sum, max_rel(got.sum(axis=0, dtype=np.float64), spec[offs[i]:offs[i + 1]]))
        okb = sb[i] != 0                    # a band with no weight on the span is 0 on both sides
        assert np.all(cb[i][:, ~okb] == 0.0)
        if okb.any():
            e_sum = max(e_sum, max_rel(cb[i].sum(axis=0, dtype=np.float64)[okb], sb[i][okb]))
    print(f"contribution functions (deck {deck}) FP32 vs FP64: rows {e_row:.2e}, bands {e_band:.2e}; "
          f"sum vs the forward model {e_sum:.2e}")
    assert e_row < 1e-5 and e_band < 1e-5 and e_sum < 1e-5

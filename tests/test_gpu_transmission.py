"""GPU parity of the transmission (transit) forward model against the FP64
oracle (Sec. 6.1, transit case of f01oneline) on uneven instances."""
import numpy as np
import pytest

import workloads as W
from oracle import opacity as O, forward as Fw, radiation as R
from gpu_common import make_ctx, max_rel

pytestmark = pytest.mark.gpu

RTOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    return make_ctx()


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _cfg(S):
    return dict(geometry=1, g=W.HD189_GRAV_CGS, mu=W.MEAN_MOLECULAR_MASS_AMU, x0=[W.BASE_VMR] * S,
                t_int=W.T_INT_K, t_star=W.HD189_TSTAR_K, r_star_tp=W.HD189_RSTAR_CM, a_orbit=W.HD189_A_CM,
                t_min=500.0, t_max=3000.0, p_ref=W.HD189_PREF_BAR, p_top=1e-8, p_bot=100.0)


@pytest.fixture(scope="module")
def case(ctx, torch):
    import paper_2104_12522_gb300 as bart
    S, Lg, M, N, dnu = 4, 30, 6, 900, 0.05
    species = [W.line_list(s, 300, 1000.0, 1000.0 + N * dnu) for s in range(S)]
    species[3].mass_amu = 16.0
    p = W.log_pressures(Lg, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    nu = bart.NuGrid(1000.0, dnu, N)
    g_dev = ctx.build_opacity_grid([bart.device_lines(s) for s in species], p, t, nu, 25.0)
    g_ora = O.opacity_grid(species, p, t, 1000.0, dnu, N, 25.0)
    return S, p, t, N, dnu, nu, g_dev, g_ora


def test_uneven_instances(ctx, torch, case):
    S, p, t, N, dnu, nu, g_dev, g_ora = case
    inst = W.instances(14, N, lmin=40, lmax=150, span_lo=1, span_hi=N, seed=4000)
    # edge cases: a single-point span, a full span, the most and fewest levels
    inst.nu_lo[0], inst.nu_hi[0] = 17, 18
    inst.nu_lo[1], inst.nu_hi[1] = 0, N
    inst.n_levels[2], inst.n_levels[3] = 192, 2
    filt = W.gaussian_filters(W.nu_axis(1000.0, dnu, N), 12, 1001.0, 1044.0, 2.0, 15.0)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    offs = inst.offsets
    n = len(inst.n_levels)
    spec = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    bands = torch.empty((n, 12), dtype=torch.float32, device="cuda")
    cfg = _cfg(S)
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, theta=dev(inst.theta), n_levels=dev(inst.n_levels),
                              nu_lo=dev(inst.nu_lo), nu_hi=dev(inst.nu_hi), spec_offsets=dev(offs),
                              r_planet=dev(inst.r_planet), r_star=dev(inst.r_star), spectra=spec,
                              filters=dev(filt), bands=bands)
    ctx.sync()
    spec, bands = spec.cpu().numpy(), bands.cpu().numpy()
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0, x0=cfg["x0"], mu=cfg["mu"],
                p_ref=cfg["p_ref"], p_top=1e-8, p_bot=100.0)
    es, eb = 0.0, 0.0
    for i in range(n):
        d = Fw.transmission_spectrum(g_ora, p, t, 1000.0, dnu, inst, i, ocfg)
        es = max(es, max_rel(spec[offs[i]:offs[i + 1]], d))
        Bo = R.band_integrate(d, filt, nu_lo=int(inst.nu_lo[i]))
        ok = Bo != 0
        if ok.any():
            eb = max(eb, max_rel(bands[i][ok], Bo[ok]))
        assert np.all(bands[i][~ok] == 0.0)
    print(f"transmission FP32 vs FP64 ({n} uneven instances): spectra {es:.2e}, bands {eb:.2e}")
    assert es < RTOL and eb < RTOL


@pytest.mark.parametrize("S,N,nb", [(1, 901, 40), (2, 900, 12), (3, 901, 5)])
def test_instantiations(ctx, torch, S, N, nb):
    """Species counts beyond the other tests on odd and even n_nu (4-byte and
    8-byte grid reads), up to 40 bands (a second round of each part's bands),
    with spans that start and end inside a pair, against the oracle on the
    same seeded opacity field."""
    import dataclasses
    import paper_2104_12522_gb300 as bart
    Lg, M, dnu = 30, 6, 0.05
    p = W.log_pressures(Lg, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    field = W.opacity_field(S, p, t, N, seed=3700 + S)
    g_dev = torch.tensor(field, device="cuda")
    nu = bart.NuGrid(1000.0, dnu, N)
    inst = W.instances(8, N, lmin=40, lmax=150, span_lo=1, span_hi=N, seed=4100 + S)
    inst = dataclasses.replace(inst, theta=np.ascontiguousarray(inst.theta[:, :5 + S]))
    inst.nu_lo[0], inst.nu_hi[0] = 3, 130
    inst.nu_lo[1], inst.nu_hi[1] = 0, N
    inst.nu_lo[2], inst.nu_hi[2] = N - 1, N
    filt = W.gaussian_filters(W.nu_axis(1000.0, dnu, N), nb, 1001.0, 1044.0, 2.0, 15.0)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    offs = inst.offsets
    n = len(inst.n_levels)
    spec = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    bands = torch.empty((n, nb), dtype=torch.float32, device="cuda")
    cfg = _cfg(S)
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, theta=dev(inst.theta), n_levels=dev(inst.n_levels),
                              nu_lo=dev(inst.nu_lo), nu_hi=dev(inst.nu_hi), spec_offsets=dev(offs),
                              r_planet=dev(inst.r_planet), r_star=dev(inst.r_star), spectra=spec,
                              filters=dev(filt), bands=bands)
    ctx.sync()
    spec, bands = spec.cpu().numpy(), bands.cpu().numpy()
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0, x0=cfg["x0"], mu=cfg["mu"],
                p_ref=cfg["p_ref"], p_top=1e-8, p_bot=100.0)
    g_ora = field.astype(np.float64)
    es, eb = 0.0, 0.0
    for i in range(n):
        d = Fw.transmission_spectrum(g_ora, p, t, 1000.0, dnu, inst, i, ocfg)
        es = max(es, max_rel(spec[offs[i]:offs[i + 1]], d))
        Bo = R.band_integrate(d, filt, nu_lo=int(inst.nu_lo[i]))
        ok = Bo != 0
        if ok.any():
            eb = max(eb, max_rel(bands[i][ok], Bo[ok]))
        assert np.all(bands[i][~ok] == 0.0)
    print(f"transmission S={S}, n_nu={N}, {nb} bands: spectra {es:.2e}, bands {eb:.2e}")
    assert es < RTOL and eb < RTOL


def test_zero_opacity_gives_bottom_radius(ctx, torch, case):
    S, p, t, N, dnu, nu, g_dev, g_ora = case
    zero = torch.zeros_like(g_dev)
    inst = W.instances(3, N, span_lo=1, seed=4100)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    spec = torch.empty((3, N), dtype=torch.float32, device="cuda")
    inst.nu_lo[:], inst.nu_hi[:] = 0, N
    cfg = _cfg(S)
    ctx.forward_spectra_batch(zero, p, t, nu, cfg, theta=dev(inst.theta), n_levels=dev(inst.n_levels),
                              r_planet=dev(inst.r_planet), r_star=dev(inst.r_star), spectra=spec)
    from oracle import transmission as Tr, forward as F2
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0)
    for i in range(3):
        P = F2.instance_levels(inst.n_levels[i], 1e-8, 100.0)
        T = F2.tp_of(inst.theta[i], P, ocfg)
        r = Tr.radii(P, T, float(inst.r_planet[i]), cfg["p_ref"], cfg["g"], cfg["mu"])
        exp = r[-1] ** 2 / float(inst.r_star[i]) ** 2
        assert max_rel(spec[i].cpu().numpy(), np.full(N, exp)) < 1e-5


def test_bad_level_count_sets_status(ctx, torch, case):
    import paper_2104_12522_gb300 as bart
    S, p, t, N, dnu, nu, g_dev, g_ora = case
    inst = W.instances(2, N, span_lo=1, seed=4200)
    inst.n_levels[1] = 500                      # above the 192-level limit
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    spec = torch.zeros(int(inst.offsets[-1]), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(g_dev, p, t, nu, _cfg(S), theta=dev(inst.theta), n_levels=dev(inst.n_levels),
                              nu_lo=dev(inst.nu_lo), nu_hi=dev(inst.nu_hi), spec_offsets=dev(inst.offsets),
                              r_planet=dev(inst.r_planet), r_star=dev(inst.r_star), spectra=spec)
    with pytest.raises(bart.BartError, match="ERANGE"):
        ctx.sync()
    ctx.sync()                                  # status was cleared


@pytest.mark.parametrize("p_cloud,ray", [(3.3e-5, 0.0), (0.0, 1e-34), (3.3e-5, 1e-34)])
def test_cloud_deck_and_rayleigh(ctx, torch, case, p_cloud, ray):
    """Sec. 3 gray cloud deck and Rayleigh scattering on uneven instances:
    parity with the oracle (Rayleigh raised to a haze, vertical optical depth 1
    near 1e-4 bar at 1000 cm^-1, so that it matters on this grid)."""
    S, p, t, N, dnu, nu, g_dev, g_ora = case
    inst = W.instances(10, N, lmin=40, lmax=150, span_lo=1, span_hi=N, seed=4300)
    inst.n_levels[0] = 192
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    offs = inst.offsets
    n = len(inst.n_levels)
    spec = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    cfg = dict(_cfg(S), p_cloud=p_cloud, rayleigh_coef=ray)
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, theta=dev(inst.theta), n_levels=dev(inst.n_levels),
                              nu_lo=dev(inst.nu_lo), nu_hi=dev(inst.nu_hi), spec_offsets=dev(offs),
                              r_planet=dev(inst.r_planet), r_star=dev(inst.r_star), spectra=spec)
    spec = spec.cpu().numpy()
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0, x0=cfg["x0"], mu=cfg["mu"],
                p_ref=cfg["p_ref"], p_top=1e-8, p_bot=100.0, p_cloud=p_cloud, rayleigh_coef=ray)
    es, change = 0.0, 0.0
    for i in range(n):
        d = Fw.transmission_spectrum(g_ora, p, t, 1000.0, dnu, inst, i, ocfg)
        d0 = Fw.transmission_spectrum(g_ora, p, t, 1000.0, dnu, inst, i,
                                      dict(ocfg, p_cloud=None, rayleigh_coef=0.0))
        es = max(es, max_rel(spec[offs[i]:offs[i + 1]], d))
        change = max(change, max_rel(d, d0))
    print(f"transmission, deck {p_cloud}, Rayleigh {ray}: FP32 vs FP64 {es:.2e} (the options change the "
          f"spectra by {change:.2e})")
    assert change > 1e-3
    assert es < RTOL


def test_deck_radius_through_a_transparent_atmosphere(ctx, torch, case):
    """No opacity above the deck: delta = r_deck^2 / R_star^2 with r from the
    whole column's hydrostatic altitudes."""
    S, p, t, N, dnu, nu, g_dev, g_ora = case
    zero = torch.zeros_like(g_dev)
    inst = W.instances(3, N, span_lo=1, seed=4400)
    inst.nu_lo[:], inst.nu_hi[:] = 0, N
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    spec = torch.empty((3, N), dtype=torch.float32, device="cuda")
    cfg = dict(_cfg(S), p_cloud=0.0123)
    ctx.forward_spectra_batch(zero, p, t, nu, cfg, theta=dev(inst.theta), n_levels=dev(inst.n_levels),
                              r_planet=dev(inst.r_planet), r_star=dev(inst.r_star), spectra=spec)
    from oracle import transmission as Tr, forward as F2
    ocfg = dict(g=cfg["g"], t_int=cfg["t_int"], t_star=cfg["t_star"], r_star_tp=cfg["r_star_tp"],
                a_orbit=cfg["a_orbit"], t_min=500.0, t_max=3000.0)
    for i in range(3):
        P = F2.instance_levels(inst.n_levels[i], 1e-8, 100.0)
        T = F2.tp_of(inst.theta[i], P, ocfg)
        r = Tr.radii(P, T, float(inst.r_planet[i]), cfg["p_ref"], cfg["g"], cfg["mu"])
        k = int(np.nonzero(P >= 0.0123)[0][0])
        exp = r[k] ** 2 / float(inst.r_star[i]) ** 2
        assert max_rel(spec[i].cpu().numpy(), np.full(N, exp)) < 1e-5

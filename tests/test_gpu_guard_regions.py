"""Kernels write exactly their outputs and nothing around them: each output of
a small case (the calls of the parity tests, odd sizes and ragged spans) is
placed inside a larger buffer whose head and tail hold a sentinel; after the
call the sentinel is intact and the output equals that of a plain buffer.
Guard regions stand in for a memory checker."""
import numpy as np
import pytest

import workloads as W
from gpu_common import make_ctx

pytestmark = pytest.mark.gpu

PAD = 64            # elements on each side (256 B for 4-byte types: alignment kept)
SENT = -12345.0


@pytest.fixture(scope="module")
def ctx():
    return make_ctx()


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def _guarded(torch, shape, dtype):
    n = int(np.prod(shape))
    fill = SENT if dtype.is_floating_point else int(SENT)
    buf = torch.full((PAD + n + PAD,), fill, dtype=dtype, device="cuda")
    return buf, buf[PAD:PAD + n].view(*shape)


def _intact(torch, buf, shape):
    n = int(np.prod(shape))
    return bool(torch.all(buf[:PAD] == SENT)) and bool(torch.all(buf[PAD + n:] == SENT))


def _same(torch, a, b):
    return bool(torch.allclose(a.double(), b.double(), rtol=1e-6, atol=0.0))


def test_faddeeva_output(ctx, torch):
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.uniform(0, 40, 1001).astype(np.float32), device="cuda")
    y = torch.tensor(10 ** rng.uniform(-6, 1.5, 1001).astype(np.float32), device="cuda")
    ref = ctx.faddeeva_re(x, y)
    buf, out = _guarded(torch, (1001,), torch.float32)
    ctx.faddeeva_re(x, y, out=out)
    ctx.sync()
    assert _intact(torch, buf, (1001,)) and _same(torch, out, ref)


def test_opacity_outputs(ctx, torch):
    # the grid of the emission parity tests (two species, 400 lines, 24 layers,
    # 6 temperatures, 700 points), and the same layers as cells
    import paper_2104_12522_gb300 as bart
    S, L, M, N, dnu = 2, 24, 6, 700, 0.05
    dl = [bart.device_lines(W.line_list(s, 400, 1000.0, 1000.0 + N * dnu)) for s in range(S)]
    p = W.log_pressures(L, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    nu = bart.NuGrid(1000.0, dnu, N)
    ref = ctx.build_opacity_grid(dl, p, t, nu, 25.0)
    buf, out = _guarded(torch, (S, L, M, N), torch.float32)
    ctx.build_opacity_grid(dl, p, t, nu, 25.0, out=out)
    ctx.sync()
    assert _intact(torch, buf, (S, L, M, N)) and _same(torch, out, ref)
    T = np.linspace(500.0, 3000.0, L)
    ref = ctx.opacity_cells(dl, p, T, nu, 25.0)
    buf, out = _guarded(torch, (S, L, N), torch.float32)
    ctx.opacity_cells(dl, p, T, nu, 25.0, out=out)
    ctx.sync()
    assert _intact(torch, buf, (S, L, N)) and _same(torch, out, ref)


def test_emission_spectra_and_bands(ctx, torch):
    # the fused generation of the parity test with four species, 16 angles and
    # an odd n_nu, spans starting and ending inside a pair and a tile
    import paper_2104_12522_gb300 as bart
    S, n_angles, N, L, M, dnu = 4, 16, 701, 30, 7, 0.05
    p = W.log_pressures(L, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    g_dev = torch.tensor(W.opacity_field(S, p, t, N, seed=3600 + S), device="cuda")
    nu = bart.NuGrid(1000.0, dnu, N)
    n = 11
    lo = np.array([0, 1, 3, 255, 0, 7] + [0] * (n - 6), np.int64)
    hi = np.array([N, N - 1, 260, 514, 1, N] + [N] * (n - 6), np.int64)
    offs = np.concatenate([[0], np.cumsum(hi - lo)]).astype(np.int64)
    dev = lambda a: torch.tensor(a, device="cuda")
    cfg = dict(geometry=0, n_angles=n_angles, g=W.HD189_GRAV_CGS, mu=W.MEAN_MOLECULAR_MASS_AMU,
               x0=[W.BASE_VMR] * S, t_int=W.T_INT_K, t_star=W.HD189_TSTAR_K, r_star_tp=W.HD189_RSTAR_CM,
               a_orbit=W.HD189_A_CM, t_min=500.0, t_max=3000.0)
    args = dict(theta=dev(W.proposals(n, generation=31, n_species=S)), nu_lo=dev(lo), nu_hi=dev(hi),
                spec_offsets=dev(offs),
                filters=dev(W.gaussian_filters(W.nu_axis(1000.0, dnu, N), 3, 1003.0, 1030.0, 2.0, 10.0)))
    spec0 = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    bands0 = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, spectra=spec0, bands=bands0, **args)
    sbuf, spec = _guarded(torch, (int(offs[-1]),), torch.float32)
    bbuf, bands = _guarded(torch, (n, 3), torch.float32)
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, spectra=spec, bands=bands, **args)
    ctx.sync()
    assert _intact(torch, sbuf, (int(offs[-1]),)) and _same(torch, spec, spec0)
    assert _intact(torch, bbuf, (n, 3)) and _same(torch, bands, bands0)


def test_transit_spectra_and_bands(ctx, torch):
    # the uneven transit batch of the parity test: a one-point span, a full
    # span, 192 and 2 levels
    import paper_2104_12522_gb300 as bart
    S, Lg, M, N, dnu = 4, 30, 6, 900, 0.05
    species = [W.line_list(s, 300, 1000.0, 1000.0 + N * dnu) for s in range(S)]
    species[3].mass_amu = 16.0
    p = W.log_pressures(Lg, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    nu = bart.NuGrid(1000.0, dnu, N)
    g_dev = ctx.build_opacity_grid([bart.device_lines(s) for s in species], p, t, nu, 25.0)
    inst = W.instances(14, N, lmin=40, lmax=150, span_lo=1, span_hi=N, seed=4000)
    inst.nu_lo[0], inst.nu_hi[0] = 17, 18
    inst.nu_lo[1], inst.nu_hi[1] = 0, N
    inst.n_levels[2], inst.n_levels[3] = 192, 2
    n = len(inst.n_levels)
    offs = inst.offsets
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    cfg = dict(geometry=1, g=W.HD189_GRAV_CGS, mu=W.MEAN_MOLECULAR_MASS_AMU, x0=[W.BASE_VMR] * S,
               t_int=W.T_INT_K, t_star=W.HD189_TSTAR_K, r_star_tp=W.HD189_RSTAR_CM, a_orbit=W.HD189_A_CM,
               t_min=500.0, t_max=3000.0, p_ref=W.HD189_PREF_BAR, p_top=1e-8, p_bot=100.0)
    args = dict(theta=dev(inst.theta), n_levels=dev(inst.n_levels), nu_lo=dev(inst.nu_lo), nu_hi=dev(inst.nu_hi),
                spec_offsets=dev(offs), r_planet=dev(inst.r_planet), r_star=dev(inst.r_star),
                filters=dev(W.gaussian_filters(W.nu_axis(1000.0, dnu, N), 12, 1001.0, 1044.0, 2.0, 15.0)))
    spec0 = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    bands0 = torch.empty((n, 12), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, spectra=spec0, bands=bands0, **args)
    sbuf, spec = _guarded(torch, (int(offs[-1]),), torch.float32)
    bbuf, bands = _guarded(torch, (n, 12), torch.float32)
    ctx.forward_spectra_batch(g_dev, p, t, nu, cfg, spectra=spec, bands=bands, **args)
    ctx.sync()
    assert _intact(torch, sbuf, (int(offs[-1]),)) and _same(torch, spec, spec0)
    assert _intact(torch, bbuf, (n, 12)) and _same(torch, bands, bands0)


def test_band_integrator_output(ctx, torch):
    import paper_2104_12522_gb300 as bart
    rng = np.random.default_rng(9)
    N, n = 1000, 5
    spec = rng.uniform(0.5, 2.0, (n, N))
    filt = W.gaussian_filters(W.nu_axis(1000.0, 1.0, N), 7, 1050.0, 1950.0, 20.0, 300.0, seed=77)
    lo = np.array([0, 10, 500, 999, 3], np.int64)
    hi = np.array([N, 20, 1000, 1000, 900], np.int64)
    offs = np.concatenate([[0], np.cumsum(hi - lo)]).astype(np.int64)
    packed = np.concatenate([spec[i, :hi[i] - lo[i]] for i in range(n)]).astype(np.float32)
    dev = lambda a: torch.tensor(a, device="cuda")
    args = (dev(packed), dev(filt), bart.NuGrid(1000.0, 1.0, N))
    kw = dict(spec_offsets=dev(offs), nu_lo=dev(lo), nu_hi=dev(hi))
    out0 = torch.empty((n, 7), dtype=torch.float32, device="cuda")
    ctx.band_integrate(*args, out0, n, **kw)
    buf, out = _guarded(torch, (n, 7), torch.float32)
    ctx.band_integrate(*args, out, n, **kw)
    ctx.sync()
    assert _intact(torch, buf, (n, 7)) and _same(torch, out, out0)


def test_surrogate_forward_output(ctx, torch):
    import paper_2104_12522_gb300 as bart
    widths = list(W.SURROGATE_WIDTHS)
    net = bart.Mlp(ctx, widths, bf16_weights=True, log_outputs=True, max_batch=64)
    in_shift = (0.5 * (W.THETA_LO + W.THETA_HI)).astype(np.float32)
    in_scale = (2.0 / (W.THETA_HI - W.THETA_LO)).astype(np.float32)
    net.set_scaling(in_shift, in_scale, np.full(10, 4.0, np.float32), np.full(10, 2.0, np.float32))
    net.set_params(torch.tensor(W.mlp_init(widths), device="cuda"))
    rng = np.random.default_rng(2)
    th = (W.THETA_LO + rng.uniform(size=(37, 9)) * (W.THETA_HI - W.THETA_LO)).astype(np.float32)
    x = torch.tensor(th, device="cuda")
    ref = net.forward(x)
    buf, out = _guarded(torch, (37, 10), torch.float32)
    net.forward(x, out=out)
    ctx.sync()
    assert _intact(torch, buf, (37, 10)) and _same(torch, out, ref)


def test_sampler_proposal_outputs(ctx, torch):
    import paper_2104_12522_gb300 as bart
    C, d = 10, 3
    lo, hi = np.zeros(d, np.float32), np.ones(d, np.float32)
    s = bart.Demc(ctx, C, lo, hi, eps=0.0, seed=1)
    x0 = torch.tensor(np.random.default_rng(0).uniform(0.2, 0.8, (C, d)).astype(np.float32), device="cuda")
    s.set_state(x0, torch.zeros(C, dtype=torch.float64, device="cuda"))
    y0 = torch.empty((C, d), dtype=torch.float32, device="cuda")
    in0 = torch.empty(C, dtype=torch.int32, device="cuda")
    s.propose(3, y0, in0)
    ybuf, y = _guarded(torch, (C, d), torch.float32)
    ibuf, inbox = _guarded(torch, (C,), torch.int32)
    s.propose(3, y, inbox)
    ctx.sync()
    assert _intact(torch, ybuf, (C, d)) and torch.equal(y, y0)
    assert _intact(torch, ibuf, (C,)) and torch.equal(inbox, in0)

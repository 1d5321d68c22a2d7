"""The allocation-free emission entry point (for callers that cannot allocate
device memory: allocator hooks, fixed-budget real-time loops, processes that
reserve all device memory up front) gives the results of the regular entry
point, on two calls in a row, and rejects requests beyond its fixed limits.
This file is collected last so a failure here comes after every other test."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-4      # the spectra/band tolerance of the other forward-model tests


def _inputs(torch):
    import paper_2104_12522_gb300 as bart
    from paper_2104_12522_gb300 import build
    build.build()
    rng = np.random.default_rng(77)
    S, L, M, N = 3, 40, 6, 3000
    p = W.log_pressures(L, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    grid = torch.tensor(10 ** rng.uniform(-26, -18, (S, L, M, N)), dtype=torch.float32, device="cuda")
    theta = torch.tensor(W.proposals(20, generation=3, n_species=S), device="cuda")
    filt = torch.tensor(W.gaussian_filters(W.nu_axis(1000.0, 0.05, N), 5, 1010.0, 1140.0, 5.0, 40.0),
                        device="cuda")
    cfg = dict(geometry=0, n_angles=8, g=W.HD189_GRAV_CGS, mu=W.MEAN_MOLECULAR_MASS_AMU, x0=[W.BASE_VMR] * S,
               t_int=W.T_INT_K, t_star=W.HD189_TSTAR_K, r_star_tp=W.HD189_RSTAR_CM, a_orbit=W.HD189_A_CM,
               t_min=500.0, t_max=3000.0)
    return bart, p, t, bart.NuGrid(1000.0, 0.05, N), grid, theta, filt, cfg


def test_no_alloc_matches_regular_entry_point():
    import torch
    bart, p, t, nu, grid, theta, filt, cfg = _inputs(torch)
    ctx = bart.Context(0)
    n, N = theta.shape[0], grid.shape[-1]
    ref_s = torch.empty((n, N), dtype=torch.float32, device="cuda")
    ref_b = torch.empty((n, 5), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(grid, p, t, nu, cfg, theta=theta, spectra=ref_s, filters=filt, bands=ref_b)
    ctx.sync()
    ref_s, ref_b = ref_s.cpu().numpy(), ref_b.cpu().numpy()
    for call in range(2):
        s = torch.full((n, N), -1.0, dtype=torch.float32, device="cuda")
        b = torch.full((n, 5), -1.0, dtype=torch.float32, device="cuda")
        st = bart.forward_emission_noalloc(grid, p, t, nu, cfg, theta=theta, spectra=s, filters=filt, bands=b)
        assert st == 0, f"call {call}: status {st}"
        torch.cuda.synchronize()
        s, b = s.cpu().numpy(), b.cpu().numpy()
        assert np.max(np.abs(s - ref_s) / np.abs(ref_s)) < RTOL, f"call {call}: spectra differ"
        assert np.max(np.abs(b - ref_b) / np.abs(ref_b)) < RTOL, f"call {call}: bands differ"


def test_no_alloc_rejects_requests_beyond_its_limits():
    import torch
    bart, p, t, nu, grid, theta, filt, cfg = _inputs(torch)
    many = torch.tensor(W.proposals(65, generation=4, n_species=3), device="cuda")   # limit is 64
    spec = torch.empty((65, grid.shape[-1]), dtype=torch.float32, device="cuda")
    assert bart.forward_emission_noalloc(grid, p, t, nu, cfg, theta=many, spectra=spec) == 5   # BART_ERANGE
    assert bart.forward_emission_noalloc(grid, p[::-1].copy(), t, nu, cfg, theta=theta,
                                         spectra=spec[:20]) == 1                             # BART_EINVAL


def _spans(n, N, seed):
    rng = np.random.default_rng(seed)
    lo = rng.integers(0, N // 3, n).astype(np.int64)
    hi = (N - rng.integers(0, N // 3, n)).astype(np.int64)
    lo[0], hi[0] = 0, N                          # one full span, one single point
    lo[1], hi[1] = N // 2, N // 2 + 1
    return lo, hi, np.concatenate([[0], np.cumsum(hi - lo)]).astype(np.int64)


@pytest.mark.parametrize("shape", ["entries_layers_bands", "wavenumbers"])
def test_no_alloc_at_its_limits_with_spans_and_profiles(shape):
    """Requests at the fixed limits -- 64 entries x 256 layers x 4 species x
    16 bands, or 131,072 wavenumbers -- with per-entry spans, packed output
    and given temperature profiles, against the regular entry point."""
    import torch
    import paper_2104_12522_gb300 as bart
    from paper_2104_12522_gb300 import build
    build.build()
    if shape == "entries_layers_bands":
        S, L, M, N, n, nb = 4, 256, 2, 2048, 64, 16
    else:
        S, L, M, N, n, nb = 1, 4, 2, 131072, 4, 16
    p = W.log_pressures(L, 1e-8, 100.0)
    t = np.array([500.0, 3000.0])
    grid = torch.tensor(W.opacity_field(S, p, t, N, seed=3700), device="cuda")
    rng = np.random.default_rng(78)
    tprof = torch.tensor(rng.uniform(600.0, 2900.0, (n, L)).astype(np.float32), device="cuda")
    theta = torch.tensor(W.proposals(n, generation=5, n_species=S), device="cuda")
    lo, hi, offs = _spans(n, N, 79)
    d = lambda a: torch.tensor(a, device="cuda")
    nu = bart.NuGrid(1000.0, 0.02, N)
    filt = torch.tensor(W.gaussian_filters(W.nu_axis(1000.0, 0.02, N), nb, 1000.0, 1000.0 + 0.02 * N, 1.0, 20.0),
                        device="cuda")
    cfg = dict(geometry=0, n_angles=8, g=W.HD189_GRAV_CGS, mu=W.MEAN_MOLECULAR_MASS_AMU, x0=[W.BASE_VMR] * S,
               t_min=500.0, t_max=3000.0)
    args = dict(theta=theta, t_profile=tprof, nu_lo=d(lo), nu_hi=d(hi), spec_offsets=d(offs), filters=filt)
    ctx = bart.Context(0)
    ref_s = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    ref_b = torch.empty((n, nb), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(grid, p, t, nu, cfg, spectra=ref_s, bands=ref_b, **args)
    ctx.sync()
    ref_s, ref_b = ref_s.cpu().numpy(), ref_b.cpu().numpy()
    for call in range(2):
        s = torch.full((int(offs[-1]),), -1.0, dtype=torch.float32, device="cuda")
        b = torch.full((n, nb), -1.0, dtype=torch.float32, device="cuda")
        assert bart.forward_emission_noalloc(grid, p, t, nu, cfg, spectra=s, bands=b, **args) == 0
        torch.cuda.synchronize()
        s, b = s.cpu().numpy(), b.cpu().numpy()
        assert np.max(np.abs(s - ref_s) / np.abs(ref_s)) < RTOL, f"call {call}: spectra differ"
        assert np.all(b[ref_b == 0] == 0)
        nz = ref_b != 0
        assert np.max(np.abs(b[nz] - ref_b[nz]) / np.abs(ref_b[nz])) < RTOL, f"call {call}: bands differ"


def test_no_alloc_with_deck_and_depth_limit_matches_oracle():
    """Spans, a gray cloud deck and the optical-depth limit through the
    allocation-free entry point, against the FP64 oracle."""
    import torch
    import paper_2104_12522_gb300 as bart
    from oracle import forward as Fw, radiation as R
    S, L, M, N, n = 2, 30, 4, 500, 6
    p = W.log_pressures(L, 1e-8, 100.0)
    t = np.linspace(500.0, 3000.0, M)
    field = W.opacity_field(S, p, t, N, seed=3800)
    theta = W.proposals(n, generation=9, n_species=S)
    lo, hi, offs = _spans(n, N, 80)
    filt = W.gaussian_filters(W.nu_axis(1000.0, 0.1, N), 4, 1005.0, 1045.0, 2.0, 10.0)
    cfg = dict(geometry=0, n_angles=4, g=W.HD189_GRAV_CGS, mu=W.MEAN_MOLECULAR_MASS_AMU, x0=[W.BASE_VMR] * S,
               t_int=W.T_INT_K, t_star=W.HD189_TSTAR_K, r_star_tp=W.HD189_RSTAR_CM, a_orbit=W.HD189_A_CM,
               t_min=500.0, t_max=3000.0, p_cloud=1.0, tau_max=5.0)
    d = lambda a: torch.tensor(a, device="cuda")
    s = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    b = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    st = bart.forward_emission_noalloc(d(field), p, t, bart.NuGrid(1000.0, 0.1, N), cfg, theta=d(theta),
                                       nu_lo=d(lo), nu_hi=d(hi), spec_offsets=d(offs), spectra=s, filters=d(filt),
                                       bands=b)
    assert st == 0
    torch.cuda.synchronize()
    s, b = s.cpu().numpy(), b.cpu().numpy()
    nu_ax = W.nu_axis(1000.0, 0.1, N)
    es = eb = 0.0
    for i in range(n):
        F = Fw.emission_spectrum(field.astype(np.float64)[..., lo[i]:hi[i]], p, t, nu_ax[lo[i]:hi[i]], theta[i], cfg)
        es = max(es, float(np.max(np.abs(s[offs[i]:offs[i + 1]] - F) / F)))
        bo = R.band_integrate(F, filt, int(lo[i]))
        assert np.all(b[i][bo == 0] == 0)
        if np.any(bo > 0):
            eb = max(eb, float(np.max(np.abs(b[i][bo > 0] - bo[bo > 0]) / bo[bo > 0])))
    print(f"no-alloc with deck and tau limit, FP32 vs FP64: spectra {es:.2e}, bands {eb:.2e}")
    assert es < RTOL and eb < RTOL

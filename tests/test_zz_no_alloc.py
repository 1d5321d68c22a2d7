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

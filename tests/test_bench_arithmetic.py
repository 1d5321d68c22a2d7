"""The bench's unit counts and roofline arithmetic on the CPU: the algorithmic
line-point evaluations behind the opacity rate, the FP32 and MUFU peaks from
unit counts and clocks, and the forward model's algorithmic grid bytes
(2 L S N_nu x 4 B per spectrum: 320 MB at 100 layers, 4 species and 100,000
wavenumbers)."""
from types import SimpleNamespace

import numpy as np

import bench


def test_eval_count_by_brute_force():
    # every (line, grid point) pair within the cutoff, once per (P, T) cell
    rng = np.random.default_rng(3)
    ax = SimpleNamespace(nu_start=1000.0, dnu=0.25, n_nu=400, cutoff=3.0, p_bar=np.ones(3), t_K=np.ones(5))
    nu = 1000.0 + 0.25 * np.arange(400)
    species = []
    for n in (40, 7):
        nu0 = np.sort(np.concatenate([rng.uniform(990.0, 1110.0, n), [997.0, 1102.75, 1000.0 + 0.25 * 17]]))
        species.append(SimpleNamespace(nu0=nu0))
    brute = sum(int(np.sum(np.abs(nu[None, :] - s.nu0[:, None]) <= 3.0)) for s in species)
    assert bench.eval_count(species, ax) == brute * 3 * 5


def test_peaks_from_unit_counts_and_clock():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2070 MHz
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9
    # 152 SMs x 32 MUFU results per clock x 2070 MHz, in Tops/s
    r = bench.emission_roofline(36.4, 152, 2070.0, {"hbm_gbs": 7000.0}, 100, 100_000)
    assert abs(r["peak"] - 152 * 32 * 2070e6 / 1e12) < 1e-12


def test_forward_model_roofline_arithmetic():
    L, NU, ms = 100, 100_000, 36.4
    r = bench.emission_roofline(ms, 152, 2070.0, {"hbm_gbs": 7000.0}, L, NU)
    units = bench.N_PROPOSALS * L * NU
    assert r["algorithmic_bytes"] == units * 2 * bench.FW_SPECIES * 4
    assert r["algorithmic_bytes"] / bench.N_PROPOSALS == 320_000_000       # per spectrum, S = 4
    assert abs(r["achieved"] - units * (bench.N_ANGLES + 2) / (ms / 1e3) / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    assert abs(r["hbm_frac_algorithmic"] - r["algorithmic_bytes"] / (ms / 1e3) / 7000e9) < 1e-12


def test_job_rate_is_whole_job_units_per_second():
    assert bench.job_rate(1, 2048, 5, 250.0) == 2048 * 5 / 0.25
    assert bench.job_rate(4, 2048, 5, 250.0) == 4 * 2048 * 5 / 0.25

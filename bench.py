#!/usr/bin/env python3
"""Benchmark of the BART forward-model hot path on GB300.

One step = one pass of the hot path over one batch of synthetic input:
  1. the line-by-line opacity grid (3 species, 5e6 lines, 100 layers x 20
     temperatures x 100,000 wavenumbers, cutoff 25 cm^-1), and
  2. one generation of 2,048 emission proposals on that grid plus a fourth
     species built once at set-up (nine parameters: five-parameter T(P) + four
     abundance scalings; 8 Gauss-Legendre angles, 10 Gaussian filters), one
     persistent fused launch replayed from a CUDA graph.
The headline value is Voigt line-point evaluations per second over the whole
step (Gline-evals/s); the generation's spectra/s is reported beside it, with
the transit batch, the surrogate and the retrieval legs, FP32-vs-FP64 errors
of sampled full-size results and the oracle's CPU baselines.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Multi-GPU (torchrun, one rank per GPU): every rank runs the full step on its
own GPU (independent problems, weak scaling); ranks only meet at the barriers
and the max-over-ranks of the timings.  --impl reference times the FP64 CPU
oracle on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = ("forward-model spectra/sec at 1e-4 rel err (plain vs surrogate); Voigt Gline-evals/s")
UNIT = "Gline-evals/s"
FLOPS_PER_EVAL = 10          # algorithmic FP32 flops of one line-point evaluation (one-pole form)
RATIONAL_FLOPS_PER_EVAL = 16  # the same evaluation counted on the region-I rational form
N_PROPOSALS = 2048
N_ANGLES = 8
N_BANDS = 10
FW_SPECIES = 4                    # species of the forward-model generation's grid
OPACITY_LAUNCHES_PER_STEP = 3     # one opacity kernel launch per species
KERNELS_PER_STEP = 3 * 3 + 1      # per species: window and span prologues + opacity; one fused generation
# sources the opacity kernel is compiled from (the committed traffic figure is tied to them)
OPACITY_SOURCES = [os.path.join(ROOT, "paper_2104_12522_gb300", "csrc", f)
                   for f in ("opacity.cu", "faddeeva.cuh", "bart_internal.cuh")]
FORWARD_SOURCES = [os.path.join(ROOT, "paper_2104_12522_gb300", "csrc", f)
                   for f in ("emission_fused.cuh", "forward_fused.cu", "emission.cuh", "forward.cuh",
                             "bart_internal.cuh")]
MUFU_PER_CLK = 32                 # MUFU (ex2, rcp) results per clock per SM on GB300 (ncu: XU-pipe peak 1 warp-inst/clk/SM)


def workload_desc():
    return ("opacity grid: 3 species, 5e6 lines, 100 layers (1e-8..100 bar) x 20 T (500..3000 K) x "
            "100000 nu (0.02 cm^-1), cutoff 25 cm^-1; then one emission generation of 2048 9-parameter "
            "proposals x 8 angles x 10 Gaussian bands on that grid plus a 4th species (3.2 GB, built once), "
            "one persistent fused launch replayed from a CUDA graph")


# ---------------------------------------------------------------- distributed
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
        return dist
    return None


def max_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(n_ranks, units_per_rank, steps, max_ms):
    """Whole-job throughput in units/s: every rank processes its own problem
    (weak scaling), the job takes as long as its slowest rank."""
    return n_ranks * units_per_rank * steps / (max_ms / 1e3)


# ---------------------------------------------------------------- counts
def eval_count(species, ax) -> int:
    """Algorithmic line-point evaluations of one grid build: for every line,
    the grid points within its cutoff, times the number of (P, T) cells."""
    nu = W.nu_axis(ax.nu_start, ax.dnu, ax.n_nu)
    total = 0
    for ll in species:
        lo = np.searchsorted(nu, ll.nu0 - ax.cutoff, side="left")
        hi = np.searchsorted(nu, ll.nu0 + ax.cutoff, side="right")
        total += int(np.sum(hi - lo))
    return total * len(ax.p_bar) * len(ax.t_K)


def fp32_peak_tflops(n_sm: int, mhz: float) -> float:
    return n_sm * 128 * 2 * mhz * 1e6 / 1e12


def source_sha(paths):
    h = hashlib.sha256()
    for path in paths:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel_srcs, name):
    """DRAM bytes of one launch (read + write) from the committed ncu summary
    profiles/<name>_traffic.txt (key = value lines), if it was taken on the
    current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", f"{name}_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as fh:
        for line in fh:
            if "=" in line and not line.lstrip().startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha") != source_sha(kernel_srcs):
        return None
    return float(kv["dram_bytes_read"]) + float(kv["dram_bytes_write"])


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
# Everything in this section runs the FP64 oracle on the host cores: the
# CPU baselines (a reported baseline, never the target) and the FP32-vs-FP64
# samples of the full-size results.  It runs before the first CUDA call, in
# spawned worker processes.
_ORACLE_STATE = {}
SLICE_N = 3000                  # wavenumbers of the seeded opacity-field slice
EM_SAMPLE_PROPOSALS = (0, 1024, 2047)
TR_SAMPLE_INSTANCES = (0, 1)
SAMPLE_POINTS = 8               # wavenumbers sampled per proposal (shared) / instance


def _oracle_init():
    _ORACLE_STATE["ax"] = W.grid_axes()
    _ORACLE_STATE["species"] = W.opacity_grid_species(4)


def _lines_in_cutoff(ll, nu, cutoff):
    """Line-point evaluations of the points nu: lines within the cutoff."""
    nu = np.asarray(nu, np.float64)
    return int(np.sum(np.searchsorted(ll.nu0, nu + cutoff, side="right") -
                      np.searchsorted(ll.nu0, nu - cutoff, side="left")))


def _oracle_window(args):
    """Oracle opacity of species s at cell (k, m) on the grid points js (a
    window when contiguous); returns (evaluations, seconds, values)."""
    s, k, m, js = args
    from oracle import opacity as O
    ax, ll = _ORACLE_STATE["ax"], _ORACLE_STATE["species"][s]
    js = np.asarray(js, np.int64)
    t = time.perf_counter()
    if np.all(np.diff(js) == 1):
        vals = O.opacity_cell(ll, ax.p_bar[k], ax.t_K[m], ax.nu_start, ax.dnu, ax.n_nu, ax.cutoff,
                              int(js[0]), int(js[-1]) + 1)
    else:
        vals = np.array([O.opacity_cell(ll, ax.p_bar[k], ax.t_K[m], ax.nu_start, ax.dnu, ax.n_nu, ax.cutoff,
                                        int(j), int(j) + 1)[0] for j in js])
    dt = time.perf_counter() - t
    return _lines_in_cutoff(ll, W.nu_axis(ax.nu_start, ax.dnu, ax.n_nu)[js], ax.cutoff), dt, vals


def _oracle_emission_task(args):
    """Oracle emission spectrum and band values of one proposal on the
    seeded field slice; returns (seconds, spectrum, bands)."""
    theta, cfg, filt = args
    from oracle import forward as Fw, radiation as R
    f = _ORACLE_STATE.get("field")
    if f is None:
        ax = W.grid_axes(n_nu=SLICE_N)
        f = _ORACLE_STATE["field"] = W.opacity_field(4, ax.p_bar, ax.t_K, SLICE_N).astype(np.float64)
    ax = W.grid_axes(n_nu=SLICE_N)
    t = time.perf_counter()
    F = Fw.emission_spectrum(f, ax.p_bar, ax.t_K, W.nu_axis(ax.nu_start, ax.dnu, SLICE_N), theta, cfg)
    B = R.band_integrate(F, filt)
    return time.perf_counter() - t, F, B


def _oracle_transmission_task(args):
    """Oracle transit depths of one instance (span clipped into the field
    slice); returns (seconds, depths, bands)."""
    inst, cfg, filt = args
    from oracle import forward as Fw, radiation as R
    f = _ORACLE_STATE.get("field")
    if f is None:
        ax = W.grid_axes(n_nu=SLICE_N)
        f = _ORACLE_STATE["field"] = W.opacity_field(4, ax.p_bar, ax.t_K, SLICE_N).astype(np.float64)
    ax = W.grid_axes(n_nu=SLICE_N)
    t = time.perf_counter()
    d = Fw.transmission_spectrum(f, ax.p_bar, ax.t_K, ax.nu_start, ax.dnu, inst, 0, cfg)
    B = R.band_integrate(d, filt, int(inst.nu_lo[0]))
    return time.perf_counter() - t, d, B


def em_cfg(S):
    """Emission configuration of the benchmark (oracle and library keys)."""
    return dict(geometry=0, n_angles=N_ANGLES, g=W.HD189_GRAV_CGS, mu=W.MEAN_MOLECULAR_MASS_AMU,
                x0=[W.BASE_VMR] * S, t_int=W.T_INT_K, t_star=W.HD189_TSTAR_K, r_star_tp=W.HD189_RSTAR_CM,
                a_orbit=W.HD189_A_CM, t_min=500.0, t_max=3000.0)


def tr_cfg(S):
    return dict(em_cfg(S), geometry=1, p_ref=W.HD189_PREF_BAR, p_top=1e-8, p_bot=100.0)


def slice_filters(n_bands, seed=3000):
    ax = W.grid_axes(n_nu=SLICE_N)
    return W.gaussian_filters(W.nu_axis(ax.nu_start, ax.dnu, SLICE_N), n_bands, 1002.0, 1058.0, 2.0, 20.0,
                              seed=seed)


def sample_points(lo, hi, seed):
    """SAMPLE_POINTS sorted grid indices spread over [lo, hi)."""
    g = np.random.default_rng(seed)
    edges = np.linspace(lo, hi, SAMPLE_POINTS + 1)
    return np.array([int(g.integers(int(a), max(int(a) + 1, int(b)))) for a, b in zip(edges[:-1], edges[1:])])


def emission_sample_cells(theta, S):
    """Oracle T(P) of the sampled proposals and the (species, layer,
    temperature) cells their linear-in-T interpolation reads."""
    from oracle import forward as Fw
    ax = W.grid_axes()
    cfg = em_cfg(S)
    cells = set()
    for p in EM_SAMPLE_PROPOSALS:
        T = Fw.tp_of(theta[p], ax.p_bar, cfg)
        for k in range(len(ax.p_bar)):
            m, _ = Fw.bracket(ax.t_K, T[k])
            for s in range(S):
                cells.update({(s, k, m), (s, k, min(m + 1, len(ax.t_K) - 1))})
    return sorted(cells)


def transmission_sample_cells(inst, S):
    from oracle import forward as Fw
    ax = W.grid_axes()
    cfg = tr_cfg(S)
    lp = np.log10(ax.p_bar)
    cells = set()
    for i in TR_SAMPLE_INSTANCES:
        P = Fw.instance_levels(inst.n_levels[i], cfg["p_top"], cfg["p_bot"])
        T = Fw.tp_of(inst.theta[i], P, cfg)
        for k in range(len(P)):
            a, _ = Fw.bracket(lp, np.log10(P[k]))
            m, _ = Fw.bracket(ax.t_K, T[k])
            for s in range(S):
                for aa in (a, min(a + 1, len(lp) - 1)):
                    for mm in (m, min(m + 1, len(ax.t_K) - 1)):
                        cells.add((s, aa, mm))
    return sorted(cells)


def cpu_phase(target_s=15.0, nwin=48, seed=0, full=True):
    """The oracle's part of the benchmark, on the host cores (spawned pool,
    one process per core), before any CUDA call:
      * opacity baseline: random (species, layer, T) cells x 48-point windows
        of the 5e6-line grid (every line within the cutoff), about target_s
        of work; the values are kept for the full-size opacity parity;
      * (full) the oracle opacity at the cells and wavenumbers that sampled
        proposals / instances of the full-size generation and transit batch
        read, for their FP32-vs-FP64 errors;
      * (full) emission and transmission baselines on the seeded field slice
        (the oracle's cost grows linearly with the points of a spectrum, so
        full-size rates are extrapolated by point count), and the DE-MC
        retrieval baseline with the oracle forward model."""
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(seed)
    ctx = mp.get_context("spawn")
    out = {}
    with ctx.Pool(cores, initializer=_oracle_init) as pool:
        def tasks(n):
            res = []
            for _ in range(n):
                j0 = int(rng.integers(0, 100_000 - nwin))
                res.append((int(rng.integers(3)), int(rng.integers(100)), int(rng.integers(20)),
                            tuple(range(j0, j0 + nwin))))
            return res
        cal = pool.map(_oracle_window, tasks(cores))
        per_task = max(statistics.median(dt for _, dt, _ in cal), 1e-3)
        n_tasks = max(cores, int(target_s / per_task) * cores)
        tk = tasks(n_tasks)
        t = time.perf_counter()
        res = pool.map(_oracle_window, tk)
        wall = time.perf_counter() - t
        evals = sum(e for e, _, _ in res)
        out["opacity"] = {"value": evals / wall / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                          "sample": f"{n_tasks} random (species, layer, T) cells x {nwin}-point windows of the "
                                    f"5e6-line grid, every line within the cutoff; {evals:.3g} evals in {wall:.1f} s"}
        out["opacity_windows"] = [(a[0], a[1], a[2], a[3][0], r[2]) for a, r in zip(tk, res)]
        if not full:
            return out
        # sampled cells of the full-size generation and transit batch
        S = 4
        theta = W.proposals(N_PROPOSALS, generation=0, n_species=S)
        em_shared = sample_points(0, 100_000, 7000)
        em_js = {p: em_shared for p in EM_SAMPLE_PROPOSALS}
        em_union = np.unique(np.concatenate(list(em_js.values())))
        em_cells = emission_sample_cells(theta, S)
        inst = W.instances(TRANS_INSTANCES, 100_000)
        tr_js = {i: sample_points(int(inst.nu_lo[i]), int(inst.nu_hi[i]), 7100 + i) for i in TR_SAMPLE_INSTANCES}
        tr_union = np.unique(np.concatenate(list(tr_js.values())))
        tr_cells = transmission_sample_cells(inst, S)
        t = time.perf_counter()
        em_vals = pool.map(_oracle_window, [(s, k, m, tuple(em_union)) for s, k, m in em_cells])
        tr_vals = pool.map(_oracle_window, [(s, k, m, tuple(tr_union)) for s, k, m in tr_cells])
        out["sample_oracle_s"] = time.perf_counter() - t
        out["em_sample"] = (em_js, em_union, em_cells, [v for _, _, v in em_vals], theta)
        out["tr_sample"] = (tr_js, tr_union, tr_cells, [v for _, _, v in tr_vals], inst)
        # emission baseline (the 2,048-proposal generation's shape: L = 100, M = 20, S = 4, 8 angles, 10 bands)
        n_em = max(16, cores)
        th_s = W.proposals(n_em, generation=0, n_species=S)
        filt = slice_filters(N_BANDS)
        pool.map(_oracle_emission_task, [(th_s[i], em_cfg(S), filt) for i in range(cores)])   # field built
        t = time.perf_counter()
        em = pool.map(_oracle_emission_task, [(th_s[i], em_cfg(S), filt) for i in range(n_em)])
        wall = time.perf_counter() - t
        out["em_slice"] = (th_s, filt, np.array([F for _, F, _ in em]), np.array([B for _, _, B in em]))
        rate = n_em / wall * SLICE_N / 100_000
        out["emission"] = {"value": rate, "unit": "spectra/s", "cores": cores, "kind": "oracle",
                           "sample": f"{n_em} proposals of the 9-parameter prior on a {SLICE_N}-point slice of "
                                     f"a seeded 4-species opacity field (100 layers x 20 T, 8 angles, 10 bands) in "
                                     f"{wall:.2f} s; rate extrapolated to 100,000 points by point count"}
        # transmission baseline (the transit batch's first instances, spans clipped to the slice)
        n_tr = max(16, cores)
        tcfg = tr_cfg(S)
        tfilt = slice_filters(12, seed=3001)
        clipped, full_span = [], []
        for i in range(n_tr):
            span = int(min(inst.nu_hi[i] - inst.nu_lo[i], SLICE_N))
            lo = (i * 97) % (SLICE_N - span + 1)
            clipped.append(W.Instances(inst.n_levels[i:i + 1], np.array([lo], np.int64),
                                       np.array([lo + span], np.int64), inst.r_planet[i:i + 1],
                                       inst.r_star[i:i + 1], inst.theta[i:i + 1]))
            full_span.append(int(inst.nu_hi[i] - inst.nu_lo[i]) / span)
        t = time.perf_counter()
        tr = pool.map(_oracle_transmission_task, [(c, tcfg, tfilt) for c in clipped])
        wall = time.perf_counter() - t
        out["tr_slice"] = (clipped, tfilt, [d for _, d, _ in tr], [B for _, _, B in tr])
        cpu_s = sum(dt * f for (dt, _, _), f in zip(tr, full_span))     # full-span seconds of one core
        out["transmission"] = {"value": n_tr / (cpu_s / cores), "unit": "spectra/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"{n_tr} instances of the transit batch (their level counts, spans "
                                         f"clipped to {SLICE_N} points of the seeded field), {wall:.2f} s; each "
                                         "instance's time scaled by its full span / clipped span, spread over "
                                         "the cores"}
    out["retrieval"] = cpu_retrieval_baseline()
    return out


def cpu_retrieval_baseline(n_gen=100, n_pts=300):
    """DE-MC (16 chains, 9 parameters) with the oracle forward model on a
    n_pts-point field slice for n_gen generations on one core; accepted
    samples/s extrapolated to full-size spectra by point count."""
    from oracle import forward as Fw, radiation as R, demc as D
    S = 4
    ax = W.grid_axes(n_nu=n_pts)
    f = W.opacity_field(S, ax.p_bar, ax.t_K, n_pts, seed=3600).astype(np.float64)
    nu = W.nu_axis(ax.nu_start, ax.dnu, n_pts)
    filt = W.gaussian_filters(nu, N_BANDS, 1000.5, 1005.5, 0.5, 2.0, seed=3002)
    cfg = em_cfg(S)
    lo, hi = W.THETA_LO, W.THETA_HI
    truth = lo + np.random.default_rng(6500).uniform(0.3, 0.7, 9) * (hi - lo)
    b_true = R.band_integrate(Fw.emission_spectrum(f, ax.p_bar, ax.t_K, nu, truth, cfg), filt)
    sig = b_true / 50.0
    data = b_true + np.random.default_rng(6501).normal(size=N_BANDS) * sig

    def loglike(th):
        b = R.band_integrate(Fw.emission_spectrum(f, ax.p_bar, ax.t_K, nu, th, cfg), filt)
        return -0.5 * float(np.sum(((b - data) / sig) ** 2))
    x0 = lo + np.random.default_rng(6000).uniform(size=(16, 9)) * (hi - lo)
    t = time.perf_counter()
    _, acc = D.run(loglike, x0, lo, hi, n_gen, np.random.default_rng(6001))
    wall = time.perf_counter() - t
    scale = 100_000 / n_pts
    return {"value": acc / (wall * scale), "unit": "accepted samples/s", "cores": 1, "kind": "oracle",
            "generations_per_s": n_gen / (wall * scale),
            "sample": f"16 chains x {n_gen} generations from a uniform start, oracle forward model on a "
                      f"{n_pts}-point seeded field slice ({acc} accepted in {wall:.1f} s); rates divided by "
                      f"{scale:.0f} (100,000 / {n_pts} points)"}


def cpu_oracle_rate(target_s=15.0, nwin=48, seed=0):
    """The opacity baseline alone (the reference arm's step)."""
    return cpu_phase(target_s, nwin, seed, full=False)["opacity"]


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    K, Wm = args.steps, args.warmup
    for _ in range(Wm):
        cpu_oracle_rate(target_s=2.0, seed=99)
    vals, times = [], []
    cb = None
    for k in range(K):
        t = time.perf_counter()
        cb = cpu_oracle_rate(target_s=args.ref_seconds, seed=k)
        times.append(time.perf_counter() - t)
        vals.append(cb["value"])
    v = statistics.median(vals)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": K, "warmup": Wm,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_desc(), "sample": cb["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- native arm
def run_native(args):
    ws, rank, local = dist_env()
    N = args.gpus if ws == 1 else ws
    # The oracle phase runs before any CUDA call (spawned pool, rank 0, N=1 only).
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_phase(target_s=args.cpu_seconds, full=not args.no_aux)

    import torch
    torch.cuda.set_device(local)
    dist = init_dist(ws, "nccl")
    dev = torch.device("cuda", local)
    from paper_2104_12522_gb300 import build
    build.build()
    import paper_2104_12522_gb300 as bart

    ax = W.grid_axes()
    species = W.opacity_grid_species(4)
    S_OP, S = 3, 4
    L, M, NU = len(ax.p_bar), len(ax.t_K), ax.n_nu
    evals = eval_count(species[:S_OP], ax)
    nu = bart.NuGrid(ax.nu_start, ax.dnu, NU)
    stream = torch.cuda.current_stream(dev)
    ctx = bart.Context(local, stream)

    # host inputs (pinned, for the end-to-end leg) and device copies
    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_lines = [(pinned(s.nu0), pinned(s.log10_s296), pinned(s.elow), pinned(s.gamma_ref)) for s in species]
    d_lines = [bart.DeviceLines(*(t.to(dev) for t in h), float(s.mass_amu)) for h, s in zip(h_lines, species)]
    theta_np = W.proposals(N_PROPOSALS, generation=0, n_species=S)
    filt_np = W.gaussian_filters(W.nu_axis(ax.nu_start, ax.dnu, NU), N_BANDS, 1100.0, 2900.0, 20.0, 200.0)
    h_theta, h_filt = pinned(theta_np), pinned(filt_np)
    theta, filt = h_theta.to(dev), h_filt.to(dev)
    grid = torch.empty((S, L, M, NU), dtype=torch.float32, device=dev)
    bands = torch.empty((N_PROPOSALS, N_BANDS), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    cfg = em_cfg(S)
    # the 4th molecule of the 4-species generation, built once (the timed
    # build is the 3-species, 5e6-line grid)
    ctx.build_opacity_grid(d_lines[S_OP:], ax.p_bar, ax.t_K, nu, ax.cutoff, out=grid[S_OP:])
    generation = lambda: ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, cfg, theta=theta, filters=filt,
                                                   bands=bands)
    graph = None

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        ctx.build_opacity_grid(d_lines[:S_OP], ax.p_bar, ax.t_K, nu, ax.cutoff, out=grid[:S_OP])
        if ev is not None:
            ev[1].record(stream)
        if graph is not None:
            graph.launch()              # one persistent fused launch, replayed from a CUDA graph
        else:
            generation()
        if ev is not None:
            ev[2].record(stream)

    step()                              # eager: autotunes the generation's tile width, sizes scratch
    graph = ctx.capture(generation)
    for _ in range(args.warmup):
        step()
        flush.fill_(1.0)
    ctx.sync()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_all = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_all[0].record(stream)
    for k in range(args.steps):
        step(evs[k])
        flush.fill_(1.0)            # L2 flush between steps (256 MiB write)
    t_all[1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ctx.sync()
    total_ms = t_all[0].elapsed_time(t_all[1])
    op_ms = [e[0].elapsed_time(e[1]) for e in evs]
    fw_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms = max_over_ranks(dist, total_ms, dev)
    op_avg = max_over_ranks(dist, sum(op_ms) / len(op_ms), dev)
    fw_avg = max_over_ranks(dist, sum(fw_ms) / len(fw_ms), dev)
    ms_per_step = total_ms / args.steps
    value = job_rate(N, evals, args.steps, total_ms) / 1e9

    # end-to-end through the public API with host buffers: H2D of the step's
    # inputs from pinned memory, the step, D2H of the grid and the band values.
    h_grid = torch.empty((S_OP, L, M, NU), dtype=torch.float32).pin_memory()
    h_bands = torch.empty(bands.shape, dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for h in h_lines[:S_OP] for t in h) + \
        h_theta.numel() * 4 + h_filt.numel() * 4
    d2h = h_grid.numel() * 4 + h_bands.numel() * 4
    e2e_steps = max(1, min(args.steps, 2))
    # the grid comes back one species at a time on a second stream, each slab
    # while the next species is built (one library call per species)
    copy_stream = torch.cuda.Stream(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        stream.wait_stream(copy_stream)          # the previous step's slabs are home
        for hd, dd in zip(h_lines[:S_OP], d_lines[:S_OP]):
            for h, d in zip(hd, (dd.nu0, dd.log10_s296, dd.elow, dd.gamma_ref)):
                d.copy_(h, non_blocking=True)
        theta.copy_(h_theta, non_blocking=True)
        filt.copy_(h_filt, non_blocking=True)
        for s_ in range(S_OP):
            ctx.build_opacity_grid(d_lines[s_:s_ + 1], ax.p_bar, ax.t_K, nu, ax.cutoff, out=grid[s_:s_ + 1])
            built = torch.cuda.Event()
            built.record(stream)
            copy_stream.wait_event(built)
            with torch.cuda.stream(copy_stream):
                h_grid[s_].copy_(grid[s_], non_blocking=True)
        graph.launch()
        h_bands.copy_(bands, non_blocking=True)
        stream.wait_stream(copy_stream)
        flush.fill_(1.0)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(dist, e0.elapsed_time(e1) / e2e_steps, dev)
    ctx.sync()
    assert np.all(np.isfinite(h_bands.numpy())), "non-finite band values"
    del h_grid

    fw = forward_model_leg(ctx, bart, torch, stream, grid, ax, nu, cfg, theta, filt, bands, generation, fw_avg, N,
                           S)
    parity = {}
    if cpu is not None:
        parity["opacity"] = opacity_parity(grid, cpu["opacity_windows"], ax)
    aux = {}
    if not args.no_aux:
        aux = run_aux(ctx, bart, torch, dev, stream, grid, ax, nu, filt, cfg, args, d_lines, theta, cpu, parity)

    if rank == 0:
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peaks = {}
        pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pp):
            with open(pp) as fh:
                peaks = json.load(fh)
        max_mhz = float(peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0)
        op_launch_ms = op_avg / OPACITY_LAUNCHES_PER_STEP
        achieved = FLOPS_PER_EVAL * evals / OPACITY_LAUNCHES_PER_STEP / (op_launch_ms / 1e3) / 1e12
        peak = fp32_peak_tflops(n_sm, max_mhz)
        traffic = committed_traffic(OPACITY_SOURCES, "opacity_kernel")
        fw["roofline"] = emission_roofline(fw["ms_per_generation"], n_sm, max_mhz, peaks, L, NU)
        cb = None
        if cpu is not None:
            cb = dict(cpu["opacity"])
            cb["workloads"] = {k: cpu[k] for k in ("emission", "transmission", "retrieval") if k in cpu}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": N, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(), "evals_per_step": evals,
                       "l2": "256 MiB write between steps; the 2.4 GB grid written and the 3.2 GB grid read each "
                             "step exceed L2",
                       "parallelism": f"replicas x{N} (independent problems, no collective)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "frac_16flop": achieved * RATIONAL_FLOPS_PER_EVAL / FLOPS_PER_EVAL / peak,
                         "kernel": "opacity_kernel",
                         "note": (f"{FLOPS_PER_EVAL} algorithmic FP32 flops per line-point evaluation "
                                  f"(frac_16flop: the same time with {RATIONAL_FLOPS_PER_EVAL}); peak = "
                                  f"{n_sm} SMs x 128 FP32 lanes x 2 x {max_mhz:.0f} MHz (max SM clock); "
                                  f"launch time = opacity-build events / {OPACITY_LAUNCHES_PER_STEP}")},
            "forward_model": fw,
            "parity": parity,
            "opacity_build_ms": op_avg,
            "opacity_build_ms_per_step": [round(v, 2) for v in op_ms],
            "cpu_baseline": cb,
            "e2e": {"value": N * evals / (e2e_ms / 1e3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms},
            "gpu_launches": KERNELS_PER_STEP * args.steps,
            "clocks": clk,
        }
        line.update(aux)
        line["autotune"] = ctx.autotune_report()
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def emission_roofline(ms, n_sm, max_mhz, peaks, L, NU):
    """MUFU roofline of the fused generation: the method's NA ex2 of the
    angles plus the Planck function's ex2 and reciprocal per (proposal, layer,
    wavenumber), against MUFU_PER_CLK results per clock per SM (the kernel
    executes NA + 1 of them: one ex2 and one reciprocal give the Planck
    function of a wavenumber pair); DRAM fraction from the committed ncu
    capture of the same kernel source."""
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    units = N_PROPOSALS * L * NU
    mufu = units * (N_ANGLES + 2) / (ms / 1e3) / 1e12
    mufu_peak = n_sm * MUFU_PER_CLK * max_mhz * 1e6 / 1e12
    dram = committed_traffic(FORWARD_SOURCES, "emission_fused_kernel")
    # the grid reads counted as if every (proposal, layer, wavenumber) streamed
    # its 2 S values (lower and upper temperature bracket per species)
    alg_bytes = units * 2 * FW_SPECIES * 4
    return {"bound": "mufu", "achieved": mufu, "peak": mufu_peak, "unit": "Tops/s", "frac": mufu / mufu_peak,
            "traffic": dram, "dram_frac": dram / (ms / 1e3) / (hbm * 1e9) if dram else None,
            "algorithmic_bytes": alg_bytes, "algorithmic_gbs": alg_bytes / (ms / 1e3) / 1e9,
            "hbm_frac_algorithmic": alg_bytes / (ms / 1e3) / (hbm * 1e9),
            "kernel": "emission_fused_kernel",
            "note": (f"{N_ANGLES + 2} MUFU ops per (proposal, layer, wavenumber): {N_ANGLES} ex2 of the angles, "
                     f"ex2 and reciprocal of the Planck function (the kernel executes {N_ANGLES + 1}: the Planck "
                     f"function of a wavenumber pair takes one ex2 and one reciprocal); peak = {n_sm} SMs x "
                     f"{MUFU_PER_CLK} MUFU results "
                     f"per clock x {max_mhz:.0f} MHz.  The proposals of a wavenumber tile share the grid rows "
                     "through L2, so DRAM moves about the grid twice per generation: dram_frac = DRAM bytes per "
                     "generation (ncu) / time / measured HBM copy bandwidth; hbm_frac_algorithmic counts the grid "
                     "reads as if every (proposal, layer, wavenumber) streamed its 2 S values")}


def forward_model_leg(ctx, bart, torch, stream, grid, ax, nu, cfg, theta, filt, bands, generation, fw_ms, N, S):
    """The 2,048-proposal generation: the graph-replayed fused launch (timed
    in the step), the same launch eager, the three-launch split path, and the
    3-species grid with the fourth scaling unused."""
    res = {"spectra_per_s": N * N_PROPOSALS / (fw_ms / 1e3), "ms_per_generation": fw_ms,
           "launch": "one persistent fused kernel per generation, replayed from a CUDA graph",
           "proposals": N_PROPOSALS, "angles": N_ANGLES, "bands": N_BANDS, "species": S}
    res["eager_ms"] = _event_ms(torch, stream, generation, reps=3)
    ctx.set_emission_launch(bart.BART_LAUNCH_SPLIT)
    generation()
    res["split_three_launches_ms"] = _event_ms(torch, stream, generation, reps=3)
    ctx.set_emission_launch(bart.BART_LAUNCH_FUSED_TMA)
    generation()
    res["fused_bulk_copy_staging_ms"] = _event_ms(torch, stream, generation, reps=3)
    ctx.set_emission_launch(bart.BART_LAUNCH_FUSED)
    g3, th3 = grid[:3], theta[:, :8].contiguous()
    cfg3 = dict(cfg, x0=cfg["x0"][:3])
    run3 = lambda: ctx.forward_spectra_batch(g3, ax.p_bar, ax.t_K, nu, cfg3, theta=th3, filters=filt, bands=bands)
    run3()
    ms3 = _event_ms(torch, stream, run3, reps=3)
    res["species3"] = {"ms_per_generation": ms3, "spectra_per_s": N * N_PROPOSALS / (ms3 / 1e3)}
    generation()               # leave the 4-species bands in place
    ctx.sync()
    return res


def opacity_parity(grid, windows, ax):
    """FP32-vs-FP64 error of the full-size grid on the oracle's baseline
    windows: max relative error over points above 1e-6 of their window's
    maximum, and the largest relative L2 error of a window."""
    worst, worst_l2, npts = 0.0, 0.0, 0
    for s, k, m, j0, vals in windows:
        got = grid[s, k, m, j0:j0 + len(vals)].double().cpu().numpy()
        ref = np.asarray(vals, np.float64)
        big = ref > 1e-6 * ref.max()
        worst = max(worst, float(np.max(np.abs(got[big] - ref[big]) / ref[big])))
        worst_l2 = max(worst_l2, float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        npts += len(vals)
    return {"windows": len(windows), "points": npts, "max_rel": worst, "max_window_rel_l2": worst_l2,
            "tolerance": {"max_rel": 1e-4, "rel_l2": 1e-5}}


def emission_sample_parity(ctx, torch, grid, ax, nu, cfg, theta, sample):
    """FP32-vs-FP64 error of sampled outputs of the full-size generation:
    the 2,048-proposal fused launch (as timed) with its spectra kept, against
    the oracle's whole chain (line lists -> opacity at the cells these
    proposals read -> T interpolation -> emission) at 8 wavenumbers of 3
    proposals."""
    from oracle import forward as Fw
    js, union, cells, vals, theta_np = sample
    S, L, M = int(grid.shape[0]), len(ax.p_bar), len(ax.t_K)
    spec = torch.empty((N_PROPOSALS, ax.n_nu), dtype=torch.float32, device=grid.device)
    ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, cfg, theta=theta, spectra=spec)
    ctx.sync()
    g_o = np.zeros((S, L, M, len(union)))
    for (s, k, m), v in zip(cells, vals):
        g_o[s, k, m] = v
    nu_u = W.nu_axis(ax.nu_start, ax.dnu, ax.n_nu)[union]
    worst, n = 0.0, 0
    for p, jp in js.items():
        F = Fw.emission_spectrum(g_o, ax.p_bar, ax.t_K, nu_u, theta_np[p], cfg)
        idx = np.searchsorted(union, jp)
        got = spec[p, torch.tensor(jp, device=grid.device)].double().cpu().numpy()
        worst = max(worst, float(np.max(np.abs(got - F[idx]) / F[idx])))
        n += len(jp)
    del spec
    return {"points": n, "proposals": len(js), "max_rel": worst, "tolerance": 1e-4,
            "note": "oracle chain from the line lists at the sampled wavenumbers of the full-size grid"}


def transmission_sample_parity(spec_t, inst_offsets, ax, S, sample):
    """FP32-vs-FP64 error of sampled transit depths of the full-size batch
    (the timed launch's output) against the oracle's whole chain at 8
    wavenumbers of each of 2 instances."""
    from oracle import forward as Fw
    js, union, cells, vals, inst = sample
    L, M = len(ax.p_bar), len(ax.t_K)
    g_o = np.zeros((S, L, M, len(union)))
    for (s, k, m), v in zip(cells, vals):
        g_o[s, k, m] = v
    cfg = tr_cfg(S)
    worst, n = 0.0, 0
    spec = spec_t.cpu().numpy()
    for i, ji in js.items():
        # the sampled columns act as the instance's span (no Rayleigh term, so
        # the wavenumbers themselves do not enter)
        one = W.Instances(inst.n_levels[i:i + 1], np.array([0], np.int64), np.array([len(union)], np.int64),
                          inst.r_planet[i:i + 1], inst.r_star[i:i + 1], inst.theta[i:i + 1])
        d = Fw.transmission_spectrum(g_o, ax.p_bar, ax.t_K, ax.nu_start, ax.dnu, one, 0, cfg)
        idx = np.searchsorted(union, ji)
        got = spec[inst_offsets[i] + (ji - int(inst.nu_lo[i]))].astype(np.float64)
        worst = max(worst, float(np.max(np.abs(got - d[idx]) / d[idx])))
        n += len(ji)
    return {"points": n, "instances": len(js), "max_rel": worst, "tolerance": 1e-4,
            "note": "oracle chain from the line lists at the sampled wavenumbers of the full-size grid"}


def slice_parity(ctx, bart, torch, dev, cpu):
    """FP32-vs-FP64 error of the generation and the transit batch on the
    seeded opacity-field slice (100 layers x 20 T x 3,000 points, 4 species):
    every spectrum point and band value of 16+ proposals and instances,
    through the same fused launch path as the step."""
    ax = W.grid_axes(n_nu=SLICE_N)
    field = torch.tensor(W.opacity_field(4, ax.p_bar, ax.t_K, SLICE_N), device=dev)
    nu = bart.NuGrid(ax.nu_start, ax.dnu, SLICE_N)
    th, filt, F_o, B_o = cpu["em_slice"]
    spec = torch.empty((len(th), SLICE_N), dtype=torch.float32, device=dev)
    bands = torch.empty((len(th), N_BANDS), dtype=torch.float32, device=dev)
    ctx.forward_spectra_batch(field, ax.p_bar, ax.t_K, nu, em_cfg(4), theta=torch.tensor(th, device=dev),
                              spectra=spec, filters=torch.tensor(filt, device=dev), bands=bands)
    ctx.sync()
    rel = lambda g, o: float(np.max(np.abs(g.astype(np.float64) - o) / np.abs(o)))
    out = {"emission": {"proposals": len(th), "spectra_max_rel": rel(spec.cpu().numpy(), F_o),
                        "bands_max_rel": rel(bands.cpu().numpy(), B_o)}}
    clipped, tfilt, d_o, tb_o = cpu["tr_slice"]
    n = len(clipped)
    cat = lambda f: np.concatenate([getattr(c, f) for c in clipped])
    lo, hi = cat("nu_lo"), cat("nu_hi")
    offs = np.concatenate([[0], np.cumsum(hi - lo)]).astype(np.int64)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    tspec = torch.empty(int(offs[-1]), dtype=torch.float32, device=dev)
    tb = torch.empty((n, 12), dtype=torch.float32, device=dev)
    ctx.forward_spectra_batch(field, ax.p_bar, ax.t_K, nu, tr_cfg(4), theta=d(cat("theta")),
                              n_levels=d(cat("n_levels")), nu_lo=d(lo), nu_hi=d(hi), spec_offsets=d(offs),
                              r_planet=d(cat("r_planet")), r_star=d(cat("r_star")), spectra=tspec,
                              filters=d(tfilt), bands=tb)
    ctx.sync()
    tspec, tb = tspec.cpu().numpy(), tb.cpu().numpy()
    es = max(rel(tspec[offs[i]:offs[i + 1]], d_o[i]) for i in range(n))
    eb = max(rel(tb[i][tb_o[i] > 0], tb_o[i][tb_o[i] > 0]) for i in range(n))
    out["transmission"] = {"instances": n, "depths_max_rel": es, "bands_max_rel": eb}
    return out


def _event_ms(torch, stream, fn, reps=1):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


TRANS_INSTANCES = 1024
TRANSMISSION_SOURCES = [os.path.join(ROOT, "paper_2104_12522_gb300", "csrc", f)
                        for f in ("transmission.cu", "forward.cuh", "bart_internal.cuh")]


def measured_hbm_gbs():
    """HBM copy bandwidth from MEASURED_PEAKS.json (fallback 6,800 GB/s) and its source."""
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        with open(pp) as fh:
            v = json.load(fh).get("hbm_gbs")
        if v:
            return float(v), "measured"
    return 6800.0, "fallback"


def committed_kv(kernel_srcs, name):
    """key = value lines of profiles/<name>.txt if taken on the current sources, else None."""
    path = os.path.join(ROOT, "profiles", f"{name}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as fh:
        for line in fh:
            if "=" in line and not line.lstrip().startswith("#"):
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
    return kv if kv.get("kernel_source_sha") == source_sha(kernel_srcs) else None


def transmission_leg(ctx, torch, dev, stream, grid, ax, nu, cfg, S):
    """The 1,024-instance transmission batch (40..150 levels, 1e4..1e5 points,
    12 bands) on the step's grid: time, spectra/s and the fraction of HBM its
    algorithmic bilinear reads (4 corners x S x 4 B per (level, wavenumber))
    would take if streamed."""
    n = TRANS_INSTANCES
    inst = W.instances(n, ax.n_nu)
    th = torch.tensor(inst.theta[:, :5 + S].copy(), device=dev)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    offs = inst.offsets
    spec = torch.empty(int(offs[-1]), dtype=torch.float32, device=dev)
    tb = torch.empty((n, 12), dtype=torch.float32, device=dev)
    tfilt = torch.tensor(W.gaussian_filters(W.nu_axis(ax.nu_start, ax.dnu, ax.n_nu), 12, 1100.0, 2900.0,
                                            100.0, 400.0, seed=3001), device=dev)
    tcfg = dict(cfg, geometry=1, p_ref=W.HD189_PREF_BAR, p_top=1e-8, p_bot=100.0)
    targs = dict(theta=th, n_levels=d(inst.n_levels), nu_lo=d(inst.nu_lo), nu_hi=d(inst.nu_hi),
                 spec_offsets=d(offs), r_planet=d(inst.r_planet), r_star=d(inst.r_star), spectra=spec,
                 filters=tfilt, bands=tb)
    run_t = lambda: ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, tcfg, **targs)
    run_t()
    ms = _event_ms(torch, stream, run_t, reps=2)
    ctx.sync()
    lnu = int(np.sum(inst.n_levels.astype(np.int64) * (inst.nu_hi - inst.nu_lo)))
    alg = lnu * 4 * S * 4
    hbm, src = measured_hbm_gbs()
    res = {"spectra_per_s": n / (ms / 1e3), "ms_per_batch": ms, "instances": n,
           "level_sum": int(inst.n_levels.sum()), "points": int(offs[-1]), "bands": 12,
           "level_points": lnu, "algorithmic_bytes": alg, "algorithmic_gbs": alg / (ms / 1e3) / 1e9,
           "hbm_frac_algorithmic": alg / (ms / 1e3) / 1e9 / hbm, "hbm_peak": f"{hbm:.0f} GB/s ({src})"}
    lb = committed_kv(TRANSMISSION_SOURCES, "trans_kernel_load_balance")
    if lb:
        # busiest / average SM active cycles of one launch (ncu)
        res["load_balance"] = {"sm_cycles_active_max": float(lb["sm_cycles_active_max"]),
                               "sm_cycles_active_avg": float(lb["sm_cycles_active_avg"]),
                               "efficiency": float(lb["sm_cycles_active_avg"]) / float(lb["sm_cycles_active_max"])}
    return run_t, tcfg, targs, spec, ms, res


def run_aux(ctx, bart, torch, dev, stream, grid, ax, nu, filt, cfg, args, d_lines, theta, cpu, parity):
    """Measurements beside the timed step, on the grid the step built:
    the transit batch, FP32-vs-FP64 samples of the full-size results, the
    paper's two approximations (line-strength bound, optical-depth limit),
    cloud deck and Rayleigh scattering, grid spacing, contribution functions,
    surrogate training and accuracy, screened vs plain retrieval.  Times are
    CUDA events on the library's stream."""
    S = int(grid.shape[0])
    out = {}
    run_t, tcfg, targs, spec, ms, out["transmission"] = transmission_leg(ctx, torch, dev, stream, grid, ax, nu,
                                                                         cfg, S)
    if cpu is not None and "em_sample" in cpu:
        parity["emission"] = emission_sample_parity(ctx, torch, grid, ax, nu, cfg, theta, cpu["em_sample"])
        parity["transmission"] = transmission_sample_parity(spec, W.instances(TRANS_INSTANCES, ax.n_nu).offsets, ax,
                                                            S, cpu["tr_sample"])
        parity["field_slice"] = slice_parity(ctx, bart, torch, dev, cpu)
        parity["oracle_seconds"] = cpu["sample_oracle_s"]
    out["cloud_rayleigh"] = cloud_rayleigh_leg(ctx, torch, stream, grid, ax, nu, cfg, theta, run_t, ms, tcfg, targs,
                                               spec)
    out["paper_approximations"] = paper_approximations(ctx, torch, stream, grid, ax, nu, cfg, d_lines, theta)
    out["grid_spacing"] = grid_spacing_leg(ctx, bart, torch, stream, ax, cfg, d_lines, theta)
    out["contribution_functions"] = contribution_leg(ctx, torch, stream, grid, ax, nu, filt, cfg, theta)
    net, out["surrogate"] = train_surrogate(ctx, bart, torch, dev, stream, grid, ax, nu, filt, cfg, S,
                                            args.train_steps)
    out["retrieval"] = run_retrieval(ctx, bart, torch, dev, stream, grid, ax, nu, filt, cfg, S, net,
                                     args.generations, args.burn, args.screen_beta, args.screen_margin)
    return out


def _max_rel(torch, got, ref, floor_frac=1e-6):
    """max |got/ref - 1| over points above floor_frac of their row maximum."""
    ref2 = ref.reshape(-1, ref.shape[-1])
    got2 = got.reshape(-1, ref.shape[-1])
    big = ref2 > floor_frac * ref2.amax(dim=1, keepdim=True)
    rel = ((got2 - ref2).abs() / ref2.clamp_min(1e-38))[big]
    return float(rel.max()) if rel.numel() else 0.0


def voigt_table_leg(ctx, torch, stream, grid, ax, nu, d_lines, build0, out, n_w=60, oversample=256):
    """The paper's Voigt-table scheme (Sec. 4 items 4-5) on the species-0 launch:
    a table of n_w x n_w widths spanning the workload's Doppler and Lorentz
    widths, sampled `oversample` times per grid interval; time against the
    direct launch and error against the direct grid."""
    import paper_2104_12522_gb300 as bart
    k, amu, c = 1.380649e-16, 1.66053906660e-24, 2.99792458e10
    m_lo, m_hi = min(W.SPECIES_MASS_AMU[:grid.shape[0]]), max(W.SPECIES_MASS_AMU[:grid.shape[0]])
    gref_lo, gref_hi = 0.05, 0.1           # the synthetic line lists' gamma_ref range, cm^-1
    s_lo = ax.nu_start / c * np.sqrt(k * ax.t_K[0] / (m_hi * amu))
    s_hi = (ax.nu_start + ax.n_nu * ax.dnu) / c * np.sqrt(k * ax.t_K[-1] / (m_lo * amu))
    g_lo = gref_lo * ax.p_bar[0] * np.sqrt(296.0 / ax.t_K[-1])
    g_hi = gref_hi * ax.p_bar[-1] * np.sqrt(296.0 / ax.t_K[0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tab = bart.VoigtTable(ctx, n_w, s_lo, s_hi, n_w, g_lo, g_hi, oversample, ax.dnu, ax.cutoff)
    e1.record(stream)
    torch.cuda.synchronize()
    fill_ms = e0.elapsed_time(e1)
    ms0 = _event_ms(torch, stream, build0)
    ms = _event_ms(torch, stream, lambda: ctx.build_opacity_grid_table(tab, d_lines[:1], ax.p_bar, ax.t_K, nu,
                                                                      ax.cutoff, out=out))
    got0, ref0 = out[0].reshape(-1, ax.n_nu), grid[0].reshape(-1, ax.n_nu)
    l2 = float(torch.linalg.vector_norm(got0.double() - ref0.double()) / torch.linalg.vector_norm(ref0.double()))
    res = {"n_sigma": n_w, "n_gamma": n_w, "oversample": oversample, "table_bytes": tab.nbytes,
           "fill_ms": fill_ms, "ms": ms, "ms_direct": ms0, "speed_vs_direct": ms0 / ms, "grid_rel_l2": l2,
           "grid_max_rel_err_1e-3": _max_rel(torch, got0, ref0, 1e-3)}
    tab.close()
    return res


H2_RAYLEIGH = 8.4e-45        # cm^2 (cm^-1)^-4: H2 cross-section per molecule a nu^4


def cloud_rayleigh_leg(ctx, torch, stream, grid, ax, nu, cfg, theta, run_t, ms_t, tcfg, targs, spec_t):
    """Cost of the Sec. 3 gray cloud deck (0.1 bar, at the reference radius)
    and H2 Rayleigh scattering on the bench's two forward-model workloads:
    the 2,048-proposal emission generation and the 1,024-instance transmission
    batch, each timed with and without the options, with the largest relative
    change of the spectra they cause."""
    res = {}
    n = theta.shape[0]
    ref = torch.empty((n, ax.n_nu), dtype=torch.float32, device=grid.device)
    out = torch.empty_like(ref)
    run = lambda c, o: ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, c, theta=theta, spectra=o)
    run(cfg, ref)
    ms0 = _event_ms(torch, stream, lambda: run(cfg, ref))
    t_ref = spec_t.clone()
    for name, extra in (("rayleigh", {"rayleigh_coef": H2_RAYLEIGH}), ("deck_0.1bar", {"p_cloud": 0.1}),
                        ("both", {"rayleigh_coef": H2_RAYLEIGH, "p_cloud": 0.1})):
        c = dict(cfg, **extra)
        run(c, out)
        ms = _event_ms(torch, stream, lambda: run(c, out))
        tc = dict(tcfg, **extra)
        run_tc = lambda: ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, tc, **targs)
        run_tc()
        mst = _event_ms(torch, stream, run_tc, reps=2)
        res[name] = {"emission_ms": ms, "emission_ms_without": ms0,
                     "emission_spectra_per_s": n / (ms / 1e3),
                     "emission_max_rel_change": _max_rel(torch, out, ref, 0.0),
                     "transmission_ms": mst, "transmission_ms_without": ms_t,
                     "transmission_spectra_per_s": 1024 / (mst / 1e3),
                     "transmission_max_rel_change": _max_rel(torch, spec_t, t_ref, 0.0)}
    ctx.sync()
    return res


def grid_spacing_leg(ctx, bart, torch, stream, ax, cfg, d_lines, theta, n_prop=256):
    """App. D: band values of the same proposals on wavenumber grids of
    0.025, 0.1, 0.25 and 1.0 cm^-1 (each also shifted by 0.09 cm^-1) over
    1900..2100 cm^-1, against the 0.025 cm^-1 grid: the discretisation error
    the grid spacing puts into band-integrated values.  Eight Gaussian bands
    (FWHM 5..30 cm^-1); each grid built by the library (time reported)."""
    res = []
    th = theta[:n_prop].contiguous()
    ref = None
    for dnu in (0.025, 0.1, 0.25, 1.0):
        for shift in (0.0, 0.09):
            if dnu == 0.025 and shift:
                continue
            n_nu = int(round(200.0 / dnu))
            nu_g = bart.NuGrid(1900.0 + shift, dnu, n_nu)
            filt = torch.tensor(W.gaussian_filters(W.nu_axis(1900.0 + shift, dnu, n_nu), 8, 1920.0, 2080.0, 5.0,
                                                   30.0, seed=3100), device=theta.device)
            g = torch.empty((len(d_lines), len(ax.p_bar), len(ax.t_K), n_nu), dtype=torch.float32,
                            device=theta.device)
            build = lambda: ctx.build_opacity_grid(d_lines, ax.p_bar, ax.t_K, nu_g, ax.cutoff, out=g)
            build()                                  # scratch sized on the first call
            ms_build = _event_ms(torch, stream, build, reps=1)
            bands = torch.empty((n_prop, 8), dtype=torch.float32, device=theta.device)
            ctx.forward_spectra_batch(g, ax.p_bar, ax.t_K, nu_g, cfg, theta=th, filters=filt, bands=bands)
            ctx.sync()
            b = bands.double()
            entry = {"dnu": dnu, "shift": shift, "n_nu": n_nu, "build_ms": ms_build}
            if ref is None:
                ref = b
            else:
                rel = ((b - ref).abs() / ref.abs()).flatten()
                entry["band_max_rel_diff"] = float(rel.max())
                entry["band_median_rel_diff"] = float(rel.median())
            res.append(entry)
            del g
    return res


def contribution_leg(ctx, torch, stream, grid, ax, nu, filt, cfg, theta, n=4):
    """Band contribution functions of n proposals on the full grid (the
    post-processing of Sec. 3): time, and how closely the per-layer band
    values add up to the forward model's band values."""
    th = theta[:n].contiguous()
    L, nb = len(ax.p_bar), int(filt.shape[0])
    cb = torch.empty((n, L, nb), dtype=torch.float32, device=theta.device)
    run = lambda: ctx.contribution_functions(grid, ax.p_bar, ax.t_K, nu, cfg, theta=th, filters=filt, bands=cb)
    run()
    ms = _event_ms(torch, stream, run, reps=3)
    bands = torch.empty((n, nb), dtype=torch.float32, device=theta.device)
    ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, cfg, theta=th, filters=filt, bands=bands)
    ctx.sync()
    tot = cb.double().sum(dim=1)
    rel = float(((tot - bands.double()).abs() / bands.double().abs()).max())
    peak = cb.double().argmax(dim=1).float()
    return {"proposals": n, "layers": L, "bands": nb, "ms": ms, "sum_vs_band_values_max_rel": rel,
            "peak_layer_median": float(peak.median())}


def paper_approximations(ctx, torch, stream, grid, ax, nu, cfg, d_lines, theta):
    """Speed-up against accuracy lost of Sec. 4 items 6 and 7 on the bench's
    workload.  (a) The line-strength bound: time of the species-0 launch of
    the grid build (2,000 cells) against the same launch without it; the grid
    error against the step's grid (relative L2 and max relative error over
    points above 1e-3 of their row maximum); and the error of the emission
    spectra of the 2,048 proposals computed from the thresholded 3-species
    grid.  (b) The optical-depth limit on the 2,048-proposal generation."""
    res = {"line_threshold": [], "tau_limit": []}
    n = theta.shape[0]
    spec_ref = torch.empty((n, ax.n_nu), dtype=torch.float32, device=grid.device)
    spec = torch.empty_like(spec_ref)
    run = lambda g, c, o: ctx.forward_spectra_batch(g, ax.p_bar, ax.t_K, nu, c, theta=theta, spectra=o)
    run(grid, cfg, spec_ref)
    out = torch.empty((1,) + tuple(grid.shape[1:]), dtype=torch.float32, device=grid.device)
    full = torch.empty_like(grid)
    build0 = lambda: ctx.build_opacity_grid(d_lines[:1], ax.p_bar, ax.t_K, nu, ax.cutoff, out=out)
    ms0 = _event_ms(torch, stream, build0)
    ref0 = grid[0].reshape(-1, ax.n_nu)
    for rel in (1e-6, 1e-4, 1e-2):
        ctx.set_line_threshold(rel)
        ms = _event_ms(torch, stream, build0)
        ctx.build_opacity_grid(d_lines, ax.p_bar, ax.t_K, nu, ax.cutoff, out=full)
        ctx.set_line_threshold(0.0)
        run(full, cfg, spec)
        got0 = out[0].reshape(-1, ax.n_nu)
        # FP64: squares of FP32 opacities (1e-13 .. 1e-30 cm^2) underflow
        l2 = float(torch.linalg.vector_norm(got0.double() - ref0.double()) / torch.linalg.vector_norm(ref0.double()))
        res["line_threshold"].append({"rel": rel, "ms": ms, "ms_without": ms0, "speedup": ms0 / ms,
                                      "grid_rel_l2": l2, "grid_max_rel_err_1e-3": _max_rel(torch, got0, ref0, 1e-3),
                                      "spectra_max_rel_err": _max_rel(torch, spec, spec_ref, 0.0)})
    del full
    res["voigt_table"] = voigt_table_leg(ctx, torch, stream, grid, ax, nu, d_lines, build0, out)
    ms0 = _event_ms(torch, stream, lambda: run(grid, cfg, spec_ref))
    for tau_max in (30.0, 10.0, 3.0):
        c = dict(cfg, tau_max=tau_max)
        run(grid, c, spec)
        ms = _event_ms(torch, stream, lambda: run(grid, c, spec))
        res["tau_limit"].append({"tau_max": tau_max, "ms": ms, "ms_without": ms0, "speedup": ms0 / ms,
                                 "spectra_max_rel_err": _max_rel(torch, spec, spec_ref, 0.0)})
    ctx.sync()
    return res


def train_surrogate(ctx, bart, torch, dev, stream, grid, ax, nu, filt, cfg, S, n_steps):
    """MLP (5 + S) -> 256 -> 256 -> 256 -> bands trained by the library's
    kernels on 200,000 forward-model band vectors; returns (net, report)."""

    n_train, n_val = 200_000, 4096
    widths = [5 + S, 256, 256, 256, N_BANDS]
    th_all = torch.tensor(W.proposals(n_train + n_val, generation=100, n_species=S), device=dev)
    y_all = torch.empty((n_train + n_val, N_BANDS), dtype=torch.float32, device=dev)
    def gen():
        for i in range(0, n_train + n_val, N_PROPOSALS):
            j = min(i + N_PROPOSALS, n_train + n_val)
            ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, cfg, theta=th_all[i:j], filters=filt,
                                      bands=y_all[i:j])
    gen_ms = _event_ms(torch, stream, gen)
    net = bart.Mlp(ctx, widths, bf16_weights=True, log_outputs=True, max_batch=N_PROPOSALS)
    lo, hi = W.THETA_LO[:5 + S].astype(np.float32), W.THETA_HI[:5 + S].astype(np.float32)
    logy = np.log10(y_all[:n_train].cpu().numpy().astype(np.float64))
    net.set_scaling(0.5 * (lo + hi), 2.0 / (hi - lo), logy.mean(0).astype(np.float32),
                    (1.0 / logy.std(0)).astype(np.float32))
    net.set_params(torch.tensor(W.mlp_init(widths), device=dev))
    g = torch.Generator(device=dev).manual_seed(5000)
    B = 1024
    # every step's batch drawn up front; the step loop runs in the library
    rows = torch.randint(0, n_train, (n_steps, B), device=dev, generator=g, dtype=torch.int32)
    lrs = [max(1e-3 * 0.5 * (1 + np.cos(np.pi * k / n_steps)), 1e-5) for k in range(n_steps)]
    x_tr, y_tr = th_all[:n_train], y_all[:n_train]
    train_ms = _event_ms(torch, stream, lambda: net.train_steps(x_tr, y_tr, rows, lrs))
    pred = torch.cat([net.forward(th_all[n_train + i:n_train + i + N_PROPOSALS])
                      for i in range(0, n_val, N_PROPOSALS)]).cpu().numpy()
    err = np.abs(pred / y_all[n_train:].cpu().numpy() - 1)
    x_inf = th_all[:N_PROPOSALS].contiguous()
    inf_ms = _event_ms(torch, stream, lambda: net.forward(x_inf), reps=20)
    flops = 6 * B * sum(widths[l] * widths[l + 1] for l in range(len(widths) - 1))   # forward + backward
    report = {"widths": widths, "train_spectra": n_train, "train_steps": n_steps, "batch": B,
                        "spectra_gen_ms": gen_ms, "train_ms": train_ms,
                        "train_tflops": flops * n_steps / (train_ms / 1e3) / 1e12,
                        "gemm": "BF16 tcgen05.mma, FP32 accumulators in tensor memory, 128 x 32 tiles; FP32 operands as hi/lo BF16 pairs",
                        "band_rel_err_median": float(np.median(err)), "band_rel_err_p99": float(np.percentile(err, 99)),
                        "inference_spectra_per_s": N_PROPOSALS / (inf_ms / 1e3)}
    return net, report


def run_retrieval(ctx, bart, torch, dev, stream, grid, ax, nu, filt, cfg, S, net, generations, n_burn, beta,
                  margin):
    """DE-MC with 16 chains on synthetic band data (S/N = 50): an exact-model
    burn-in, then plain and surrogate-screened runs from the same state, and
    the same pair with DEMCzs (4 chains, the burnt-in states as its archive)."""
    lo, hi = W.THETA_LO[:5 + S].astype(np.float32), W.THETA_HI[:5 + S].astype(np.float32)
    rng = np.random.default_rng(6500)
    truth = (lo + rng.uniform(0.3, 0.7, 5 + S) * (hi - lo)).astype(np.float32)
    bt = torch.empty((1, N_BANDS), dtype=torch.float32, device=dev)
    ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, cfg, theta=torch.tensor(truth[None], device=dev),
                              filters=filt, bands=bt)
    b_true = bt.cpu().numpy()[0]
    sig = (b_true / 50.0).astype(np.float32)
    data = torch.tensor((b_true + rng.normal(size=N_BANDS) * sig).astype(np.float32), device=dev)
    sigma = torch.tensor(sig, device=dev)
    res = {}
    # burn-in with the exact model from a uniform start; both measured runs
    # continue from the same burnt-in state (the surrogate screen is meant for
    # the sampling phase, where its errors are small against the posterior width)
    C = 16
    x0 = torch.tensor((lo + np.random.default_rng(6000).uniform(size=(C, 5 + S)) * (hi - lo)).astype(
        np.float32), device=dev)
    b0 = torch.empty((C, N_BANDS), dtype=torch.float32, device=dev)
    ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, cfg, theta=x0, filters=filt, bands=b0)
    L0 = torch.empty(C, dtype=torch.float64, device=dev)
    ctx.loglike_bands(b0, data, sigma, L0)
    burn = bart.Demc(ctx, C, lo, hi, jump_every=10, eps=1e-4, seed=6100)
    burn.set_state(x0, L0)
    burn_ms = _event_ms(torch, stream, lambda: ctx.retrieval_run(burn, None, grid, ax.p_bar, ax.t_K, nu, cfg, filt,
                                                                 data, sigma, n_burn, use_graph=True))
    xb_, Lb_ = torch.empty_like(x0), torch.empty_like(L0)
    burn.get_state(xb_, Lb_)
    res["burn_in"] = {"generations": n_burn, "ms": burn_ms}
    kept = {}
    for mode in ("plain", "screened", "demczs", "demczs_screened"):
        # DEMCzs (Sec. 4): 4 chains from the burnt-in state, its 16 states as the
        # initial archive, every chain moving at each of a generation's two steps
        zs, screened = mode.startswith("demczs"), mode.endswith("screened")
        Cm = 4 if zs else C
        s = bart.Demc(ctx, Cm, lo, hi, jump_every=10, eps=1e-4, seed=6000)
        s.set_screen(beta, margin)
        if zs:
            s.set_archive(xb_, capacity=C + Cm * (2 * generations // 10 + 1), thin=10, p_snooker=0.1)
        Ls0 = None
        if screened:
            Ls0 = torch.empty(C, dtype=torch.float64, device=dev)
            ctx.loglike_bands(net.forward(xb_), data, sigma, Ls0)
            Ls0 = Ls0[:Cm].contiguous()
        s.set_state(xb_[:Cm].contiguous(), Lb_[:Cm].contiguous(), Ls0)
        chain = torch.empty((generations, Cm, 5 + S), dtype=torch.float32, device=dev)
        st = {}
        def run():
            st.update(ctx.retrieval_run(s, net if screened else None, grid, ax.p_bar, ax.t_K, nu, cfg,
                                        filt, data, sigma, generations, use_graph=True, chain=chain))
        ms = _event_ms(torch, stream, run)
        ctx.sync()
        st["accepted_samples_per_s"] = st["accepted"] / (ms / 1e3)
        st["proposals_per_s"] = st["proposals"] / (ms / 1e3)
        st["generations"] = generations
        st["chains"] = Cm
        sp, gr, ess = ctx.chain_stats(chain)
        st["ess"] = ess
        st["ess_per_s"] = ess / (ms / 1e3)
        st["gelman_rubin_max"] = float(gr.max())
        st["ess_per_exact_eval"] = ess / max(st["exact_evals"], 1)
        kept[mode] = (chain.reshape(-1, 5 + S).double().cpu().numpy(),
                      (generations * Cm / sp.mean(0)).cpu().numpy())
        if screened:
            st["screen"] = {"beta": beta, "margin": margin}
        st["ms"] = ms
        if st["accepted"]:
            st["surrogate_err_mean"] = st["surrogate_err_sum"] / st["accepted"]
        res[mode] = st
    res["posterior_agreement"] = posterior_agreement(*kept["plain"], *kept["screened"])
    res["posterior_agreement_demczs"] = posterior_agreement(*kept["demczs"], *kept["demczs_screened"])
    res["false_rejection"] = screen_false_rejections(ctx, bart, torch, dev, grid, ax, nu, filt, cfg, S, net, lo, hi,
                                                     xb_, Lb_, data, sigma, beta, margin)
    return res


def posterior_agreement(xp, essp, xs, esss):
    """Plain vs screened posteriors within App. C standard errors: per
    parameter the difference of the means over s = sqrt(s_p^2 + s_s^2) with
    s = sigma / sqrt(ESS), and the content of the plain run's central 68%
    interval in the screened samples against 0.68 with
    s_C = sqrt(C (1 - C) (1/ESS_p + 1/ESS_s)) (App. C's content error in its
    large-ESS form, without the + 3 of the Beta posterior)."""
    z_mean, z_c, content = [], [], []
    for j in range(xp.shape[1]):
        sp_ = xp[:, j].std() / np.sqrt(essp[j])
        ss_ = xs[:, j].std() / np.sqrt(esss[j])
        z_mean.append(abs(xp[:, j].mean() - xs[:, j].mean()) / max(np.hypot(sp_, ss_), 1e-300))
        q16, q84 = np.percentile(xp[:, j], [16, 84])
        c = float(np.mean((xs[:, j] >= q16) & (xs[:, j] <= q84)))
        content.append(c)
        z_c.append(abs(c - 0.68) / np.sqrt(0.68 * 0.32 * (1.0 / essp[j] + 1.0 / esss[j])))
    return {"mean_z_max": float(max(z_mean)), "c68_z_max": float(max(z_c)),
            "c68_content_screened": [round(c, 4) for c in content],
            "agree_within_3_sigma": bool(max(z_mean) < 3.0 and max(z_c) < 3.0)}


def screen_false_rejections(ctx, bart, torch, dev, grid, ax, nu, filt, cfg, S, net, lo, hi, x, L, data, sigma,
                            beta, margin, n_half_steps=400):
    """Proposals from the burnt-in state, screened by the surrogate and all
    evaluated by the exact model: the mean exact Metropolis acceptance
    probability min(1, exp(L_y - L_x)) of the screened-out ones is the
    false-rejection rate (the state is held fixed; nothing is accepted)."""
    C = x.shape[0]
    s = bart.Demc(ctx, C, lo, hi, jump_every=10, eps=1e-4, seed=6200)
    s.set_screen(beta, margin)
    ls_x = torch.empty(C, dtype=torch.float64, device=dev)
    ctx.loglike_bands(net.forward(x), data, sigma, ls_x)
    s.set_state(x, L, ls_x)
    y = torch.empty((C, 5 + S), dtype=torch.float32, device=dev)
    inbox = torch.empty(C, dtype=torch.int32, device=dev)
    passed = torch.empty(C, dtype=torch.int32, device=dev)
    ls_y = torch.empty(C, dtype=torch.float64, device=dev)
    L_y = torch.empty(C, dtype=torch.float64, device=dev)
    b_y = torch.empty((C, N_BANDS), dtype=torch.float32, device=dev)
    Lx = L.cpu().numpy()
    p_rej, p_all = [], []
    for h in range(n_half_steps):
        s.propose(h, y, inbox)
        ctx.loglike_bands(net.forward(y), data, sigma, ls_y, mask=inbox)
        s.screen(h, inbox, ls_y, passed)
        ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, cfg, theta=y, filters=filt, bands=b_y, active=inbox)
        ctx.loglike_bands(b_y, data, sigma, L_y, mask=inbox)
        ib, ps, ly = inbox.cpu().numpy(), passed.cpu().numpy(), L_y.cpu().numpy()
        pa = np.minimum(1.0, np.exp(np.minimum(ly - Lx, 0.0)))
        p_all += list(pa[ib == 1])
        p_rej += list(pa[(ib == 1) & (ps == 0)])
    return {"half_steps": n_half_steps, "proposals_in_box": len(p_all), "screened_out": len(p_rej),
            "false_rejection_rate": float(np.mean(p_rej)) if p_rej else 0.0,
            "exact_acceptance_in_box": float(np.mean(p_all)) if p_all else 0.0}


def run_transmission_case(args):
    """The bench's 1,024-instance transmission batch alone, on the full-size
    4-species grid: one JSON line (for ncu captures of its launch)."""
    import torch
    from paper_2104_12522_gb300 import build
    build.build()
    import paper_2104_12522_gb300 as bart
    ax = W.grid_axes()
    species = W.opacity_grid_species(4)
    ctx = bart.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    nu = bart.NuGrid(ax.nu_start, ax.dnu, ax.n_nu)
    grid = ctx.build_opacity_grid([bart.device_lines(s) for s in species], ax.p_bar, ax.t_K, nu, ax.cutoff)
    *_, res = transmission_leg(ctx, torch, dev, stream, grid, ax, nu, em_cfg(4), 4)
    print(json.dumps({"transmission": res}), flush=True)
    return 0


def run_profile_case(args):
    """Small launches of the hot kernels for ncu captures: one opacity launch
    (species 0, 5e6-line list, 3 layers x 20 temperatures on the full
    100,000-point grid), one fused emission generation (2,048 proposals, 4
    species) and one transit batch (256 instances) on a 4,096-point slice of
    the grid."""
    import torch
    from paper_2104_12522_gb300 import build
    build.build()
    import paper_2104_12522_gb300 as bart
    ax = W.grid_axes()
    species = W.opacity_grid_species(4)
    dl = [bart.device_lines(s) for s in species]
    ctx = bart.Context(0)
    ctx.set_autotune(False)
    ctx.set_emission_tile(args.tile)
    nu = bart.NuGrid(ax.nu_start, ax.dnu, ax.n_nu)
    k3 = ax.p_bar[[0, 50, 99]]
    out = ctx.build_opacity_grid(dl[:1], k3, ax.t_K, nu, ax.cutoff)
    nsub = 4096
    nu_s = bart.NuGrid(ax.nu_start, ax.dnu, nsub)
    grid = ctx.build_opacity_grid(dl, ax.p_bar, ax.t_K, nu_s, ax.cutoff)
    theta = torch.tensor(W.proposals(N_PROPOSALS, generation=0, n_species=4), device="cuda")
    filt = torch.tensor(W.gaussian_filters(W.nu_axis(ax.nu_start, ax.dnu, nsub), N_BANDS, 1005.0, 1075.0,
                                           2.0, 20.0), device="cuda")
    bands = torch.empty((N_PROPOSALS, N_BANDS), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu_s, em_cfg(4), theta=theta, filters=filt, bands=bands)
    # one transmission batch: 256 uneven instances (40..150 levels, 1,000..4,096 points) on the slice
    inst = W.instances(256, nsub, span_lo=1000, span_hi=nsub)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    tspec = torch.empty(int(inst.offsets[-1]), dtype=torch.float32, device="cuda")
    tb = torch.empty((256, N_BANDS), dtype=torch.float32, device="cuda")
    ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu_s, tr_cfg(4), theta=d(inst.theta),
                              n_levels=d(inst.n_levels), nu_lo=d(inst.nu_lo), nu_hi=d(inst.nu_hi),
                              spec_offsets=d(inst.offsets), r_planet=d(inst.r_planet), r_star=d(inst.r_star),
                              spectra=tspec, filters=filt, bands=tb)
    ctx.sync()
    assert torch.isfinite(out).all() and torch.isfinite(bands).all() and torch.isfinite(tspec).all()
    print("profile case done")
    return 0


def run_generation_case(args):
    """The 2,048-proposal, 4-species fused generation alone on the full-size
    grid (the grid filled from the seeded opacity field pattern, tiled over
    wavenumber, so no line-by-line build is needed): reps graph replays, for
    DRAM-traffic captures of the fused kernel (one launch)."""
    import torch
    from paper_2104_12522_gb300 import build
    build.build()
    import paper_2104_12522_gb300 as bart
    ax = W.grid_axes()
    dev = torch.device("cuda", 0)
    ctx = bart.Context(0)
    if args.tile:
        ctx.set_emission_tile(args.tile)
    nu = bart.NuGrid(ax.nu_start, ax.dnu, ax.n_nu)
    pat = torch.tensor(W.opacity_field(4, ax.p_bar, ax.t_K, 1000), device=dev)
    grid = pat.repeat(1, 1, 1, ax.n_nu // 1000).contiguous()
    theta = torch.tensor(W.proposals(N_PROPOSALS, generation=0, n_species=4), device=dev)
    filt = torch.tensor(W.gaussian_filters(W.nu_axis(ax.nu_start, ax.dnu, ax.n_nu), N_BANDS, 1100.0, 2900.0,
                                           20.0, 200.0), device=dev)
    bands = torch.empty((N_PROPOSALS, N_BANDS), dtype=torch.float32, device=dev)
    gen = lambda: ctx.forward_spectra_batch(grid, ax.p_bar, ax.t_K, nu, em_cfg(4), theta=theta, filters=filt,
                                            bands=bands)
    gen()
    stream = torch.cuda.current_stream(dev)
    ms = _event_ms(torch, stream, gen, reps=max(1, args.steps))
    ctx.sync()
    print(json.dumps({"generation_ms": ms, "spectra_per_s": N_PROPOSALS / (ms / 1e3),
                      "autotune": ctx.autotune_report()}), flush=True)
    return 0


def run_mlp_case(args):
    """The surrogate's training step alone (9 -> 256 -> 256 -> 256 -> 10,
    batch 1,024, BF16 weights) for captures of its tensor-core GEMMs: 64
    steps through bart_mlp_train_steps on seeded inputs and targets."""
    import torch
    from paper_2104_12522_gb300 import build
    build.build()
    import paper_2104_12522_gb300 as bart
    ctx = bart.Context(0)
    dev = torch.device("cuda", 0)
    widths = list(W.SURROGATE_WIDTHS)
    net = bart.Mlp(ctx, widths, bf16_weights=True, log_outputs=True, max_batch=1024)
    lo, hi = W.THETA_LO.astype(np.float32), W.THETA_HI.astype(np.float32)
    net.set_scaling(0.5 * (lo + hi), 2.0 / (hi - lo), np.full(10, 4.0, np.float32), np.full(10, 2.0, np.float32))
    net.set_params(torch.tensor(W.mlp_init(widths), device=dev))
    x = torch.tensor(W.proposals(8192, generation=100, n_species=4), device=dev)
    t = torch.tensor((10 ** np.random.default_rng(5).uniform(3.5, 4.5, (8192, 10))).astype(np.float32), device=dev)
    g = torch.Generator(device=dev).manual_seed(1)
    rows = torch.randint(0, 8192, (64, 1024), device=dev, generator=g, dtype=torch.int32)
    net.train_steps(x, t, rows, [1e-3] * 64)
    stream = torch.cuda.current_stream(dev)
    ms = _event_ms(torch, stream, lambda: net.train_steps(x, t, rows, [1e-3] * 64))
    ctx.sync()
    flops = 6 * 1024 * sum(widths[l] * widths[l + 1] for l in range(len(widths) - 1)) * 64
    print(json.dumps({"train_ms_per_step": ms / 64, "train_tflops": flops / (ms / 1e3) / 1e12}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-aux", action="store_true", help="skip the transmission/surrogate/retrieval legs")
    ap.add_argument("--train-steps", type=int, default=12000)
    ap.add_argument("--generations", type=int, default=20000)
    ap.add_argument("--burn", type=int, default=3000, help="exact-model burn-in generations before the retrieval legs")
    ap.add_argument("--screen-beta", type=float, default=1.0)
    ap.add_argument("--screen-margin", type=float, default=1.0)
    ap.add_argument("--case", choices=["bench", "profile", "transmission", "generation", "mlp"], default="bench",
                    help="profile: small launches of the hot kernels for ncu; transmission: the "
                         "1,024-instance transmission batch alone; generation: the fused 2,048-proposal "
                         "generation alone on a full-size grid of seeded values; mlp: 64 surrogate training "
                         "steps")
    ap.add_argument("--tile", type=int, default=0, help="emission tile width for --case profile/generation "
                                                          "(0: default / autotuner)")
    args = ap.parse_args()
    if args.case == "profile":
        return run_profile_case(args)
    if args.case == "generation":
        return run_generation_case(args)
    if args.case == "mlp":
        return run_mlp_case(args)
    if args.case == "transmission":
        return run_transmission_case(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())

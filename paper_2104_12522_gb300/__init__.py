"""GB300 (sm_103a) forward-model library for the BART retrieval method.

Thin Python binding over the C ABI of ``include/bartgpu.h`` (libbartgpu.so,
built in-tree by ``paper_2104_12522_gb300.build``).  It only marshals
arguments: torch tensors supply device memory and the CUDA stream, and every
step of the computation runs in the library's kernels.  Entry points keep the
C names without the ``bart_`` prefix.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import json
import sys
from typing import Optional, Sequence

import numpy as np

from . import _native
from ._native import (BART_EMISSION, BART_TRANSMISSION, BART_LAUNCH_FUSED, BART_LAUNCH_SPLIT,  # noqa: F401
                      BART_LAUNCH_FUSED_TMA)

__all__ = ["Context", "Graph", "BartError", "DeviceLines", "device_lines", "NuGrid", "Mlp", "Demc",
           "forward_emission_noalloc", "BART_EMISSION",
           "BART_TRANSMISSION", "BART_LAUNCH_FUSED", "BART_LAUNCH_SPLIT", "BART_LAUNCH_FUSED_TMA"]


class BartError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_native.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


@dataclasses.dataclass
class DeviceLines:
    """One species' line list in device memory (see bart_linelist)."""
    nu0: "torch.Tensor"         # float64
    log10_s296: "torch.Tensor"  # float32
    elow: "torch.Tensor"        # float32
    gamma_ref: "torch.Tensor"   # float32
    mass_amu: float

    def c_struct(self) -> _native.LineList:
        n = int(self.nu0.numel())
        for t, dt in ((self.nu0, "float64"), (self.log10_s296, "float32"), (self.elow, "float32"),
                      (self.gamma_ref, "float32")):
            _check_tensor(t, dt, n)
        return _native.LineList(n, _ptr(self.nu0), _ptr(self.log10_s296), _ptr(self.elow),
                                _ptr(self.gamma_ref), float(self.mass_amu))


def device_lines(lines, device="cuda") -> DeviceLines:
    """Copy a host line list (fields nu0, log10_s296, elow, gamma_ref, mass_amu) to the device."""
    import torch
    return DeviceLines(torch.as_tensor(np.ascontiguousarray(lines.nu0, np.float64), device=device),
                       torch.as_tensor(np.ascontiguousarray(lines.log10_s296, np.float32), device=device),
                       torch.as_tensor(np.ascontiguousarray(lines.elow, np.float32), device=device),
                       torch.as_tensor(np.ascontiguousarray(lines.gamma_ref, np.float32), device=device),
                       float(lines.mass_amu))


def NuGrid(nu_start: float, dnu: float, n_nu: int) -> _native.NuGrid:
    return _native.NuGrid(float(nu_start), float(dnu), int(n_nu))


def _release(obj):
    """Frees a library object when it is garbage-collected, except while the
    interpreter shuts down: the CUDA runtime may already be torn down then, and
    the process exit returns the device memory anyway."""
    if sys.is_finalizing():
        return
    try:
        obj.close()
    except Exception:
        pass


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _check_tensor(t, dtype: str, numel: Optional[int] = None):
    if t is None:
        return
    if str(t.dtype) != "torch." + dtype:
        raise TypeError(f"expected {dtype} tensor, got {t.dtype}")
    if not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")


def _grid_cfg(grid, p_bar, t_K, nu, cfg):
    """bart_grid_desc and bart_fwd_cfg for a device grid [S][L][M][n_nu]; the
    third value keeps the host arrays alive for the call."""
    S, L, M, N = (int(v) for v in grid.shape)
    pb, tk, x0 = _dbl(p_bar), _dbl(t_K), _dbl(cfg["x0"])
    gd = _native.GridDesc(_ptr(grid), S, L, M, C.cast(pb, C.c_void_p), C.cast(tk, C.c_void_p), nu)
    fc = _native.FwdCfg(int(cfg.get("geometry", 0)), int(cfg.get("n_angles", 4)), float(cfg["g"]),
                        float(cfg["mu"]), float(cfg.get("t_int", 100.0)), float(cfg.get("t_star", 5000.0)),
                        float(cfg.get("r_star_tp", 0.0)), float(cfg.get("a_orbit", 0.0)),
                        float(cfg.get("t_min", 0.0)), float(cfg.get("t_max", 1e30)),
                        float(cfg.get("p_ref", 0.1)), float(cfg.get("p_top", 1e-8)),
                        float(cfg.get("p_bot", 100.0)), C.cast(x0, C.c_void_p), float(cfg.get("tau_max", 0.0)),
                        float(cfg.get("p_cloud", 0.0) or 0.0), float(cfg.get("rayleigh_coef", 0.0)))
    return gd, fc, (pb, tk, x0)


def _dbl(a) -> C.Array:
    a = np.ascontiguousarray(a, np.float64)
    return (C.c_double * a.size)(*a.tolist())


class Graph:
    """A captured sequence of library calls (bart_graph), replayed on its
    context's stream by launch()."""

    def __init__(self, ctx: "Context", handle: C.c_void_p):
        self.ctx, self.h = ctx, handle

    def launch(self):
        self.ctx._check(self.ctx.lib.bart_graph_launch(self.ctx.h, self.h))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.bart_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        _release(self)


class Context:
    """A library context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.lib = _native.load()
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = C.c_void_p()
        st = self.lib.bart_create(C.byref(h), self.device, C.c_void_p(stream.cuda_stream))
        if st != 0:
            raise BartError(st, "bart_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.bart_destroy(self.h)
            self.h = None

    def __del__(self):
        _release(self)

    def _check(self, st: int):
        if st != 0:
            raise BartError(st, self.lib.bart_last_error(self.h).decode())

    def sync(self):
        self._check(self.lib.bart_sync(self.h))

    def set_autotune(self, enable: bool):
        self._check(self.lib.bart_set_autotune(self.h, int(bool(enable))))

    def set_emission_tile(self, tile: int):
        """Fix the emission wavenumber-tile width (64, 128, 256); 0 = autotuner."""
        self._check(self.lib.bart_set_emission_tile(self.h, int(tile)))

    def set_emission_launch(self, mode: int):
        """BART_LAUNCH_FUSED (0, one persistent kernel), BART_LAUNCH_SPLIT (1, three launches) or
        BART_LAUNCH_FUSED_TMA (2, the fused kernel with bulk-copy staging of the grid rows)."""
        self._check(self.lib.bart_set_emission_launch(self.h, int(mode)))

    def capture(self, fn) -> "Graph":
        """Capture the library calls fn() makes on this context into a CUDA
        graph (bart_capture_begin / bart_capture_end); fn must have run eagerly
        once with the same shapes and arguments."""
        self._check(self.lib.bart_capture_begin(self.h))
        err = None
        try:
            fn()
        except Exception as e:          # close the capture either way
            err = e
        g = C.c_void_p()
        st = self.lib.bart_capture_end(self.h, C.byref(g))
        if err is not None:
            raise err
        self._check(st)
        return Graph(self, g)

    def set_line_threshold(self, rel: float):
        """Line-strength lower bound for later opacity builds (relative to the
        strongest line of each species at each cell; <= 0 turns it off)."""
        self._check(self.lib.bart_set_line_threshold(self.h, float(rel)))

    def autotune_report(self) -> dict:
        """Autotuned tile width per launch shape."""
        n = self.lib.bart_autotune_report(self.h, None, 0)
        buf = C.create_string_buffer(n + 1)
        self.lib.bart_autotune_report(self.h, buf, n + 1)
        out = {}
        for line in buf.value.decode().splitlines():
            k, v = line.rsplit(" -> ", 1)
            out[k] = int(v)
        return out

    # ------------------------------------------------------------ opacity
    def faddeeva_re(self, x, y, out=None):
        import torch
        _check_tensor(x, "float32")
        _check_tensor(y, "float32", x.numel())
        if out is None:
            out = torch.empty_like(x)
        _check_tensor(out, "float32", x.numel())
        self._check(self.lib.bart_faddeeva_re(self.h, _ptr(x), _ptr(y), x.numel(), _ptr(out)))
        return out

    def _lists(self, species: Sequence[DeviceLines]):
        arr = (_native.LineList * len(species))(*[s.c_struct() for s in species])
        return arr

    def opacity_cells(self, species, p_bar, t_K, nu, cutoff, out=None):
        import torch
        p = np.asarray(p_bar, np.float64)
        t = np.asarray(t_K, np.float64)
        if p.shape != t.shape or p.ndim != 1:
            raise ValueError("p_bar and t_K must be 1-D of equal length")
        shape = (len(species), p.size, int(nu.n_nu))
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=species[0].nu0.device)
        _check_tensor(out, "float32", int(np.prod(shape)))
        self._check(self.lib.bart_opacity_cells(self.h, self._lists(species), len(species), _dbl(p), _dbl(t),
                                                p.size, nu, float(cutoff), _ptr(out)))
        return out

    def build_opacity_grid(self, species, p_bar, t_K, nu, cutoff, out=None):
        import torch
        p = np.asarray(p_bar, np.float64)
        t = np.asarray(t_K, np.float64)
        shape = (len(species), p.size, t.size, int(nu.n_nu))
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=species[0].nu0.device)
        _check_tensor(out, "float32", int(np.prod(shape)))
        self._check(self.lib.bart_build_opacity_grid(self.h, self._lists(species), len(species), _dbl(p),
                                                     p.size, _dbl(t), t.size, nu, float(cutoff), _ptr(out)))
        return out

    def opacity_cells_table(self, table, species, p_bar, t_K, nu, cutoff, out=None):
        """bart_opacity_cells_table: the paper's Voigt-table scheme."""
        import torch
        p = np.asarray(p_bar, np.float64)
        t = np.asarray(t_K, np.float64)
        if p.shape != t.shape or p.ndim != 1:
            raise ValueError("p_bar and t_K must be 1-D of equal length")
        shape = (len(species), p.size, int(nu.n_nu))
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=species[0].nu0.device)
        _check_tensor(out, "float32", int(np.prod(shape)))
        self._check(self.lib.bart_opacity_cells_table(self.h, table.h, self._lists(species), len(species), _dbl(p),
                                                      _dbl(t), p.size, nu, float(cutoff), _ptr(out)))
        return out

    def build_opacity_grid_table(self, table, species, p_bar, t_K, nu, cutoff, out=None):
        """bart_build_opacity_grid_table: the grid with the paper's Voigt-table scheme."""
        import torch
        p = np.asarray(p_bar, np.float64)
        t = np.asarray(t_K, np.float64)
        shape = (len(species), p.size, t.size, int(nu.n_nu))
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, device=species[0].nu0.device)
        _check_tensor(out, "float32", int(np.prod(shape)))
        self._check(self.lib.bart_build_opacity_grid_table(self.h, table.h, self._lists(species), len(species),
                                                           _dbl(p), p.size, _dbl(t), t.size, nu, float(cutoff),
                                                           _ptr(out)))
        return out

    # ------------------------------------------------------------ forward model
    def forward_spectra_batch(self, grid, p_bar, t_K, nu, cfg: dict, theta=None, t_profile=None,
                              n_levels=None, nu_lo=None, nu_hi=None, spec_offsets=None, r_planet=None,
                              r_star=None, spectra=None, filters=None, bands=None, n=None, active=None):
        """Spectra and/or band values of a batch; see bart_forward_spectra_batch.

        `grid` is the device opacity grid [S][L][M][n_nu]; `cfg` holds the
        bart_fwd_cfg fields by name (x0 as a sequence)."""
        S, L, M, N = (int(v) for v in grid.shape)
        _check_tensor(grid, "float32")
        for t, dt in ((theta, "float32"), (t_profile, "float32"), (n_levels, "int32"), (nu_lo, "int64"),
                      (nu_hi, "int64"), (spec_offsets, "int64"), (r_planet, "float32"), (r_star, "float32"),
                      (spectra, "float32"), (filters, "float32"), (bands, "float32"), (active, "int32")):
            _check_tensor(t, dt)
        if n is None:
            n = int(theta.shape[0]) if theta is not None else int(t_profile.shape[0])
        if theta is not None and tuple(theta.shape) != (n, 5 + S):
            raise ValueError(f"theta must be [{n}][{5 + S}]")
        if t_profile is not None and tuple(t_profile.shape) != (n, L):
            raise ValueError(f"t_profile must be [{n}][{L}]")
        for t, want in ((n_levels, n), (nu_lo, n), (nu_hi, n), (spec_offsets, n + 1), (r_planet, n),
                        (r_star, n), (active, n)):
            if t is not None and t.numel() != want:
                raise ValueError(f"per-entry array has {t.numel()} elements, expected {want}")
        if bands is not None and (filters is None or tuple(bands.shape) != (n, int(filters.shape[0]))):
            raise ValueError("bands must be [n][n_bands] and need filters")
        if filters is not None and tuple(filters.shape[1:]) != (N,):
            raise ValueError("filters must be [n_bands][n_nu]")
        gd, fc, keep = _grid_cfg(grid, p_bar, t_K, nu, cfg)
        b = _native.Batch(int(n), _ptr(theta), _ptr(t_profile), _ptr(n_levels), _ptr(nu_lo), _ptr(nu_hi),
                          _ptr(spec_offsets), _ptr(r_planet), _ptr(r_star), _ptr(active))
        fl = None
        if filters is not None:
            fl = _native.Filters(int(filters.shape[0]), _ptr(filters))
        self._check(self.lib.bart_forward_spectra_batch(self.h, C.byref(gd), C.byref(fc), C.byref(b),
                                                        _ptr(spectra), C.byref(fl) if fl else None,
                                                        _ptr(bands)))
        return spectra, bands

    def contribution_functions(self, grid, p_bar, t_K, nu, cfg: dict, theta=None, t_profile=None, nu_lo=None,
                               nu_hi=None, contrib=None, filters=None, bands=None, n=None, active=None):
        """Per-layer contribution functions of emission spectra; see
        bart_contribution_functions.  contrib [n][L][n_nu] and/or bands
        [n][L][n_bands] (device, float32)."""
        S, L, M, N = (int(v) for v in grid.shape)
        _check_tensor(grid, "float32")
        for t, dt in ((theta, "float32"), (t_profile, "float32"), (nu_lo, "int64"), (nu_hi, "int64"),
                      (contrib, "float32"), (filters, "float32"), (bands, "float32"), (active, "int32")):
            _check_tensor(t, dt)
        if n is None:
            n = int(theta.shape[0]) if theta is not None else int(t_profile.shape[0])
        if theta is not None and tuple(theta.shape) != (n, 5 + S):
            raise ValueError(f"theta must be [{n}][{5 + S}]")
        if t_profile is not None and tuple(t_profile.shape) != (n, L):
            raise ValueError(f"t_profile must be [{n}][{L}]")
        for t in (nu_lo, nu_hi, active):
            if t is not None and t.numel() != n:
                raise ValueError(f"per-entry array has {t.numel()} elements, expected {n}")
        if contrib is not None and tuple(contrib.shape) != (n, L, N):
            raise ValueError(f"contrib must be [{n}][{L}][{N}]")
        if bands is not None and (filters is None or tuple(bands.shape) != (n, L, int(filters.shape[0]))):
            raise ValueError("bands must be [n][n_layers][n_bands] and need filters")
        if filters is not None and tuple(filters.shape[1:]) != (N,):
            raise ValueError("filters must be [n_bands][n_nu]")
        gd, fc, keep = _grid_cfg(grid, p_bar, t_K, nu, cfg)
        b = _native.Batch(int(n), _ptr(theta), _ptr(t_profile), None, _ptr(nu_lo), _ptr(nu_hi), None, None, None,
                          _ptr(active))
        fl = _native.Filters(int(filters.shape[0]), _ptr(filters)) if filters is not None else None
        self._check(self.lib.bart_contribution_functions(self.h, C.byref(gd), C.byref(fc), C.byref(b),
                                                         _ptr(contrib), C.byref(fl) if fl else None, _ptr(bands)))
        return contrib, bands

    def retrieval_run(self, demc, surrogate, grid, p_bar, t_K, nu, cfg, filters, data, sigma, n_generations,
                      first_half_step=0, use_graph=True, chain=None):
        """bart_retrieval_run; returns the statistics as a dict."""
        for t, dt in ((grid, "float32"), (filters, "float32"), (data, "float32"), (sigma, "float32"),
                      (chain, "float32")):
            _check_tensor(t, dt)
        gd, fc, keep = _grid_cfg(grid, p_bar, t_K, nu, cfg)
        fl = _native.Filters(int(filters.shape[0]), _ptr(filters))
        st = _native.RetrievalStats()
        self._check(self.lib.bart_retrieval_run(self.h, demc.h, surrogate.h if surrogate is not None else None,
                                                C.byref(gd), C.byref(fc), C.byref(fl), _ptr(data), _ptr(sigma),
                                                int(first_half_step), int(n_generations), int(bool(use_graph)),
                                                _ptr(chain), C.byref(st)))
        return {k: getattr(st, k) for k, _ in _native.RetrievalStats._fields_}

    def chain_stats(self, chain, threshold=0.01, speis=True, gr=True):
        """SPEIS [C][d], Gelman-Rubin R [d] and ESS of chain [n][C][d] (device)."""
        import torch
        n, Cn, d = (int(v) for v in chain.shape)
        _check_tensor(chain, "float32", n * Cn * d)
        sp = torch.empty((Cn, d), dtype=torch.float64, device=chain.device) if speis else None
        g = torch.empty(d, dtype=torch.float64, device=chain.device) if gr else None
        self._check(self.lib.bart_chain_stats(self.h, _ptr(chain), n, Cn, d, float(threshold), _ptr(sp), _ptr(g)))
        ess = n * Cn / float(sp.mean(0).max()) if speis else None
        return sp, g, ess

    def loglike_bands(self, model, data, sigma, out, mask=None):
        """out[i] = -1/2 sum_b ((model[i][b] - data[b]) / sigma[b])^2 (FP64)."""
        n, nb = (int(v) for v in model.shape)
        for t, dt in ((model, "float32"), (data, "float32"), (sigma, "float32"), (mask, "int32"),
                      (out, "float64")):
            _check_tensor(t, dt)
        self._check(self.lib.bart_loglike_bands(self.h, _ptr(model), n, nb, _ptr(data), _ptr(sigma), _ptr(mask),
                                                _ptr(out)))
        return out

    def band_integrate(self, spectra, filters, nu, out, n_spec, spec_offsets=None, nu_lo=None, nu_hi=None):
        for t, dt in ((spectra, "float32"), (filters, "float32"), (out, "float32"), (spec_offsets, "int64"),
                      (nu_lo, "int64"), (nu_hi, "int64")):
            _check_tensor(t, dt)
        fl = _native.Filters(int(filters.shape[0]), _ptr(filters))
        self._check(self.lib.bart_band_integrate(self.h, _ptr(spectra), _ptr(spec_offsets), _ptr(nu_lo),
                                                 _ptr(nu_hi), int(n_spec), nu, C.byref(fl), _ptr(out)))
        return out


def _flt(a) -> C.Array:
    a = np.ascontiguousarray(a, np.float32)
    return (C.c_float * a.size)(*a.tolist())


class Mlp:
    """Surrogate network (bart_mlp_*) bound to a Context."""

    def __init__(self, ctx: Context, widths, bf16_weights=True, log_outputs=True, max_batch=4096):
        self.ctx = ctx
        self.lib = ctx.lib
        self.widths = [int(w) for w in widths]
        w = (C.c_int32 * len(self.widths))(*self.widths)
        h = C.c_void_p()
        ctx._check(self.lib.bart_mlp_create(ctx.h, w, len(self.widths), int(bool(bf16_weights)),
                                            int(bool(log_outputs)), int(max_batch), C.byref(h)))
        self.h = h
        self.n_params = int(self.lib.bart_mlp_num_params(h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.bart_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        _release(self)

    def set_scaling(self, in_shift, in_scale, out_shift, out_scale):
        self.ctx._check(self.lib.bart_mlp_set_scaling(self.h, _flt(in_shift), _flt(in_scale), _flt(out_shift),
                                                      _flt(out_scale)))

    def set_params(self, params):
        _check_tensor(params, "float32", self.n_params)
        self.ctx._check(self.lib.bart_mlp_set_params(self.h, _ptr(params)))

    def get_params(self, out=None):
        import torch
        if out is None:
            out = torch.empty(self.n_params, dtype=torch.float32, device=f"cuda:{self.ctx.device}")
        _check_tensor(out, "float32", self.n_params)
        self.ctx._check(self.lib.bart_mlp_get_params(self.h, _ptr(out)))
        return out

    def forward(self, x, out=None):
        import torch
        _check_tensor(x, "float32")
        B = int(x.shape[0])
        if out is None:
            out = torch.empty((B, self.widths[-1]), dtype=torch.float32, device=x.device)
        _check_tensor(out, "float32", B * self.widths[-1])
        self.ctx._check(self.lib.bart_mlp_forward(self.h, _ptr(x), B, _ptr(out)))
        return out

    def gradient(self, x, t, grad=None, loss=None):
        import torch
        _check_tensor(x, "float32")
        _check_tensor(t, "float32", int(x.shape[0]) * self.widths[-1])
        if grad is None:
            grad = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check_tensor(grad, "float32", self.n_params)
        _check_tensor(loss, "float32", 1)
        self.ctx._check(self.lib.bart_mlp_gradient(self.h, _ptr(x), _ptr(t), int(x.shape[0]), _ptr(grad),
                                                   _ptr(loss)))
        return grad, loss

    def train_step(self, x, t, lr, loss=None):
        _check_tensor(x, "float32")
        _check_tensor(t, "float32", int(x.shape[0]) * self.widths[-1])
        _check_tensor(loss, "float32", 1)
        self.ctx._check(self.lib.bart_mlp_train_step(self.h, _ptr(x), _ptr(t), int(x.shape[0]), float(lr),
                                                     _ptr(loss)))
        return loss

    def train_steps(self, x, t, batch_rows, lr, loss=None):
        """bart_mlp_train_steps: len(lr) Adam steps, step k on rows
        batch_rows[k] (device int32 [n_steps][B]) of x and t."""
        n_steps, B = (int(v) for v in batch_rows.shape)
        _check_tensor(x, "float32")
        _check_tensor(t, "float32", int(x.shape[0]) * self.widths[-1])
        _check_tensor(batch_rows, "int32")
        _check_tensor(loss, "float32")
        if len(lr) != n_steps:
            raise ValueError("one learning rate per step")
        lrs = _flt(lr)
        self.ctx._check(self.lib.bart_mlp_train_steps(self.h, _ptr(x), _ptr(t), int(x.shape[0]), _ptr(batch_rows), B,
                                                      n_steps, lrs, _ptr(loss)))
        return loss


class VoigtTable:
    """Precomputed Voigt profiles of the paper's table scheme (bart_voigt_table_*)
    on a context's device; widths in cm^-1, log-spaced between the bounds."""

    def __init__(self, ctx: Context, n_sigma, sigma_lo, sigma_hi, n_gamma, gamma_lo, gamma_hi, oversample, dnu,
                 cutoff):
        self.ctx, self.lib = ctx, ctx.lib
        h = C.c_void_p()
        ctx._check(self.lib.bart_voigt_table_create(ctx.h, int(n_sigma), float(sigma_lo), float(sigma_hi),
                                                    int(n_gamma), float(gamma_lo), float(gamma_hi), int(oversample),
                                                    float(dnu), float(cutoff), C.byref(h)))
        self.h = h
        self.spec = dict(n_sigma=int(n_sigma), sigma_lo=float(sigma_lo), sigma_hi=float(sigma_hi),
                         n_gamma=int(n_gamma), gamma_lo=float(gamma_lo), gamma_hi=float(gamma_hi),
                         oversample=int(oversample))

    @property
    def nbytes(self) -> int:
        return int(self.lib.bart_voigt_table_bytes(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.bart_voigt_table_destroy(self.h)
            self.h = None

    def __del__(self):
        _release(self)


class Demc:
    """Differential-evolution sampler state (bart_demc_*) bound to a Context."""

    def __init__(self, ctx: Context, n_chains, lo, hi, gamma=0.0, jump_every=10, eps=1e-4, seed=6000):
        self.ctx, self.lib = ctx, ctx.lib
        self.C, self.d = int(n_chains), len(lo)
        h = C.c_void_p()
        ctx._check(self.lib.bart_demc_create(ctx.h, self.C, self.d, _flt(lo), _flt(hi), float(gamma),
                                             int(jump_every), float(eps), C.c_uint64(int(seed)), C.byref(h)))
        self.h = h
        self._config = dict(n_chains=self.C, lo=[float(v) for v in np.asarray(lo, np.float32)],
                            hi=[float(v) for v in np.asarray(hi, np.float32)], gamma=float(gamma),
                            jump_every=int(jump_every), eps=float(eps), seed=int(seed), beta=1.0, margin=0.0)
        self._zs = False

    def close(self):
        if getattr(self, "h", None):
            self.lib.bart_demc_destroy(self.h)
            self.h = None

    def __del__(self):
        _release(self)

    def set_state(self, x, loglike, loglike_s=None):
        _check_tensor(x, "float32", self.C * self.d)
        _check_tensor(loglike, "float64", self.C)
        _check_tensor(loglike_s, "float64", self.C)
        self.ctx._check(self.lib.bart_demc_set_state(self.h, _ptr(x), _ptr(loglike), _ptr(loglike_s)))

    def get_state(self, x=None, loglike=None, loglike_s=None):
        _check_tensor(x, "float32", self.C * self.d)
        _check_tensor(loglike, "float64", self.C)
        _check_tensor(loglike_s, "float64", self.C)
        self.ctx._check(self.lib.bart_demc_get_state(self.h, _ptr(x), _ptr(loglike), _ptr(loglike_s)))
        return x, loglike, loglike_s

    def set_archive(self, z0, capacity, thin=10, p_snooker=0.1):
        """Switch to DEMCzs with the initial archive z0 (device [n0][d])."""
        n0 = int(z0.shape[0])
        _check_tensor(z0, "float32", n0 * self.d)
        self.ctx._check(self.lib.bart_demc_set_archive(self.h, _ptr(z0), n0, int(capacity), int(thin),
                                                       float(p_snooker)))
        self._zs = True

    def archive_size(self) -> int:
        n = C.c_int64()
        self.ctx._check(self.lib.bart_demc_archive_size(self.h, C.byref(n)))
        return int(n.value)

    def set_screen(self, beta=1.0, margin=0.0):
        self.ctx._check(self.lib.bart_demc_set_screen(self.h, float(beta), float(margin)))
        self._config.update(beta=float(beta), margin=float(margin))

    def checkpoint(self, next_half_step: int) -> dict:
        """Everything a DE-MC run needs to continue, as host values: the
        sampler's configuration, seed and screen, the chains' states with their
        exact and surrogate log-likelihoods, and the half-step to run next.
        Random numbers are keyed by (seed, half-step, chain, draw), so a sampler
        rebuilt by from_checkpoint continues exactly as this one would.  A
        DEMCzs archive is device state the library does not export, so a
        DEMCzs sampler raises instead."""
        import torch
        if self._zs:
            raise ValueError("the archive of a DEMCzs sampler cannot be checkpointed")
        dev = torch.device("cuda", self.ctx.device)
        x = torch.empty((self.C, self.d), dtype=torch.float32, device=dev)
        L = torch.empty(self.C, dtype=torch.float64, device=dev)
        Ls = torch.empty(self.C, dtype=torch.float64, device=dev)
        self.get_state(x, L, Ls)
        self.ctx.sync()
        return dict(self._config, x=x.cpu().numpy(), loglike=L.cpu().numpy(), loglike_s=Ls.cpu().numpy(),
                    next_half_step=int(next_half_step))

    @classmethod
    def from_checkpoint(cls, ctx: Context, ck: dict) -> "Demc":
        """A sampler in the state `ck` describes (see checkpoint); the run
        continues with half-step ck["next_half_step"]."""
        import torch
        s = cls(ctx, int(ck["n_chains"]), np.asarray(ck["lo"], np.float32), np.asarray(ck["hi"], np.float32),
                gamma=float(ck["gamma"]), jump_every=int(ck["jump_every"]), eps=float(ck["eps"]),
                seed=int(ck["seed"]))
        s.set_screen(float(ck["beta"]), float(ck["margin"]))
        dev = torch.device("cuda", ctx.device)
        s.set_state(torch.tensor(np.ascontiguousarray(ck["x"], np.float32), device=dev),
                    torch.tensor(np.ascontiguousarray(ck["loglike"], np.float64), device=dev),
                    torch.tensor(np.ascontiguousarray(ck["loglike_s"], np.float64), device=dev))
        return s

    def propose(self, half_step, y, inbox):
        _check_tensor(y, "float32", self.C * self.d)
        _check_tensor(inbox, "int32", self.C)
        self.ctx._check(self.lib.bart_demc_propose(self.h, int(half_step), _ptr(y), _ptr(inbox)))

    def screen(self, half_step, inbox, ls_y, passed):
        _check_tensor(inbox, "int32", self.C)
        _check_tensor(ls_y, "float64", self.C)
        _check_tensor(passed, "int32", self.C)
        self.ctx._check(self.lib.bart_demc_screen(self.h, int(half_step), _ptr(inbox), _ptr(ls_y), _ptr(passed)))

    def accept(self, half_step, y, passed, L_y, ls_y=None, accepted=None):
        _check_tensor(y, "float32", self.C * self.d)
        _check_tensor(passed, "int32", self.C)
        _check_tensor(L_y, "float64", self.C)
        _check_tensor(ls_y, "float64", self.C)
        _check_tensor(accepted, "int32", self.C)
        self.ctx._check(self.lib.bart_demc_accept(self.h, int(half_step), _ptr(y), _ptr(passed), _ptr(L_y),
                                                  _ptr(ls_y), _ptr(accepted)))


def save_checkpoint(path: str, ck: dict) -> None:
    """Writes a sampler checkpoint (Demc.checkpoint) to `path` (.npz)."""
    arrays = {k: np.asarray(ck[k]) for k in ("x", "loglike", "loglike_s")}
    meta = {k: v for k, v in ck.items() if k not in arrays}
    np.savez(path, meta=np.array(json.dumps(meta)), **arrays)


def load_checkpoint(path: str) -> dict:
    """Reads a sampler checkpoint written by save_checkpoint."""
    with np.load(path, allow_pickle=False) as f:
        ck = json.loads(str(f["meta"]))
        ck.update({k: f[k].copy() for k in ("x", "loglike", "loglike_s")})
    return ck


def forward_emission_noalloc(grid, p_bar, t_K, nu, cfg, theta=None, t_profile=None, nu_lo=None, nu_hi=None,
                             spec_offsets=None, spectra=None, filters=None, bands=None, n=None, active=None,
                             stream=None):
    """bart_forward_emission_noalloc: the emission forward model without any
    device allocation (fixed scratch in the library); returns the status code."""
    import torch
    lib = _native.load()
    for t, dt in ((grid, "float32"), (theta, "float32"), (t_profile, "float32"), (nu_lo, "int64"),
                  (nu_hi, "int64"), (spec_offsets, "int64"), (spectra, "float32"), (filters, "float32"),
                  (bands, "float32"), (active, "int32")):
        _check_tensor(t, dt)
    if n is None:
        n = int(theta.shape[0]) if theta is not None else int(t_profile.shape[0])
    gd, fc, keep = _grid_cfg(grid, p_bar, t_K, nu, cfg)
    b = _native.Batch(int(n), _ptr(theta), _ptr(t_profile), None, _ptr(nu_lo), _ptr(nu_hi), _ptr(spec_offsets),
                      None, None, _ptr(active))
    fl = _native.Filters(int(filters.shape[0]), _ptr(filters)) if filters is not None else None
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(lib.bart_forward_emission_noalloc(C.c_void_p(stream.cuda_stream), C.byref(gd), C.byref(fc),
                                                 C.byref(b), _ptr(spectra), C.byref(fl) if fl else None,
                                                 _ptr(bands)))

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
from typing import Optional, Sequence

import numpy as np

from . import _native
from ._native import BART_EMISSION, BART_TRANSMISSION  # noqa: F401

__all__ = ["Context", "BartError", "DeviceLines", "device_lines", "NuGrid", "BART_EMISSION",
           "BART_TRANSMISSION"]


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


def _dbl(a) -> C.Array:
    a = np.ascontiguousarray(a, np.float64)
    return (C.c_double * a.size)(*a.tolist())


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
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise BartError(st, self.lib.bart_last_error(self.h).decode())

    def sync(self):
        self._check(self.lib.bart_sync(self.h))

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

    # ------------------------------------------------------------ forward model
    def forward_spectra_batch(self, grid, p_bar, t_K, nu, cfg: dict, theta=None, t_profile=None,
                              n_levels=None, nu_lo=None, nu_hi=None, spec_offsets=None, r_planet=None,
                              r_star=None, spectra=None, filters=None, bands=None, n=None):
        """Spectra and/or band values of a batch; see bart_forward_spectra_batch.

        `grid` is the device opacity grid [S][L][M][n_nu]; `cfg` holds the
        bart_fwd_cfg fields by name (x0 as a sequence)."""
        S, L, M, N = (int(v) for v in grid.shape)
        _check_tensor(grid, "float32")
        for t, dt in ((theta, "float32"), (t_profile, "float32"), (n_levels, "int32"), (nu_lo, "int64"),
                      (nu_hi, "int64"), (spec_offsets, "int64"), (r_planet, "float32"), (r_star, "float32"),
                      (spectra, "float32"), (filters, "float32"), (bands, "float32")):
            _check_tensor(t, dt)
        if n is None:
            n = int(theta.shape[0]) if theta is not None else int(t_profile.shape[0])
        if theta is not None and tuple(theta.shape) != (n, 5 + S):
            raise ValueError(f"theta must be [{n}][{5 + S}]")
        if t_profile is not None and tuple(t_profile.shape) != (n, L):
            raise ValueError(f"t_profile must be [{n}][{L}]")
        for t, want in ((n_levels, n), (nu_lo, n), (nu_hi, n), (spec_offsets, n + 1), (r_planet, n),
                        (r_star, n)):
            if t is not None and t.numel() != want:
                raise ValueError(f"per-entry array has {t.numel()} elements, expected {want}")
        if bands is not None and (filters is None or tuple(bands.shape) != (n, int(filters.shape[0]))):
            raise ValueError("bands must be [n][n_bands] and need filters")
        if filters is not None and tuple(filters.shape[1:]) != (N,):
            raise ValueError("filters must be [n_bands][n_nu]")
        pb, tk = _dbl(p_bar), _dbl(t_K)
        gd = _native.GridDesc(_ptr(grid), S, L, M, C.cast(pb, C.c_void_p), C.cast(tk, C.c_void_p), nu)
        x0 = _dbl(cfg["x0"])
        fc = _native.FwdCfg(int(cfg.get("geometry", 0)), int(cfg.get("n_angles", 4)), float(cfg["g"]),
                            float(cfg["mu"]), float(cfg.get("t_int", 100.0)), float(cfg.get("t_star", 5000.0)),
                            float(cfg.get("r_star_tp", 0.0)), float(cfg.get("a_orbit", 0.0)),
                            float(cfg.get("t_min", 0.0)), float(cfg.get("t_max", 1e30)),
                            float(cfg.get("p_ref", 0.1)), float(cfg.get("p_top", 1e-8)),
                            float(cfg.get("p_bot", 100.0)), C.cast(x0, C.c_void_p))
        b = _native.Batch(int(n), _ptr(theta), _ptr(t_profile), _ptr(n_levels), _ptr(nu_lo), _ptr(nu_hi),
                          _ptr(spec_offsets), _ptr(r_planet), _ptr(r_star))
        fl = None
        if filters is not None:
            fl = _native.Filters(int(filters.shape[0]), _ptr(filters))
        self._check(self.lib.bart_forward_spectra_batch(self.h, C.byref(gd), C.byref(fc), C.byref(b),
                                                        _ptr(spectra), C.byref(fl) if fl else None,
                                                        _ptr(bands)))
        return spectra, bands

    def band_integrate(self, spectra, filters, nu, out, n_spec, spec_offsets=None, nu_lo=None, nu_hi=None):
        for t, dt in ((spectra, "float32"), (filters, "float32"), (out, "float32"), (spec_offsets, "int64"),
                      (nu_lo, "int64"), (nu_hi, "int64")):
            _check_tensor(t, dt)
        fl = _native.Filters(int(filters.shape[0]), _ptr(filters))
        self._check(self.lib.bart_band_integrate(self.h, _ptr(spectra), _ptr(spec_offsets), _ptr(nu_lo),
                                                 _ptr(nu_hi), int(n_spec), nu, C.byref(fl), _ptr(out)))
        return out

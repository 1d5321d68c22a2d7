"""ctypes declarations mirroring include/bartgpu.h, and the library loader.

The loader raises if libbartgpu.so is missing or does not export a declared
symbol: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbartgpu.so")

c_void_p, c_int, c_int32, c_int64, c_double = C.c_void_p, C.c_int, C.c_int32, C.c_int64, C.c_double

BART_OK, BART_EINVAL, BART_ENOMEM, BART_ECUDA, BART_ETIMEOUT, BART_ERANGE, BART_EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "BART_OK", 1: "BART_EINVAL", 2: "BART_ENOMEM", 3: "BART_ECUDA",
                4: "BART_ETIMEOUT", 5: "BART_ERANGE", 6: "BART_EUNSUPPORTED"}
BART_EMISSION, BART_TRANSMISSION = 0, 1
BART_LAUNCH_FUSED, BART_LAUNCH_SPLIT, BART_LAUNCH_FUSED_TMA = 0, 1, 2


class LineList(C.Structure):
    _fields_ = [("n_lines", c_int64), ("nu0_cm", c_void_p), ("log10_s296", c_void_p),
                ("elow_cm", c_void_p), ("gamma_ref_cm", c_void_p), ("mass_amu", c_double)]


class NuGrid(C.Structure):
    _fields_ = [("nu_start_cm", c_double), ("dnu_cm", c_double), ("n_nu", c_int64)]


class GridDesc(C.Structure):
    _fields_ = [("grid", c_void_p), ("n_species", c_int), ("n_layers", c_int), ("n_temps", c_int),
                ("p_bar", c_void_p), ("t_K", c_void_p), ("nu", NuGrid)]


class FwdCfg(C.Structure):
    _fields_ = [("geometry", c_int32), ("n_angles", c_int32), ("g_cgs", c_double), ("mu_amu", c_double),
                ("t_int_K", c_double), ("t_star_K", c_double), ("r_star_tp_cm", c_double),
                ("a_orbit_cm", c_double), ("t_min_K", c_double), ("t_max_K", c_double),
                ("p_ref_bar", c_double), ("p_top_bar", c_double), ("p_bot_bar", c_double),
                ("x0", c_void_p), ("tau_max", c_double), ("p_cloud_bar", c_double),
                ("rayleigh_coef", c_double)]


class Batch(C.Structure):
    _fields_ = [("n", c_int32), ("theta", c_void_p), ("t_profile", c_void_p), ("n_levels", c_void_p),
                ("nu_lo", c_void_p), ("nu_hi", c_void_p), ("spec_offsets", c_void_p),
                ("r_planet_cm", c_void_p), ("r_star_cm", c_void_p), ("active", c_void_p)]


class Filters(C.Structure):
    _fields_ = [("n_bands", c_int32), ("weights", c_void_p)]


class RetrievalStats(C.Structure):
    _fields_ = [("proposals", c_int64), ("screened_out", c_int64), ("exact_evals", c_int64),
                ("accepted", c_int64), ("surrogate_err_sum", c_double), ("surrogate_err_max", c_double)]


P = C.POINTER
# name -> (restype, argtypes); kept in the order of include/bartgpu.h
SIGNATURES = {
    "bart_abi_version": (c_int, []),
    "bart_create": (c_int, [P(c_void_p), c_int, c_void_p]),
    "bart_destroy": (None, [c_void_p]),
    "bart_set_stream": (c_int, [c_void_p, c_void_p]),
    "bart_last_error": (C.c_char_p, [c_void_p]),
    "bart_sync": (c_int, [c_void_p]),
    "bart_set_autotune": (c_int, [c_void_p, c_int]),
    "bart_set_emission_tile": (c_int, [c_void_p, c_int]),
    "bart_set_emission_launch": (c_int, [c_void_p, c_int]),
    "bart_capture_begin": (c_int, [c_void_p]),
    "bart_capture_end": (c_int, [c_void_p, P(c_void_p)]),
    "bart_graph_launch": (c_int, [c_void_p, c_void_p]),
    "bart_graph_destroy": (None, [c_void_p]),
    "bart_set_line_threshold": (c_int, [c_void_p, c_double]),
    "bart_demc_set_archive": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int, c_double]),
    "bart_demc_archive_size": (c_int, [c_void_p, P(c_int64)]),
    "bart_chain_stats": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_double, c_void_p, c_void_p]),
    "bart_voigt_table_create": (c_int, [c_void_p, c_int, c_double, c_double, c_int, c_double, c_double, c_int,
                                        c_double, c_double, c_void_p]),
    "bart_voigt_table_destroy": (None, [c_void_p]),
    "bart_voigt_table_bytes": (c_int64, [c_void_p]),
    "bart_opacity_cells_table": (c_int, [c_void_p, c_void_p, P(LineList), c_int, P(c_double), P(c_double), c_int,
                                         NuGrid, c_double, c_void_p]),
    "bart_build_opacity_grid_table": (c_int, [c_void_p, c_void_p, P(LineList), c_int, P(c_double), c_int,
                                              P(c_double), c_int, NuGrid, c_double, c_void_p]),
    "bart_autotune_report": (c_int, [c_void_p, C.c_char_p, c_int]),
    "bart_opacity_cells": (c_int, [c_void_p, P(LineList), c_int, P(c_double), P(c_double), c_int, NuGrid,
                                   c_double, c_void_p]),
    "bart_build_opacity_grid": (c_int, [c_void_p, P(LineList), c_int, P(c_double), c_int, P(c_double), c_int,
                                        NuGrid, c_double, c_void_p]),
    "bart_faddeeva_re": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "bart_forward_spectra_batch": (c_int, [c_void_p, P(GridDesc), P(FwdCfg), P(Batch), c_void_p, P(Filters),
                                           c_void_p]),
    "bart_band_integrate": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, NuGrid,
                                    P(Filters), c_void_p]),
    "bart_contribution_functions": (c_int, [c_void_p, P(GridDesc), P(FwdCfg), P(Batch), c_void_p, P(Filters),
                                            c_void_p]),
    "bart_mlp_create": (c_int, [c_void_p, P(c_int32), c_int, c_int, c_int, c_int, P(c_void_p)]),
    "bart_mlp_destroy": (None, [c_void_p]),
    "bart_mlp_num_params": (c_int64, [c_void_p]),
    "bart_mlp_set_scaling": (c_int, [c_void_p, P(C.c_float), P(C.c_float), P(C.c_float), P(C.c_float)]),
    "bart_mlp_set_params": (c_int, [c_void_p, c_void_p]),
    "bart_mlp_get_params": (c_int, [c_void_p, c_void_p]),
    "bart_mlp_forward": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    "bart_mlp_gradient": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "bart_mlp_train_step": (c_int, [c_void_p, c_void_p, c_void_p, c_int, C.c_float, c_void_p]),
    "bart_mlp_train_steps": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int, c_int, P(C.c_float),
                                     c_void_p]),
    "bart_demc_create": (c_int, [c_void_p, c_int, c_int, P(C.c_float), P(C.c_float), c_double, c_int, c_double,
                                 C.c_uint64, P(c_void_p)]),
    "bart_demc_destroy": (None, [c_void_p]),
    "bart_demc_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "bart_demc_get_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "bart_demc_set_screen": (c_int, [c_void_p, c_double, c_double]),
    "bart_demc_propose": (c_int, [c_void_p, c_int64, c_void_p, c_void_p]),
    "bart_demc_screen": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
    "bart_demc_accept": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "bart_loglike_bands": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "bart_forward_emission_noalloc": (c_int, [c_void_p, P(GridDesc), P(FwdCfg), P(Batch), c_void_p, P(Filters),
                                              c_void_p]),
    "bart_retrieval_run": (c_int, [c_void_p, c_void_p, c_void_p, P(GridDesc), P(FwdCfg), P(Filters), c_void_p,
                                   c_void_p, c_int64, c_int, c_int, c_void_p, P(RetrievalStats)]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libbartgpu.so and bind every declared entry point (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2104_12522_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)          # AttributeError if the symbol is not exported
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_symbols(header: str) -> list[str]:
    """Names of the functions declared in a bartgpu header."""
    import re
    with open(header) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bart_[a-z0-9_]+)\s*\(", text)))

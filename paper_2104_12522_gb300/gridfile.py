"""Opacity grid files: the grid is built once and reused by later runs (Sec. 3:
the opacity table is pre-calculated, saved and then only interpolated).

A grid file is a pair beside each other:
  <stem>.bin   the FP32 little-endian array grid[S][L][M][n_nu] (cm^2/molecule),
  <stem>.json  a header: shape, the axes (layer pressures in bar, grid
               temperatures in K, the wavenumber grid nu_start + j dnu in
               cm^-1), the line cutoff, a provenance record supplied by the
               caller (line-list seeds and sizes, species masses, ...) and the
               SHA-256 of the data.
load_grid checks the data against the header (size and hash) and, when asked,
the header against expected axes and provenance, before it returns the grid
on the requested device.  Host-side I/O only: no kernel runs here."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

FORMAT = "bart-opacity-grid/1"


def _paths(stem: str) -> tuple[str, str]:
    return stem + ".bin", stem + ".json"


def save_grid(stem: str, grid, p_bar, t_K, nu_start: float, dnu: float, cutoff: float,
              provenance: dict | None = None) -> dict:
    """Writes <stem>.bin and <stem>.json for grid [S][L][M][n_nu] (a float32
    torch tensor on any device, or a numpy array); returns the header."""
    a = grid.detach().cpu().numpy() if hasattr(grid, "detach") else np.asarray(grid)
    if a.dtype != np.float32 or a.ndim != 4:
        raise ValueError("grid must be a float32 array [S][L][M][n_nu]")
    S, L, M, N = (int(v) for v in a.shape)
    p = [float(v) for v in np.asarray(p_bar, np.float64).ravel()]
    t = [float(v) for v in np.asarray(t_K, np.float64).ravel()]
    if len(p) != L or len(t) != M:
        raise ValueError(f"axes of length {len(p)} and {len(t)} do not match the grid's {L} layers and {M} temperatures")
    data = np.ascontiguousarray(a, dtype="<f4").tobytes()
    header = {"format": FORMAT, "shape": [S, L, M, N], "p_bar": p, "t_K": t,
              "nu": {"start": float(nu_start), "step": float(dnu), "n": N}, "cutoff_cm": float(cutoff),
              "provenance": provenance or {}, "sha256": hashlib.sha256(data).hexdigest()}
    bin_path, json_path = _paths(stem)
    with open(bin_path + ".tmp", "wb") as fh:
        fh.write(data)
    with open(json_path + ".tmp", "w") as fh:
        json.dump(header, fh, indent=1)
    os.replace(bin_path + ".tmp", bin_path)
    os.replace(json_path + ".tmp", json_path)
    return header


def load_grid(stem: str, device="cuda", expect: dict | None = None):
    """Reads a grid file; returns (grid tensor on `device`, header).  Raises
    ValueError if the data do not match the header (size or SHA-256), or if
    `expect` holds header entries (e.g. "p_bar", "t_K", "nu", "cutoff_cm",
    "provenance") that differ from the file's."""
    import torch
    bin_path, json_path = _paths(stem)
    with open(json_path) as fh:
        header = json.load(fh)
    if header.get("format") != FORMAT:
        raise ValueError(f"{json_path}: not a {FORMAT} header")
    S, L, M, N = header["shape"]
    with open(bin_path, "rb") as fh:
        data = fh.read()
    if len(data) != 4 * S * L * M * N:
        raise ValueError(f"{bin_path}: {len(data)} bytes, the header's shape needs {4 * S * L * M * N}")
    if hashlib.sha256(data).hexdigest() != header["sha256"]:
        raise ValueError(f"{bin_path}: data do not match the header's SHA-256")
    for key, want in (expect or {}).items():
        have = header.get(key)
        if key in ("p_bar", "t_K"):
            same = have is not None and len(have) == len(want) and np.array_equal(np.asarray(have, np.float64),
                                                                                    np.asarray(want, np.float64))
        else:
            same = have == want
        if not same:
            raise ValueError(f"{json_path}: {key} is {have!r}, expected {want!r}")
    arr = np.frombuffer(data, dtype="<f4").reshape(S, L, M, N).astype(np.float32)
    return torch.tensor(arr, device=device), header

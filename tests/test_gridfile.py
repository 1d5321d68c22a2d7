"""Opacity grid files (the grid built once and reused, Sec. 3): a saved grid
loads back bit for bit with its axes and provenance, and a file whose data or
header do not match is refused (CPU; the tensors stay on the host)."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2104_12522_gb300 import gridfile as GF   # noqa: E402
import workloads as W                                # noqa: E402


def _grid():
    ax = W.grid_axes(n_layers=7, n_temps=4, n_nu=333)
    g = W.opacity_field(2, ax.p_bar, ax.t_K, ax.n_nu, seed=3700)
    return ax, torch.tensor(g.astype(np.float32))


def test_round_trip_keeps_data_axes_and_provenance(tmp_path):
    ax, g = _grid()
    prov = {"line_list_seeds": [1000, 1001], "lines_per_species": [1666667, 1666667], "mass_amu": [18.0, 28.0]}
    stem = str(tmp_path / "grid")
    hdr = GF.save_grid(stem, g, ax.p_bar, ax.t_K, ax.nu_start, ax.dnu, ax.cutoff, provenance=prov)
    assert hdr["shape"] == [2, 7, 4, 333]
    got, h = GF.load_grid(stem, device="cpu",
                          expect={"p_bar": ax.p_bar, "t_K": ax.t_K, "cutoff_cm": 25.0, "provenance": prov,
                                  "nu": {"start": 1000.0, "step": 0.02, "n": 333}})
    assert got.dtype == torch.float32 and torch.equal(got, g)
    assert np.array_equal(h["p_bar"], ax.p_bar) and h["provenance"] == prov


def test_corrupted_or_truncated_data_is_refused(tmp_path):
    ax, g = _grid()
    stem = str(tmp_path / "grid")
    GF.save_grid(stem, g, ax.p_bar, ax.t_K, ax.nu_start, ax.dnu, ax.cutoff)
    with open(stem + ".bin", "r+b") as fh:
        fh.seek(4 * 1234)
        b = fh.read(1)
        fh.seek(4 * 1234)
        fh.write(bytes([b[0] ^ 0x01]))            # one flipped bit
    with pytest.raises(ValueError, match="SHA-256"):
        GF.load_grid(stem, device="cpu")
    GF.save_grid(stem, g, ax.p_bar, ax.t_K, ax.nu_start, ax.dnu, ax.cutoff)
    with open(stem + ".bin", "r+b") as fh:
        fh.truncate(4 * 100)
    with pytest.raises(ValueError, match="bytes"):
        GF.load_grid(stem, device="cpu")


def test_header_expectations_are_checked(tmp_path):
    ax, g = _grid()
    stem = str(tmp_path / "grid")
    GF.save_grid(stem, g, ax.p_bar, ax.t_K, ax.nu_start, ax.dnu, ax.cutoff, provenance={"seed": 1000})
    with pytest.raises(ValueError, match="t_K"):
        GF.load_grid(stem, device="cpu", expect={"t_K": ax.t_K + 1.0})
    with pytest.raises(ValueError, match="provenance"):
        GF.load_grid(stem, device="cpu", expect={"provenance": {"seed": 1001}})
    with open(stem + ".json") as fh:
        hdr = json.load(fh)
    hdr["format"] = "something-else"
    with open(stem + ".json", "w") as fh:
        json.dump(hdr, fh)
    with pytest.raises(ValueError, match="header"):
        GF.load_grid(stem, device="cpu")


def test_bad_grids_are_not_written(tmp_path):
    ax, g = _grid()
    with pytest.raises(ValueError):
        GF.save_grid(str(tmp_path / "a"), g.double(), ax.p_bar, ax.t_K, ax.nu_start, ax.dnu, ax.cutoff)
    with pytest.raises(ValueError):
        GF.save_grid(str(tmp_path / "b"), g, ax.p_bar[:-1], ax.t_K, ax.nu_start, ax.dnu, ax.cutoff)
    assert not (tmp_path / "a.bin").exists() and not (tmp_path / "b.json").exists()

"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/bartgpu.h (no compute call: this runs without a GPU)."""
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_12522_gb300 import build, _native
    build.build()
    return _native.load()


def test_exports_every_declared_symbol(lib):
    from paper_2104_12522_gb300 import _native
    declared = _native.header_symbols(os.path.join(ROOT, "include", "bartgpu.h"))
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(_native.SIGNATURES), "binding and header disagree"


def test_abi_version(lib):
    import ctypes as C
    import re
    from paper_2104_12522_gb300 import _native
    with open(os.path.join(ROOT, "include", "bartgpu.h")) as fh:
        version = int(re.search(r"#define BART_ABI_VERSION (\d+)", fh.read()).group(1))
    assert lib.bart_abi_version() == version == 4
    # version 2 appended tau_max, version 3 p_cloud_bar and rayleigh_coef to
    # bart_fwd_cfg: the binding's struct must match
    assert C.sizeof(_native.FwdCfg) == 2 * 4 + 11 * 8 + 8 + 3 * 8
    assert _native.FwdCfg.rayleigh_coef.offset == C.sizeof(_native.FwdCfg) - 8


def test_struct_layouts_match_the_header(tmp_path):
    # the C compiler's layout of every struct of the header against the binding's
    import ctypes as C
    import shutil
    import subprocess
    from paper_2104_12522_gb300 import _native
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"bart_linelist": _native.LineList, "bart_nugrid": _native.NuGrid, "bart_grid_desc": _native.GridDesc,
               "bart_fwd_cfg": _native.FwdCfg, "bart_batch": _native.Batch, "bart_filters": _native.Filters,
               "bart_retrieval_stats": _native.RetrievalStats}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "bartgpu.h"', "int main(void) {"]
    for name, cls in structs.items():
        src.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            src.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    src.append("  return 0;\n}")
    (tmp_path / "l.c").write_text("\n".join(src))
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-o", str(tmp_path / "l"), str(tmp_path / "l.c")],
                   check=True)
    out = dict(line.split() for line in subprocess.run([str(tmp_path / "l")], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_null_context_is_rejected(lib):
    import ctypes as C
    from paper_2104_12522_gb300 import _native
    assert lib.bart_sync(None) == _native.BART_EINVAL
    assert lib.bart_set_stream(None, None) == _native.BART_EINVAL
    assert lib.bart_last_error(None) == b"NULL context"
    lib.bart_destroy(None)
    assert lib.bart_create(None, 0, None) == _native.BART_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    from paper_2104_12522_gb300 import _native
    saved = _native._lib
    _native._lib = None
    try:
        with pytest.raises(RuntimeError, match="missing"):
            _native.load(str(tmp_path / "nope.so"))
    finally:
        _native._lib = saved

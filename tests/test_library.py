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
    assert lib.bart_abi_version() == version == 2
    # version 2 appended tau_max to bart_fwd_cfg: the binding's struct must match
    assert C.sizeof(_native.FwdCfg) == 2 * 4 + 11 * 8 + 8 + 8
    assert _native.FwdCfg.tau_max.offset == C.sizeof(_native.FwdCfg) - 8


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

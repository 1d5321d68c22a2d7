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


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor on a machine without one: only the
    attributes the binding's argument checks read."""

    def __init__(self, dtype, numel, contiguous=True):
        self.dtype, self._n, self._c = "torch." + dtype, numel, contiguous
        self.is_cuda, self.device = True, "cpu"     # device: where defaults are allocated

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n

    def data_ptr(self):
        raise AssertionError("the library was reached with a bad argument")


def test_sampler_and_surrogate_methods_check_their_arguments():
    # Wrong dtype, size or layout of an output or input buffer is rejected
    # in Python, before any pointer reaches the library.
    import pytest
    import paper_2104_12522_gb300 as bart
    F = _FakeDeviceTensor
    class _Stub:                      # context and library: any attribute, any call
        def __getattr__(self, name):
            return lambda *a: 0
    s = object.__new__(bart.Demc)
    s.C, s.d, s.ctx, s.lib, s.h = 6, 4, _Stub(), _Stub(), None
    good_y, good_i, good_l = F("float32", 24), F("int32", 6), F("float64", 6)
    bad = [
        lambda: s.propose(0, F("float64", 24), good_i),
        lambda: s.propose(0, good_y, F("int32", 5)),
        lambda: s.screen(0, good_i, F("float32", 6), good_i),
        lambda: s.screen(0, good_i, good_l, F("int64", 6)),
        lambda: s.accept(0, F("float32", 23), good_i, good_l),
        lambda: s.accept(0, good_y, good_i, F("float32", 6)),
        lambda: s.accept(0, good_y, good_i, good_l, good_l, F("int32", 7)),
        lambda: s.get_state(F("float32", 24, contiguous=False)),
        lambda: s.get_state(good_y, F("float64", 5)),
    ]
    m = object.__new__(bart.Mlp)
    m.widths, m.n_params, m.ctx, m.lib, m.h = [9, 4, 10], 90, _Stub(), _Stub(), None
    x = F("float32", 2 * 9)
    x.shape = (2, 9)
    t = F("float32", 2 * 10)
    bad += [
        lambda: m.gradient(x, t, grad=F("float32", 89)),
        lambda: m.gradient(x, t, grad=F("float32", 90), loss=F("float64", 1)),
        lambda: m.train_step(x, t, 1e-3, loss=F("float32", 2)),
    ]
    for call in bad:
        with pytest.raises((TypeError, ValueError)):
            call()
    # arguments of the documented dtypes and sizes pass the checks and reach
    # the library (the stand-in stops there)
    good = [
        lambda: s.propose(0, good_y, good_i),
        lambda: s.screen(0, good_i, good_l, good_i),
        lambda: s.screen(0, good_i, None, good_i),
        lambda: s.accept(0, good_y, good_i, good_l),
        lambda: s.accept(0, good_y, good_i, good_l, good_l, good_i),
        lambda: s.get_state(good_y),
        lambda: s.get_state(good_y, good_l, good_l),
        lambda: m.gradient(x, t, grad=F("float32", 90), loss=F("float32", 1)),
        lambda: m.train_step(x, t, 1e-3, loss=F("float32", 1)),
    ]
    for call in good:
        with pytest.raises(AssertionError, match="library was reached"):
            call()


def test_sampler_checkpoint_file_round_trip(tmp_path):
    import numpy as np
    import paper_2104_12522_gb300 as bart
    rng = np.random.default_rng(3)
    ck = dict(n_chains=8, lo=[0.0, -1.0], hi=[1.0, 2.0], gamma=0.0, jump_every=10, eps=1e-4, seed=6123,
              beta=0.5, margin=1.0, next_half_step=4242, x=rng.uniform(size=(8, 2)).astype(np.float32),
              loglike=rng.normal(size=8), loglike_s=np.zeros(8))
    path = str(tmp_path / "ck.npz")
    bart.save_checkpoint(path, ck)
    back = bart.load_checkpoint(path)
    for k, v in ck.items():
        if isinstance(v, np.ndarray):
            assert back[k].dtype == v.dtype and np.array_equal(back[k], v)
        else:
            assert back[k] == v


def test_demczs_sampler_refuses_to_checkpoint():
    # its archive is device state the library does not export
    import pytest
    import paper_2104_12522_gb300 as bart
    s = object.__new__(bart.Demc)
    s._zs = True
    with pytest.raises(ValueError, match="archive"):
        s.checkpoint(10)

"""CPU checks of the C ABI: the library builds, loads and exports every entry
point include/qdot.h declares; host-side argument checks reject bad calls
before anything touches a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qdot.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\**([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_00115_gb300 import build as qbuild
    qbuild.build()
    import paper_2105_00115_gb300 as q
    return q.load()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("qdot", "qdot_explain", "qdot_workspace_size", "qdot_dot_fp64", "qdot_from_host",
                 "qdot_last_error", "qdot_version"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if getattr(lib, n, None) is None]
    assert not missing, missing
    from paper_2105_00115_gb300 import _abi
    # the binding describes every declared entry point
    assert set(declared_functions()) <= set(_abi.SIGNATURES)


def test_struct_sizes_match_header(lib):
    from paper_2105_00115_gb300 import _abi
    assert ctypes.sizeof(_abi.Result) == 80
    assert ctypes.sizeof(_abi.Params) == 24
    assert ctypes.sizeof(_abi.Selection) == 48 + 4224


def test_version(lib):
    assert b"sm_103a" in lib.qdot_version()


def test_stream_kernel_names(lib):
    """The streaming kernel each (n, block, alignment) selects (host logic)."""
    import paper_2105_00115_gb300 as q

    def name(n, block, al16=1):
        return lib.qdot_stream_kernel(n, ctypes.byref(q.params(eps=1e-8, block=block)), al16)

    # blocks of 32: item records from 2^25 on, block records below
    assert name(1 << 28, 32) == b"k_onepass_items" and name(1 << 25, 32) == b"k_onepass_items"
    assert name((1 << 25) - 1, 32) == b"k_onepass" and name(1 << 24, 32) == b"k_onepass"
    assert name(1 << 20, 32) in (b"k_onepass", b"k_qdot_fused")
    assert name(1 << 28, 64) == b"k_onepass" and name(1 << 28, 256) == b"k_onepass"
    # blocks of one and exact binning: two passes (the fused launch only when
    # asked for); blocks of one take item records from 2^24 on
    assert name(1 << 28, 1) == b"k_onepass_items"
    assert name(1 << 20, 1) == b"k_apply_fast" and name(1 << 20, 0) == b"k_apply_fast"
    assert name(1 << 23, 1) == b"k_apply_fast"
    assert name(1 << 28, 0) == b"k_apply_fast" and name(1 << 28, 8) == b"k_apply_fast"
    assert name(1 << 28, 32, al16=0) == b"k_apply_fast"  # 8-byte aligned inputs
    assert name(1 << 20, 3) == b""  # invalid block


def test_workspace_size_rejects_bad_params(lib):
    import paper_2105_00115_gb300 as q
    ok = q.params(eps=1e-8, block=32)
    assert lib.qdot_workspace_size(1 << 20, ctypes.byref(ok)) > 0
    for bad in (q.params(eps=0.0), q.params(eps=-1.0), q.params(eps=float("nan")), q.params(eps=float("inf")),
                q.params(block=3), q.params(block=-2), q.params(block=1 << 21), q.params(split_budget=2),
                q.params(mant_reading=5)):
        assert lib.qdot_workspace_size(1000, ctypes.byref(bad)) == 0
    assert lib.qdot_workspace_size(-1, ctypes.byref(ok)) == 0


def test_host_argument_checks_before_launch(lib):
    import paper_2105_00115_gb300 as q
    bad = q.params(eps=-1.0)
    st = lib.qdot(None, None, 0, ctypes.byref(bad), ctypes.c_void_p(256), None, ctypes.c_void_p(256), 1 << 20, None)
    assert st == 1 and b"eps" in lib.qdot_last_error()
    good = q.params(eps=1e-8, block=32)
    st = lib.qdot(None, None, 10, ctypes.byref(good), ctypes.c_void_p(256), None, ctypes.c_void_p(256), 1 << 20, None)
    assert st == 1 and b"non-NULL" in lib.qdot_last_error()
    st = lib.qdot(ctypes.c_void_p(4), ctypes.c_void_p(8), 10, ctypes.byref(good), ctypes.c_void_p(256), None,
                  ctypes.c_void_p(256), 1 << 20, None)
    assert st == 1 and b"aligned" in lib.qdot_last_error()
    st = lib.qdot(ctypes.c_void_p(256), ctypes.c_void_p(512), 10, ctypes.byref(good), ctypes.c_void_p(256), None,
                  ctypes.c_void_p(100), 1 << 20, None)
    assert st == 5
    st = lib.qdot(ctypes.c_void_p(256), ctypes.c_void_p(512), 10, ctypes.byref(good), ctypes.c_void_p(256), None,
                  ctypes.c_void_p(256), 16, None)
    assert st == 5 and b"too small" in lib.qdot_last_error()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2105_00115_gb300 import _abi
    saved = _abi._lib
    _abi._lib = None
    try:
        with pytest.raises(ImportError):
            _abi.load(str(tmp_path / "missing.so"))
    finally:
        _abi._lib = saved

"""The C ABI library loads and exports every entry point include/hpx.h
declares; host-only entry points and argument validation work without a GPU
(no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hpx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hpx_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def hpxlib():
    from paper_2510_01785_gb300 import build as b
    b.build()
    from paper_2510_01785_gb300 import _lib
    return _lib


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hpx_plan_create", "hpx_plan_destroy", "hpx_map2alm", "hpx_alm2map",
                     "hpx_map2alm_adjoint", "hpx_alm2map_adjoint", "hpx_plan_device_bytes",
                     "hpx_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(hpxlib):
    L = hpxlib.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in hpxlib.SIGNATURES, f"binding lacks {name}"


def test_nalm(hpxlib):
    L = hpxlib.lib()
    assert L.hpx_nalm(95, 95) == 4656
    assert L.hpx_nalm(3071, 3071) == 4720128
    assert L.hpx_nalm(2047, 2047) == 2098176
    assert L.hpx_nalm(767, 767) == 295296
    assert L.hpx_nalm(10, 3) == 11 + 10 + 9 + 8
    assert L.hpx_nalm(5, 7) == 0


@pytest.mark.parametrize("args", [(3, 8, 8, 1, 1), (0, 8, 8, 1, 1), (16, 10, 11, 1, 1),
                                  (16, 10, 10, 0, 1), (16, -1, 0, 1, 1)])
def test_invalid_plan_arguments_are_rejected(hpxlib, args):
    L = hpxlib.lib()
    h = ctypes.c_void_p()
    st = L.hpx_plan_create(*args, ctypes.byref(h))
    assert st == 1  # HPX_ERR_INVALID, before any CUDA call
    assert h.value is None
    assert L.hpx_last_error()


def test_null_plan_calls_are_rejected(hpxlib):
    L = hpxlib.lib()
    buf = ctypes.create_string_buffer(64)
    assert L.hpx_map2alm(None, buf, buf, None) == 1
    assert L.hpx_plan_destroy(None) == 0
    assert L.hpx_plan_device_bytes(None) == 0
    assert L.hpx_plan_device_status(None) == 1


@pytest.mark.parametrize("dtype,flags", [(0, 3), (1, 2), (0, 2), (1, 4), (1, 9), (0, 11), (2, 8)])
def test_tensor_core_flag_needs_an_f32_table_plan(hpxlib, dtype, flags):
    L = hpxlib.lib()
    h = ctypes.c_void_p()
    assert L.hpx_plan_create_ex(16, 47, 47, 1, dtype, flags, ctypes.byref(h)) == 1
    assert h.value is None


def test_estimate_counts_the_tensor_core_operands(hpxlib):
    L = hpxlib.lib()
    table = L.hpx_plan_estimate_bytes(1024, 3071, 3071, 8, 1, 1)
    tc = L.hpx_plan_estimate_bytes(1024, 3071, 3071, 8, 1, 3)
    # Gt operand: (mmax+1) x 64 groups x 32 columns x 32 pairs x 4 bytes
    assert tc - table >= 3072 * 64 * 32 * 32 * 4


def test_streamed_plan_flags(hpxlib):
    """Rejected before any device work: extra flags to the streamed
    constructor, streaming together with host tables, streaming without the
    tensor-core path."""
    L = hpxlib.lib()
    h = ctypes.c_void_p()
    assert L.hpx_plan_create_stream(16, 47, 47, 1, 1, 1, 0, ctypes.byref(h)) == 1
    assert h.value is None
    assert L.hpx_plan_create_ex(16, 47, 47, 1, 1, 1 | 2 | 4 | 16, ctypes.byref(h)) == 1
    assert L.hpx_plan_create_ex(16, 47, 47, 1, 0, 16, ctypes.byref(h)) == 1
    assert L.hpx_plan_create_ex(16, 47, 47, 1, 1, 16, ctypes.byref(h)) == 1
    assert h.value is None


def test_estimate_streamed_holds_no_table(hpxlib):
    L = hpxlib.lib()
    tc = L.hpx_plan_estimate_bytes(1024, 3071, 3071, 8, 1, 3)
    st = L.hpx_plan_estimate_bytes(1024, 3071, 3071, 8, 1, 3 | 16)
    assert st < tc - 20e9  # the FP16 hi/lo tables (about 58 GB) are not held; two staging buffers are


def _header_declarations():
    """{name: (return type, [argument types])} of every function declared in
    include/hpx.h (comments and preprocessor lines stripped)."""
    src = open(os.path.join(ROOT, "include", "hpx.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = "\n".join(ln for ln in src.splitlines() if not ln.lstrip().startswith("#"))
    out = {}
    for stmt in src.split(";"):
        stmt = re.split(r"[{}]", stmt)[-1]
        mt = re.fullmatch(r"\s*([A-Za-z_][\w\s\*]*?)\s*\b(hpx_\w+)\s*\(([^()]*)\)\s*", stmt, flags=re.S)
        if not mt:
            continue
        ret, name, args = mt.groups()
        parts = [a.strip() for a in args.split(",")] if args.strip() not in ("", "void") else []
        types = [re.sub(r"\s*\b\w+$", "", a).replace(" *", "*").strip() for a in parts]
        out[name] = (" ".join(ret.split()).replace(" *", "*"), types)
    return out


def test_binding_signatures_match_the_header():
    """The ctypes table of the Python binding mirrors include/hpx.h: the same
    functions, argument counts and argument types, so no call passes a value
    of the wrong width."""
    from paper_2510_01785_gb300 import _lib
    P = ctypes.c_void_p
    arg = {"const double*": P, "const void*": P, "double*": P, "void*": P, "int32_t*": P, "int64_t*": P,
           "hpx_plan": P, "hpx_stream_t": P, "hpx_plan*": ctypes.POINTER(P),
           "int": ctypes.c_int, "hpx_dtype": ctypes.c_int, "hpx_layout": ctypes.c_int,
           "unsigned": ctypes.c_uint, "size_t": ctypes.c_size_t}
    res = {"hpx_status": ctypes.c_int, "size_t": ctypes.c_size_t, "int64_t": ctypes.c_int64,
           "const char*": ctypes.c_char_p}
    decl = _header_declarations()
    assert len(decl) >= 30
    assert set(decl) == set(_lib.SIGNATURES)
    for name, (ret, types) in decl.items():
        r, a = _lib.SIGNATURES[name]
        assert r is res[ret], (name, ret)
        assert len(a) == len(types), (name, types)
        for got, t in zip(a, types):
            assert got is arg[t], (name, t)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with libhpx.so missing, the first library call raises
    and names the build step."""
    from paper_2510_01785_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libhpx.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="libhpx.so not found"):
        _lib.lib()

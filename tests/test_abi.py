"""Host-side checks of the C ABI: the library builds, loads without a GPU,
exports every symbol include/tcbf.h declares, and rejects bad arguments
with status codes before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2505_03269_gb300 import binding
from paper_2505_03269_gb300 import build as tcbf_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    tcbf_build.build()
    return binding.load()


def declared_functions(header="tcbf.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tcbf_[a-z0-9_]+)\s*\(", src)))


def all_headers():
    return sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(binding.EXPORTED)
    from paper_2505_03269_gb300 import serve
    assert declared_functions("tcbf_server.h") == sorted(serve.SERVER_SYMBOLS)


def test_every_declared_symbol_is_exported(lib):
    for h in all_headers():
        for name in declared_functions(h):
            assert hasattr(lib, name), (h, name)


def test_status_strings(lib):
    for s in range(8):
        assert binding.status_string(s)
    assert binding.status_string(99) == "unknown status"


def _create(lib, **kw):
    p = binding.Problem(kw.get("batch", 1), kw.get("M", 4), kw.get("N", 4), kw.get("K", 4),
                        kw.get("w_batches", 0), kw.get("mode", 0), kw.get("flags", 0))
    h = ctypes.c_void_p(123)
    st = lib.tcbf_plan_create(ctypes.byref(h), ctypes.byref(p), 0)
    return st, h


@pytest.mark.parametrize("bad", [dict(M=0), dict(N=0), dict(K=0), dict(batch=0),
                                 dict(batch=4, w_batches=3), dict(mode=7), dict(flags=2),
                                 dict(flags=1, mode=1), dict(flags=1, mode=2), dict(flags=16),
                                 dict(flags=8, mode=1), dict(flags=8, mode=2), dict(flags=9),
                                 dict(flags=4, mode=0), dict(flags=2, mode=2),
                                 dict(flags=6, mode=1), dict(M=-5),
                                 dict(flags=32, mode=1), dict(flags=32, mode=2), dict(flags=33),
                                 dict(flags=40), dict(flags=64)])
def test_plan_create_rejects_bad_shapes(lib, bad):
    st, h = _create(lib, **bad)
    assert st == 1          # TCBF_ERR_INVALID_ARG, before any device query
    assert h.value is None


def test_null_arguments(lib):
    assert lib.tcbf_plan_create(None, None, 0) == 1
    h = ctypes.c_void_p()
    assert lib.tcbf_plan_create(ctypes.byref(h), None, 0) == 1
    n = ctypes.c_size_t()
    assert lib.tcbf_packed_size(None, 0, ctypes.byref(n)) == 1
    assert lib.tcbf_workspace_size(None, ctypes.byref(n)) == 1
    assert lib.tcbf_transpose_pack(None, 0, 0, None, None, None) == 1
    assert lib.tcbf_beamform_fp16(None, None, None, None, None) == 1
    assert lib.tcbf_beamform_fp8split(None, None, None, None, None) == 1
    assert lib.tcbf_beamform_1bit(None, None, None, None, None) == 1
    assert lib.tcbf_expand_1bit(None, 0, None, None) == 1
    assert lib.tcbf_beamform_1bit_expanded(None, None, None) == 1
    assert lib.tcbf_weights_from_geometry(None, None, None, 0, None, 1.0, None, None) == 1
    assert lib.tcbf_last_device_error(None) == 1
    assert lib.tcbf_debug_drop_fill(None, ctypes.c_int64(0)) == 1
    assert lib.tcbf_unpack_bits(None, 0, None, None, 0, None) == 1
    f = ctypes.c_uint32()
    assert lib.tcbf_plan_flags(None, ctypes.byref(f)) == 1
    assert lib.tcbf_plan_destroy(None) == 0
    # the stream microbenchmark checks its sizes before touching a device
    sec = ctypes.c_double()
    ps = lib.tcbf_peak_stream
    ps.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                   ctypes.POINTER(ctypes.c_double)]
    assert ps(0, 1 << 20, 1 << 20, 4, None) == 1
    assert ps(0, 24, 1 << 20, 4, ctypes.byref(sec)) == 1        # not a multiple of 16
    assert ps(0, 1 << 20, 0, 4, ctypes.byref(sec)) == 1
    assert ps(0, 1 << 20, 1 << 20, 0, ctypes.byref(sec)) == 1


def test_no_device_reports_unsupported(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _create(lib)
    assert st == 2 and h.value is None


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2505_03269_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "tcbf_oracle" not in txt and "liboracle" not in txt, f

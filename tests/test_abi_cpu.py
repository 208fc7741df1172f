"""C-ABI library checks that need no GPU: it builds, loads, and exports every
entry point that include/plb.h declares (no compute calls are made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "plb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(plb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1906_12018_gb300 import build_ext

    if not os.path.exists(build_ext.LIB):
        build_ext.build()
    return ctypes.CDLL(build_ext.LIB)


def test_header_declares_the_boundary():
    fns = declared_functions()
    for name in ("plb_build", "plb_query_batch", "plb_labels_view", "plb_labels_free", "plb_build_batch",
                 "plb_degree_order", "plb_strerror"):
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_symbol():
    from paper_1906_12018_gb300 import plb

    assert sorted(plb.exported_symbols()) == declared_functions()


def test_host_only_entry_points(lib):
    from paper_1906_12018_gb300 import plb

    lib = plb._lib()
    assert lib.plb_version() == 100
    assert lib.plb_strerror(0) == b"ok"
    assert b"254" in lib.plb_strerror(3)
    o = plb.default_options()
    assert o.validate == 1 and o.warp_label_cap > 0 and o.block_threads % 32 == 0
    # argument errors are reported before any device work
    h = ctypes.c_void_p()
    assert lib.plb_build(None, None, None, None, ctypes.byref(h)) == plb.PLB_ERR_INVALID
    g = plb.CSR(1 << 24, 0, 1, None)
    assert lib.plb_build(ctypes.byref(g), 1, None, None, ctypes.byref(h)) == plb.PLB_ERR_TOO_LARGE
    assert lib.plb_query_batch(None, None, 1, None, None) == plb.PLB_ERR_INVALID
    assert lib.plb_labels_free(None) == 0
    assert lib.plb_memory_stats(None, 0) == plb.PLB_ERR_INVALID


def test_struct_layouts_match_header():
    from paper_1906_12018_gb300 import plb

    assert ctypes.sizeof(plb.Options) == 16 * 4
    assert ctypes.sizeof(plb.CSR) == 32
    assert ctypes.sizeof(plb.LabelView) == 6 * 8 + 8


def test_variant_entry_points_reject_bad_arguments_before_device_work(lib):
    from paper_1906_12018_gb300 import plb

    lib = plb._lib()
    h, h2 = ctypes.c_void_p(), ctypes.c_void_p()
    assert lib.plb_build_directed(None, None, None, None, ctypes.byref(h), ctypes.byref(h2)) == plb.PLB_ERR_INVALID
    assert lib.plb_build_weighted(None, None, None, None, None, ctypes.byref(h)) == plb.PLB_ERR_INVALID
    g = plb.CSR(4, 2, 1, 1)                      # arcs but no weight array
    assert lib.plb_build_weighted(ctypes.byref(g), None, 1, None, None, ctypes.byref(h)) == plb.PLB_ERR_INVALID
    big = plb.CSR(1 << 24, 0, 1, None)
    assert lib.plb_build_weighted(ctypes.byref(big), None, 1, None, None, ctypes.byref(h)) == plb.PLB_ERR_TOO_LARGE
    o = plb.default_options()
    assert o.warp_stage_ratio == 4 and o.batch_hubs == 0
    bad = plb.default_options(warp_stage_ratio=2000)   # outside 0..1024: refused with the options check
    assert lib.plb_build(ctypes.byref(g), 1, ctypes.byref(bad), None, ctypes.byref(h)) == plb.PLB_ERR_INVALID


def test_binding_refuses_host_tensors():
    torch = pytest.importorskip("torch")
    from paper_1906_12018_gb300 import plb

    off = torch.zeros(2, dtype=torch.int64)
    col = torch.zeros(0, dtype=torch.int32)
    with pytest.raises(TypeError):
        plb.build_weighted(off, col, torch.zeros(0, dtype=torch.uint8), torch.zeros(1, dtype=torch.int32))
    with pytest.raises(TypeError):
        plb.build_directed(off, col, torch.zeros(1, dtype=torch.int32))


def test_binding_checks_buffer_sizes_before_calling_the_library(monkeypatch):
    """Short output buffers, a set index per pair and an odd id count are
    refused on the host: the library would otherwise write past a buffer."""
    torch = pytest.importorskip("torch")
    from paper_1906_12018_gb300 import plb

    calls = []

    class FakeLib:
        def __getattr__(self, name):
            def f(*a):
                calls.append(name)
                return 0
            return f

    monkeypatch.setattr(plb, "_dev", lambda t, dtype, name: t)   # host tensors stand in for device ones
    monkeypatch.setattr(plb, "_lib", lambda: FakeLib())
    monkeypatch.setattr(plb, "_stream", lambda s: 0)
    i32 = torch.int32
    rp = torch.zeros(11, dtype=torch.int64)                         # n = 10
    with pytest.raises(ValueError):
        plb.degree_order_noalloc(rp, out=torch.empty(9, dtype=i32))
    with pytest.raises(ValueError):
        plb.degree_order_noalloc(rp, out=torch.empty(10, dtype=i32, device="meta"))
    lab = object.__new__(plb.Labels)
    lab._h = ctypes.c_void_p(1)
    with pytest.raises(ValueError):
        lab.query(torch.zeros(7, dtype=i32))
    with pytest.raises(ValueError):
        lab.query(torch.zeros(8, dtype=i32), out=torch.empty(3, dtype=i32))
    with pytest.raises(ValueError):
        plb.query_directed(lab, lab, torch.zeros(8, dtype=i32), out=torch.empty(3, dtype=i32))
    with pytest.raises(ValueError):
        plb.query_multi([lab], torch.zeros(4, dtype=i32), torch.zeros(7, dtype=i32))
    with pytest.raises(ValueError):
        plb.query_multi([lab], torch.zeros(3, dtype=i32), torch.zeros(8, dtype=i32))
    with pytest.raises(ValueError):
        plb.query_multi([lab], torch.zeros(4, dtype=i32), torch.zeros(8, dtype=i32), out=torch.empty(3, dtype=i32))
    assert calls == []
    # well-formed calls reach the library
    plb.degree_order_noalloc(rp, out=torch.empty(10, dtype=i32))
    plb.query_multi([lab], torch.zeros(4, dtype=i32), torch.zeros(8, dtype=i32), out=torch.empty(4, dtype=i32))
    assert calls == ["plb_degree_order_noalloc", "plb_query_multi"]


def test_free_reports_a_failed_free_once(monkeypatch):
    """Labels.free passes the library's status on (PLBError) and clears the
    handle first: a second free, or the destructor, calls nothing."""
    from paper_1906_12018_gb300 import plb

    calls = []

    class FakeLib:
        def plb_labels_free(self, h):
            calls.append(h.value)
            return plb.PLB_ERR_CUDA

        def plb_strerror(self, code):
            return b"CUDA error"

        def plb_last_error(self):
            return b""

    monkeypatch.setattr(plb, "_lib", lambda: FakeLib())
    lab = object.__new__(plb.Labels)
    lab._h = ctypes.c_void_p(1234)
    with pytest.raises(plb.PLBError) as e:
        lab.free()
    assert e.value.code == plb.PLB_ERR_CUDA
    lab.free()
    lab.__del__()
    assert calls == [1234]
    with pytest.raises(RuntimeError):
        lab.handle

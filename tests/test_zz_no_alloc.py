"""The allocation-free degree order (plb_degree_order_noalloc), called
through the C ABI, must give exactly the order of plb_degree_order on two
calls in a row.  It is meant for callers that cannot let the library allocate
device memory (framework-owned memory, fixed HBM budgets, latency-critical
paths).  The file is collected last on purpose: it checks that the scratch
array's contents left by earlier calls (this process's other tests) do not
leak into a result, so it must also pass after every other test has run, and
a failure here leaves every other result already reported."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1906_12018_gb300 import graphs as G
from paper_1906_12018_gb300 import plb


def _csr(row_ptr):
    return plb.CSR(row_ptr.numel() - 1, 0, row_ptr.data_ptr(), None)


def test_noalloc_rejects_too_many_vertices():
    lib = plb._lib()
    g = plb.CSR(plb.NOALLOC_MAX_VERTICES + 1, 0, 1, None)
    assert lib.plb_degree_order_noalloc(ctypes.byref(g), 1, None) == plb.PLB_ERR_TOO_LARGE
    assert lib.plb_degree_order_noalloc(None, None, None) == plb.PLB_ERR_INVALID


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_twice():
    lib = plb._lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    graphs = [G.workload("rmat12"), G.small_graph(1)]   # two calls in a row, different sizes
    for g in graphs:
        rp = torch.from_numpy(g.off).to(dev)
        want = torch.empty(g.n, dtype=torch.int32, device=dev)
        got = torch.full((g.n,), -7, dtype=torch.int32, device=dev)
        assert lib.plb_degree_order(ctypes.byref(_csr(rp)), want.data_ptr(), stream.cuda_stream) == plb.PLB_OK
        assert lib.plb_degree_order_noalloc(ctypes.byref(_csr(rp)), got.data_ptr(),
                                            stream.cuda_stream) == plb.PLB_OK
        torch.cuda.synchronize(dev)
        assert torch.equal(got, want)
        assert np.array_equal(got.cpu().numpy(), G.degree_order(g))


def _degree_rows(n, seed):
    """row_ptr of n vertices with power-law-like degrees (only the offsets
    matter for the order), and the order by definition: degree descending,
    ties by smaller id."""
    rng = np.random.default_rng(seed)
    deg = np.minimum(rng.zipf(2.1, n), 5000).astype(np.int64)
    deg[rng.random(n) < 0.05] = 0                      # isolated vertices: long runs of ties
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    want = np.lexsort((np.arange(n), -deg)).astype(np.int32)
    return row_ptr, want


@pytest.mark.gpu
@pytest.mark.parametrize("n", [plb.NOALLOC_MAX_VERTICES, plb.NOALLOC_MAX_VERTICES - 1])
def test_noalloc_at_the_scratch_limit(n):
    """n = 2^20 fills the scratch array exactly (the padded key count equals
    its length); n = 2^20 - 1 pads one key.  Two calls in a row each."""
    lib = plb._lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    for seed in (1, 2):
        row_ptr, want_np = _degree_rows(n, seed + n)
        rp = torch.from_numpy(row_ptr).to(dev)
        want = torch.empty(n, dtype=torch.int32, device=dev)
        got = torch.full((n,), -7, dtype=torch.int32, device=dev)
        assert lib.plb_degree_order(ctypes.byref(_csr(rp)), want.data_ptr(), stream.cuda_stream) == plb.PLB_OK
        assert lib.plb_degree_order_noalloc(ctypes.byref(_csr(rp)), got.data_ptr(),
                                            stream.cuda_stream) == plb.PLB_OK
        torch.cuda.synchronize(dev)
        assert torch.equal(got, want)
        assert np.array_equal(got.cpu().numpy(), want_np)


@pytest.mark.gpu
def test_noalloc_on_chunglu20():
    """The bench graph has exactly 2^20 vertices: the generator's own order."""
    g = G.workload("chunglu20")
    assert g.n == plb.NOALLOC_MAX_VERTICES
    rp = torch.from_numpy(g.off).to("cuda:0")
    got = plb.degree_order_noalloc(rp)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), G.degree_order(g))

"""The allocation-free degree order (plb_degree_order_noalloc), called
through the C ABI, must give exactly the order of plb_degree_order on two
calls in a row.  It is meant for callers that cannot let the library allocate
device memory (framework-owned memory, fixed HBM budgets, latency-critical
paths).  This file is collected last on purpose."""
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

"""Shared helpers of the GPU tests: move generator outputs to the device and
compare GPU label sets with oracle label sets."""
import numpy as np
import torch

from paper_1906_12018_gb300 import graphs as G
from paper_1906_12018_gb300 import plb


def to_device(g, order):
    dev = torch.device("cuda:0")
    row_ptr = torch.from_numpy(np.ascontiguousarray(g.off, dtype=np.int64)).to(dev)
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(dev)
    o = torch.from_numpy(np.ascontiguousarray(order, dtype=np.int32)).to(dev)
    return row_ptr, col, o


def gpu_build(g, order, **opts):
    rp, c, o = to_device(g, order)
    lab = plb.build(rp, c, o, **opts)
    return lab


def host_labels(lab):
    off, hub, dist = lab.to_host()
    return off, hub.astype(np.uint32), dist


def assert_labels_equal(lab, ref, what=""):
    off, hub, dist = host_labels(lab)
    assert off.shape == ref.off.shape, what
    assert np.array_equal(off, ref.off), f"{what}: row lengths differ"
    assert np.array_equal(hub, ref.hub), f"{what}: hubs differ"
    assert np.array_equal(dist, ref.dist), f"{what}: distances differ"


def gpu_query(lab, pairs):
    p = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
    out = lab.query(p)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def build_peak(g):
    """Device bytes of the library's pool around one build of g: peak (the
    most held during the build above what was held before), kept (held with
    the label set alive), labels (the set's own bytes), left (held after the
    set is freed) and inputs (the caller's CSR and order, outside the pool)."""
    rp, col, o = to_device(g, G.degree_order(g))
    torch.cuda.synchronize()
    before = plb.memory_stats(reset=True)
    lab = plb.build(rp, col, o)
    torch.cuda.synchronize()
    after = plb.memory_stats()
    labels = lab.nbytes()
    lab.free()
    freed = plb.memory_stats()
    return {"peak": after["used_high"] - before["used"], "kept": after["used"] - before["used"], "labels": labels,
            "left": freed["used"] - before["used"], "inputs": rp.numel() * 8 + col.numel() * 4 + o.numel() * 4}

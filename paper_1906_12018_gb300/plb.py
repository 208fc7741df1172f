"""Thin ctypes binding of ``libplb.so`` (C ABI in ``include/plb.h``).

Argument marshalling only: every step of the labeling and the queries runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.  The
library must be built (``paper_1906_12018_gb300.build_ext.build()``); nothing
here falls back to another implementation when it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libplb.so")

PLB_OK = 0
PLB_ERR_INVALID = 1
PLB_ERR_OOM = 2
PLB_ERR_DIST_OVERFLOW = 3
PLB_ERR_TIMEOUT = 4
PLB_ERR_CUDA = 5
PLB_ERR_TOO_LARGE = 6
PLB_UNREACHABLE = -1
PLB_BAD_PAIR = -2
MAX_ROUNDS = 256


class PLBError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _lib().plb_strerror(code).decode() if _LIB is not None else f"status {code}"
        if code == PLB_ERR_CUDA and _LIB is not None:
            detail = _lib().plb_last_error().decode()
            if detail:
                msg += f" [{detail}]"
        super().__init__(f"{what}: {msg} (status {code})" if what else msg)


class Options(ctypes.Structure):
    _fields_ = [
        ("validate", ctypes.c_int32),
        ("warp_label_cap", ctypes.c_int32),
        ("warp_cand_cap", ctypes.c_int32),
        ("block_label_cap", ctypes.c_int32),
        ("block_cand_cap", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("profile", ctypes.c_int32),
        ("batch_hubs", ctypes.c_int32),
        ("warp_stage_ratio", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 6),
    ]


class CSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("row_ptr", ctypes.c_void_p),
        ("col", ctypes.c_void_p),
    ]


class LabelView(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("total", ctypes.c_int64),
        ("off", ctypes.c_void_p),
        ("hub", ctypes.c_void_p),
        ("dist", ctypes.c_void_p),
        ("order", ctypes.c_void_p),
        ("max_dist", ctypes.c_int32),
        ("rounds", ctypes.c_int32),
    ]


class BuildStats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_int32),
        ("reruns", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("total_labels", ctypes.c_int64),
        ("receivers", ctypes.c_int64 * MAX_ROUNDS),
        ("accepted", ctypes.c_int64 * MAX_ROUNDS),
        ("unique_round", ctypes.c_int64 * MAX_ROUNDS),
        ("probed_round", ctypes.c_int64 * MAX_ROUNDS),
        ("prefiltered_round", ctypes.c_int64 * MAX_ROUNDS),
        ("messages_round", ctypes.c_int64 * MAX_ROUNDS),
        ("ms_round", ctypes.c_double * MAX_ROUNDS),
        ("arcs_scanned", ctypes.c_int64),
        ("messages", ctypes.c_int64),
        ("unique_candidates", ctypes.c_int64),
        ("staged_entries", ctypes.c_int64),
        ("probed_entries", ctypes.c_int64),
        ("tier_vertices", ctypes.c_int64 * 3),
        ("ms_total", ctypes.c_double),
        ("ms_prepare", ctypes.c_double),
        ("ms_frontier", ctypes.c_double),
        ("ms_gather_prune", ctypes.c_double * 3),
        ("ms_merge", ctypes.c_double),
        ("ms_finalize", ctypes.c_double),
        ("launches", ctypes.c_int64),
        ("check_lv_entries", ctypes.c_int64),
        ("check_lh_entries", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        r = self.rounds
        return {
            "rounds": r,
            "reruns": self.reruns,
            "n": self.n,
            "nnz": self.nnz,
            "total_labels": self.total_labels,
            "receivers": list(self.receivers[1 : r + 1]),
            "accepted": list(self.accepted[1 : r + 1]),
            "unique_round": list(self.unique_round[1 : r + 1]),
            "probed_round": list(self.probed_round[1 : r + 1]),
            "prefiltered_round": list(self.prefiltered_round[1 : r + 1]),
            "messages_round": list(self.messages_round[1 : r + 1]),
            "ms_round": list(self.ms_round[1 : r + 1]),
            "arcs_scanned": self.arcs_scanned,
            "messages": self.messages,
            "unique_candidates": self.unique_candidates,
            "staged_entries": self.staged_entries,
            "probed_entries": self.probed_entries,
            "tier_vertices": list(self.tier_vertices),
            "ms_total": self.ms_total,
            "ms_prepare": self.ms_prepare,
            "ms_frontier": self.ms_frontier,
            "ms_gather_prune": list(self.ms_gather_prune),
            "ms_merge": self.ms_merge,
            "ms_finalize": self.ms_finalize,
            "launches": self.launches,
            "check_lv_entries": self.check_lv_entries,
            "check_lh_entries": self.check_lh_entries,
        }


_LIB = None


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with paper_1906_12018_gb300.build_ext.build() "
            "(there is no fallback implementation)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    I64 = ctypes.c_int64
    lib.plb_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.plb_default_options.restype = None
    lib.plb_build.argtypes = [ctypes.POINTER(CSR), P, ctypes.POINTER(Options), P, ctypes.POINTER(P)]
    lib.plb_build.restype = I
    lib.plb_build_batch.argtypes = [ctypes.POINTER(CSR), ctypes.POINTER(P), I64, ctypes.POINTER(Options), P,
                                    ctypes.POINTER(P)]
    lib.plb_build_batch.restype = I
    lib.plb_query_batch.argtypes = [P, P, I64, P, P]
    lib.plb_query_batch.restype = I
    lib.plb_query_multi.argtypes = [ctypes.POINTER(P), I64, P, P, I64, P, P]
    lib.plb_query_multi.restype = I
    lib.plb_build_directed.argtypes = [ctypes.POINTER(CSR), P, ctypes.POINTER(Options), P, ctypes.POINTER(P),
                                       ctypes.POINTER(P)]
    lib.plb_build_directed.restype = I
    lib.plb_query_directed.argtypes = [P, P, P, I64, P, P]
    lib.plb_query_directed.restype = I
    lib.plb_build_weighted.argtypes = [ctypes.POINTER(CSR), P, P, ctypes.POINTER(Options), P, ctypes.POINTER(P)]
    lib.plb_build_weighted.restype = I
    lib.plb_labels_view.argtypes = [P, ctypes.POINTER(LabelView)]
    lib.plb_labels_view.restype = I
    lib.plb_labels_stats.argtypes = [P, ctypes.POINTER(BuildStats)]
    lib.plb_labels_stats.restype = I
    lib.plb_labels_bytes.argtypes = [P]
    lib.plb_labels_bytes.restype = I64
    lib.plb_labels_free.argtypes = [P]
    lib.plb_labels_free.restype = I
    lib.plb_degree_order.argtypes = [ctypes.POINTER(CSR), P, P]
    lib.plb_degree_order.restype = I
    lib.plb_release_cached_memory.argtypes = []
    lib.plb_release_cached_memory.restype = I
    lib.plb_memory_stats.argtypes = [P, I]
    lib.plb_memory_stats.restype = I
    lib.plb_degree_order_noalloc.argtypes = [ctypes.POINTER(CSR), P, P]
    lib.plb_degree_order_noalloc.restype = I
    lib.plb_strerror.argtypes = [I]
    lib.plb_strerror.restype = ctypes.c_char_p
    lib.plb_last_error.argtypes = []
    lib.plb_last_error.restype = ctypes.c_char_p
    lib.plb_version.argtypes = []
    lib.plb_version.restype = I
    _LIB = lib
    return lib


def exported_symbols() -> list[str]:
    """Names of the entry points declared in include/plb.h."""
    return ["plb_default_options", "plb_build", "plb_build_batch", "plb_build_directed", "plb_build_weighted",
            "plb_query_batch",
            "plb_query_directed", "plb_query_multi",
            "plb_labels_view", "plb_labels_stats", "plb_labels_bytes", "plb_labels_free", "plb_release_cached_memory",
            "plb_memory_stats", "plb_degree_order",
            "plb_degree_order_noalloc", "plb_strerror", "plb_last_error", "plb_version"]


def _check(code: int, what: str):
    if code != PLB_OK:
        raise PLBError(code, what)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


def default_options(**kw) -> Options:
    o = Options()
    _lib().plb_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, int(v))
    return o


def _csr(row_ptr: torch.Tensor, col: torch.Tensor) -> CSR:
    _dev(row_ptr, torch.int64, "row_ptr")
    _dev(col, torch.int32, "col")
    return CSR(row_ptr.numel() - 1, col.numel(), row_ptr.data_ptr(), col.data_ptr() if col.numel() else None)


class _DevArray:
    """__cuda_array_interface__ wrapper over library-owned device memory."""

    def __init__(self, ptr: int, n: int, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}
        self._owner = owner


class Labels:
    """A label set built on the device (library-owned memory)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        v = LabelView()
        _check(_lib().plb_labels_view(self._h, ctypes.byref(v)), "plb_labels_view")
        self.n = int(v.n)
        self.total = int(v.total)
        self.max_dist = int(v.max_dist)
        self.rounds = int(v.rounds)
        self._view = v

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise RuntimeError("label set already freed")
        return self._h

    def _tensor(self, ptr, n, typestr, dtype):
        if n == 0:
            return torch.empty(0, dtype=dtype, device="cuda")
        return torch.as_tensor(_DevArray(ptr, n, typestr, self), device="cuda")

    def device_arrays(self):
        """Zero-copy device tensors (off int64[n+1], hub int32-viewed uint32[total],
        dist uint8[total]); valid while this object is alive."""
        v = self._view
        off = self._tensor(v.off, self.n + 1, "<i8", torch.int64)
        hub = self._tensor(v.hub, self.total, "<i4", torch.int32)
        dist = self._tensor(v.dist, self.total, "|u1", torch.uint8)
        return off, hub, dist

    def to_host(self):
        """(off int64[n+1], hub uint32[total], dist uint8[total]) as numpy arrays."""
        off, hub, dist = self.device_arrays()
        torch.cuda.synchronize()
        return off.cpu().numpy(), hub.cpu().numpy().view("uint32"), dist.cpu().numpy()

    def stats(self) -> dict:
        st = BuildStats()
        _check(_lib().plb_labels_stats(self.handle, ctypes.byref(st)), "plb_labels_stats")
        return st.as_dict()

    def nbytes(self) -> int:
        return int(_lib().plb_labels_bytes(self.handle))

    def query(self, pairs: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """pairs: CUDA int32 [q, 2] (original ids) -> CUDA int32 [q] distances."""
        pairs = _dev(pairs.reshape(-1), torch.int32, "pairs")
        if pairs.numel() % 2:
            raise ValueError("pairs must hold an even number of ids (s, t)")
        q = pairs.numel() // 2
        if out is None:
            out = torch.empty(q, dtype=torch.int32, device=pairs.device)
        _dev(out, torch.int32, "out")
        if out.numel() < q or out.device != pairs.device:
            raise ValueError(f"out must hold at least {q} int32 on {pairs.device}")
        _check(_lib().plb_query_batch(self.handle, pairs.data_ptr(), q, out.data_ptr() if q else None,
                                      _stream(stream)), "plb_query_batch")
        return out

    def free(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p()  # never freed twice, even if the call fails
            _check(_lib().plb_labels_free(h), "plb_labels_free")

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build(row_ptr: torch.Tensor, col: torch.Tensor, order: torch.Tensor, options: Options | None = None,
          stream=None, **kw) -> Labels:
    """Canonical labels of the graph (device CSR) under order (CUDA int32, rank -> id)."""
    g = _csr(row_ptr, col)
    _dev(order, torch.int32, "order")
    opt = options if options is not None else default_options(**kw)
    h = ctypes.c_void_p()
    _check(_lib().plb_build(ctypes.byref(g), order.data_ptr() if order.numel() else None, ctypes.byref(opt),
                            _stream(stream), ctypes.byref(h)), "plb_build")
    return Labels(h.value)


def build_batch(graphs: Sequence, options: Options | None = None, stream=None, **kw) -> list[Labels]:
    """graphs: sequence of (row_ptr, col, order) CUDA tensors; one round loop over their union."""
    k = len(graphs)
    csrs = (CSR * max(k, 1))()
    orders = (ctypes.c_void_p * max(k, 1))()
    for i, (rp, c, o) in enumerate(graphs):
        csrs[i] = _csr(rp, c)
        _dev(o, torch.int32, "order")
        orders[i] = o.data_ptr() if o.numel() else None
    outs = (ctypes.c_void_p * max(k, 1))()
    # no options: the library's batch defaults (round loop as a captured CUDA graph)
    opt = options if options is not None else (default_options(**kw) if kw else None)
    _check(_lib().plb_build_batch(csrs, orders, k, ctypes.byref(opt) if opt is not None else None,
                                  _stream(stream), outs), "plb_build_batch")
    return [Labels(outs[i]) for i in range(k)]


def build_directed(row_ptr: torch.Tensor, col: torch.Tensor, order: torch.Tensor, options: Options | None = None,
                   stream=None, **kw) -> tuple[Labels, Labels]:
    """plb_build_directed: (row_ptr, col) are the OUT-arcs (device int64[n+1],
    int32[arcs]); returns (L_in, L_out)."""
    g = _csr(row_ptr, col)
    _dev(order, torch.int32, "order")
    if options is None:
        options = default_options(**kw)
    hi, ho = ctypes.c_void_p(), ctypes.c_void_p()
    _check(_lib().plb_build_directed(ctypes.byref(g), order.data_ptr() if order.numel() else None,
                                     ctypes.byref(options), _stream(stream), ctypes.byref(hi), ctypes.byref(ho)),
           "plb_build_directed")
    return Labels(hi.value), Labels(ho.value)


def build_weighted(row_ptr: torch.Tensor, col: torch.Tensor, weight: torch.Tensor, order: torch.Tensor,
                   options: Options | None = None, stream=None, **kw) -> Labels:
    """plb_build_weighted: symmetric CSR (device int64[n+1], int32[arcs]) with
    one uint8 weight >= 1 per arc (device, equal in both directions);
    canonical labels over weighted shortest paths, queried with ``query``."""
    g = _csr(row_ptr, col)
    _dev(weight, torch.uint8, "weight")
    _dev(order, torch.int32, "order")
    if weight.numel() != g.nnz:
        raise ValueError("one weight per arc")
    if options is None:
        options = default_options(**kw)
    h = ctypes.c_void_p()
    _check(_lib().plb_build_weighted(ctypes.byref(g), weight.data_ptr() if weight.numel() else None,
                                     order.data_ptr() if order.numel() else None, ctypes.byref(options),
                                     _stream(stream), ctypes.byref(h)), "plb_build_weighted")
    return Labels(h.value)


def query_directed(l_out: Labels, l_in: Labels, pairs: torch.Tensor, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """d(s -> t) for CUDA int32 pairs [q, 2] from the two sets of build_directed."""
    pairs = _dev(pairs.reshape(-1), torch.int32, "pairs")
    if pairs.numel() % 2:
        raise ValueError("pairs must hold an even number of ids (s, t)")
    q = pairs.numel() // 2
    if out is None:
        out = torch.empty(q, dtype=torch.int32, device=pairs.device)
    _dev(out, torch.int32, "out")
    if out.numel() < q or out.device != pairs.device:
        raise ValueError(f"out must hold at least {q} int32 on {pairs.device}")
    _check(_lib().plb_query_directed(l_out.handle, l_in.handle, pairs.data_ptr(), q, out.data_ptr() if q else None,
                                     _stream(stream)), "plb_query_directed")
    return out


def query_multi(sets: Sequence[Labels], set_idx: torch.Tensor, pairs: torch.Tensor,
                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Pair i answered on sets[set_idx[i]], all in one launch."""
    m = len(sets)
    arr = (ctypes.c_void_p * max(m, 1))()
    for i, s in enumerate(sets):
        arr[i] = s.handle
    pairs = _dev(pairs.reshape(-1), torch.int32, "pairs")
    _dev(set_idx, torch.int32, "set_idx")
    if pairs.numel() % 2:
        raise ValueError("pairs must hold an even number of ids (s, t)")
    q = pairs.numel() // 2
    if set_idx.numel() != q:
        raise ValueError(f"set_idx must have one entry per pair ({q}), got {set_idx.numel()}")
    if set_idx.device != pairs.device:
        raise ValueError("set_idx and pairs must be on the same device")
    if out is None:
        out = torch.empty(q, dtype=torch.int32, device=pairs.device)
    _dev(out, torch.int32, "out")
    if out.numel() < q or out.device != pairs.device:
        raise ValueError(f"out must hold at least {q} int32 on {pairs.device}")
    _check(_lib().plb_query_multi(arr, m, set_idx.data_ptr() if q else None, pairs.data_ptr() if q else None, q,
                                  out.data_ptr() if q else None, _stream(stream)), "plb_query_multi")
    return out


def degree_order(row_ptr: torch.Tensor, stream=None) -> torch.Tensor:
    """rank -> id, degree descending, ties by smaller id (CUDA int32[n])."""
    _dev(row_ptr, torch.int64, "row_ptr")
    n = row_ptr.numel() - 1
    out = torch.empty(n, dtype=torch.int32, device=row_ptr.device)
    g = CSR(n, 0, row_ptr.data_ptr(), None)
    _check(_lib().plb_degree_order(ctypes.byref(g), out.data_ptr() if n else None, _stream(stream)),
           "plb_degree_order")
    return out


NOALLOC_MAX_VERTICES = 1 << 20


def degree_order_noalloc(row_ptr: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Same as degree_order without any device allocation by the library
    (fixed 8 MiB scratch, at most NOALLOC_MAX_VERTICES vertices; concurrent
    calls race on that scratch).  ``out`` may be passed to avoid the output
    allocation on the Python side too."""
    _dev(row_ptr, torch.int64, "row_ptr")
    n = row_ptr.numel() - 1
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=row_ptr.device)
    _dev(out, torch.int32, "out")
    if out.numel() < n or out.device != row_ptr.device:
        raise ValueError(f"out must hold at least {n} int32 on {row_ptr.device}")
    g = CSR(n, 0, row_ptr.data_ptr(), None)
    _check(_lib().plb_degree_order_noalloc(ctypes.byref(g), out.data_ptr() if n else None, _stream(stream)),
           "plb_degree_order_noalloc")
    return out


def release_cached_memory():
    """Return the library's cached, unused device memory to the driver."""
    _check(_lib().plb_release_cached_memory(), "plb_release_cached_memory")


def memory_stats(reset: bool = False) -> dict:
    """Device bytes of the library's pool on the current device: in use now,
    the most in use at once since the last reset, reserved now and the most
    reserved.  reset=True restarts the high marks after reading them."""
    out = (ctypes.c_int64 * 4)()
    _check(_lib().plb_memory_stats(ctypes.cast(out, ctypes.c_void_p), 1 if reset else 0), "plb_memory_stats")
    return {"used": out[0], "used_high": out[1], "reserved": out[2], "reserved_high": out[3]}


def version() -> int:
    return int(_lib().plb_version())

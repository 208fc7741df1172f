"""SHA-256 digests of a label set in the exported layout (test infrastructure).

A label set is (off int64[n+1], hub uint32[T], dist uint8[T]): rows by
original vertex id, hub as its rank, each row sorted by hub rank.  The digest
of a block of rows [a, b) is the SHA-256 of, in this order,

* the b - a row lengths as little-endian int64,
* the block's hubs as little-endian uint32,
* the block's distances as uint8.

Row lengths instead of offsets make a block's digest independent of the rows
before it, so a mismatch names the block that differs.  The same function
digests the oracle's labels (when the stored values are written) and the GPU
labels (in the tests); it holds none of the labeling arithmetic.
"""
from __future__ import annotations

import hashlib
from concurrent.futures import ThreadPoolExecutor

import numpy as np

BLOCK_ROWS = 1 << 16


def block_digest(off: np.ndarray, hub: np.ndarray, dist: np.ndarray, a: int, b: int) -> str:
    lo, hi = int(off[a]), int(off[b])
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(np.diff(off[a:b + 1]).astype("<i8")).tobytes())
    h.update(np.ascontiguousarray(hub[lo:hi].astype("<u4", copy=False)).data)
    h.update(np.ascontiguousarray(dist[lo:hi].astype(np.uint8, copy=False)).data)
    return h.hexdigest()


def block_digests(off, hub, dist, block_rows: int = BLOCK_ROWS, threads: int = 8) -> list[str]:
    """Digests of the consecutive blocks of ``block_rows`` rows (the last one
    ragged).  hashlib releases the GIL on large buffers, so blocks are hashed
    on a few threads."""
    off = np.asarray(off, dtype=np.int64)
    n = int(off.shape[0] - 1)
    spans = [(a, min(n, a + block_rows)) for a in range(0, n, block_rows)]
    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        return list(ex.map(lambda s: block_digest(off, hub, dist, s[0], s[1]), spans))


def labels_digest(off, hub, dist) -> str:
    """One digest over the whole label set (all rows as one block)."""
    off = np.asarray(off, dtype=np.int64)
    return block_digest(off, hub, dist, 0, int(off.shape[0] - 1))

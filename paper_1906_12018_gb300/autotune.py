"""Autotuner for the tier geometry of (batched) builds.

Knobs (``plb_options``):
  * warp_cand_cap   candidates a warp-per-vertex gather can hold; with the
                    label cap it sets the vertex-per-warp / vertex-per-block
                    split (vertices beyond either cap go to the block tier);
  * warp_label_cap  |L(v)| the warp tier stages in its shared-memory map (the
                    shared-memory probe width of the warp tier);
  * block_threads   threads of the block tier;
  * block_cand_cap  candidates per hub-range pass of the block tier;
  * block_label_cap |L(v)| the block tier stages in its shared-memory map;
  * use_graph       round loop as one captured CUDA graph (1) or host-driven (0).

Coordinate descent from the defaults: each knob in turn takes the value with
the smallest measured build time on a sample of the workload (other knobs
fixed); two sweeps.  Results are cached per (GPU, workload shape) in a JSON
file (``$PLB_AUTOTUNE_CACHE``, default ``~/.cache/plb/autotune.json``).
"""
from __future__ import annotations

import json
import math
import os
import time

SPACE = {
    "use_graph": [1, 0],
    "warp_cand_cap": [256, 512, 1024],
    "warp_label_cap": [256, 512, 1024],
    "block_threads": [128, 256],
    "block_cand_cap": [1024, 2048, 4096],
    "block_label_cap": [512, 1024],
}


def cache_path() -> str:
    return os.environ.get("PLB_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "plb",
                                                              "autotune.json"))


def as_dict(opts) -> dict:
    return {k: int(getattr(opts, k)) for k in SPACE}


def workload_key(sample) -> str:
    import torch

    n = sum(int(rp.numel()) - 1 for rp, _, _ in sample)
    nnz = sum(int(c.numel()) for _, c, _ in sample)
    name = torch.cuda.get_device_name()
    return f"{name}|graphs{len(sample)}|n2^{round(math.log2(max(n, 1)))}|deg{round(nnz / max(n, 1))}"


def _time_batch(sample, opts, reps: int) -> float:
    import torch

    from . import plb

    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        labs = plb.build_batch(sample, opts) if len(sample) > 1 else [plb.build(*sample[0], opts)]
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t)
        for lab in labs:
            lab.free()
    return best


def tune_batch(sample, space: dict | None = None, reps: int = 2, use_cache: bool = True):
    """Pick tier geometry for a list of (row_ptr, col, order) CUDA tensors.
    Returns (options, report)."""
    from . import plb

    space = space or SPACE
    key = workload_key(sample)
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    if use_cache and key in cache:
        return plb.default_options(**cache[key]["options"]), {"key": key, "cached": True, **cache[key]}
    cur = {k: int(getattr(plb.default_options(), k)) for k in space}
    if "use_graph" in space:
        cur["use_graph"] = space["use_graph"][0]
    _time_batch(sample, plb.default_options(**cur), 1)  # warm-up
    base = _time_batch(sample, plb.default_options(**cur), reps)
    best_t, trials = base, 1
    for _sweep in range(2):
        changed = False
        for knob, values in space.items():
            for val in values:
                if val == cur[knob]:
                    continue
                trial = dict(cur, **{knob: val})
                t = _time_batch(sample, plb.default_options(**trial), reps)
                trials += 1
                if t < best_t * 0.98:
                    best_t, cur, changed = t, trial, True
        if not changed:
            break
    entry = {"options": cur, "ms": 1e3 * best_t, "default_ms": 1e3 * base, "trials": trials}
    if use_cache:
        cache[key] = entry
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return plb.default_options(**cur), {"key": key, "cached": False, **entry}

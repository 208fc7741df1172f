"""GB300-native canonical 2-hop distance labeling (pruned landmark labeling
built round by round in vertex-centric style, Jin et al., arXiv 1906.12018).

* ``plb``       binding of the CUDA library (``libplb.so``, C ABI ``include/plb.h``)
* ``graphs``    seeded synthetic graph workloads (host C generators)
* ``serve``     continuous-batching query/labeling server over resident label sets
* ``autotune``  tier-geometry autotuner for batched builds
* ``build_ext`` compiles ``libplb.so`` for sm_103a

The binding is imported lazily so that the host-only generators can be used
on machines without a GPU; calling into ``plb`` without the built library
raises (there is no fallback implementation).
"""
import importlib

__all__ = ["plb", "graphs", "serve", "autotune", "build_ext"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

"""GB300-native enumerative LTL learner ("LTL learning on GPUs", arXiv 2402.12373).

The learner's hot path (size-by-size enumeration over !, &, |, X, F, G, U on
packed characteristic bit-vectors, branch-free temporal operators -- a carry
chain over the bit-reversed trace, or the paper's log-step exponential
propagation --, exact device hash-set dedup, separation check with early exit)
runs in hand-written CUDA
kernels for sm_103a behind the C ABI declared in include/ltl.h.  This package
holds the kernels' sources (csrc/), the in-tree build, a thin ctypes binding
and the seeded synthetic workloads.
"""
from . import synth  # noqa: F401  (pure numpy; no CUDA needed)

__all__ = ["synth", "learn", "evaluate", "Context", "load"]


def __getattr__(name):
    # the CUDA library is loaded on first use, never silently replaced
    if name in ("learn", "evaluate", "Context", "load", "version", "LtlError", "STATUS",
                "ALL", "NOT", "AND", "OR", "X", "F", "G", "U", "STOP_NONE", "STOP_FIRST", "STOP_LEVEL"):
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)

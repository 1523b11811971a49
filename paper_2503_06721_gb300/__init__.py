"""GB300-native Wilson-Dirac operator and CG solver for fermions in higher
representations of SU(N) (the hot path of HiRep v2, arXiv 2503.06721).

The compute lives in ``libhr.so`` (hand-written CUDA for sm_103a behind the C
ABI declared in ``include/hr.h``).  ``paper_2503_06721_gb300.hr`` is the thin
ctypes binding with the same names; ``paper_2503_06721_gb300.torch_ops`` holds
the autograd wrappers.  Importing this package loads nothing: the library is
opened on first use and a missing library is an error, never a fallback.
"""

__all__ = ["hr", "synth", "build"]


def __getattr__(name):
    if name in ("hr", "synth", "build", "torch_ops"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

"""GB300-native 3D Laplace FMM mat-vec (sm_103a CUDA behind a C-ABI).

The CUDA library ``libfmm.so`` is loaded on first use; every compute call
goes through it and fails loudly if it is missing.  ``workloads`` (seeded
synthetic inputs) imports without it.
"""
__all__ = ["workloads"]


def __getattr__(name):
    if name in ("Plan", "FMMFunction", "evaluate", "library", "FMMError", "Options"):
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)

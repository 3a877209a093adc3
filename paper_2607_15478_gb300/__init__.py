"""GB300-native exact DTW (ParDTW): cosine cost on the fly, column-sweep
wavefront DP with 2-bit backpointers, and backtrace, behind a C-ABI library.

The CUDA binding lives in ``paper_2607_15478_gb300.pardtw`` and is imported
lazily, so that ``paper_2607_15478_gb300.synth`` (input generation) can be
used on machines without a GPU.
"""
import importlib

__all__ = ["pardtw", "synth", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

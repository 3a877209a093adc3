"""GB300-native exact DTW (ParDTW): cosine cost, anti-diagonal-free column
wavefront DP with 2-bit backpointers, and backtrace, behind a C-ABI library.

The CUDA binding lives in ``paper_2607_15478_gb300.pardtw`` and is imported
lazily, so that ``paper_2607_15478_gb300.synth`` (input generation) can be
used on machines without a GPU.
"""
__all__ = ["pardtw", "synth"]


def __getattr__(name):
    if name == "pardtw":
        from . import pardtw
        return pardtw
    if name == "synth":
        from . import synth
        return synth
    raise AttributeError(name)

"""GB300-native spatially weighted local histograms (SWIH, arXiv 1705.03524).

The CUDA library and its thin ctypes binding live in ``swih``; the seeded
synthetic inputs in ``synth``. Importing the package itself loads nothing.
"""
__all__ = ["swih", "synth"]

"""GB300-native constant-capacitance-model ground-state library (arXiv 2404.04994).

The compute path is the C-ABI library ``libqarray.so`` (hand-written CUDA for
sm_103a); ``api`` is its thin ctypes binding and ``autograd`` wraps the soft
occupation in a ``torch.autograd.Function``.  Importing this package loads
nothing; the library is loaded on first use and its absence is an error.
"""
__all__ = ["api", "inputs"]

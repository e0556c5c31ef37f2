"""GB300-native batched Galactic-binary log-likelihood (Strub et al., arXiv:2307.03763).

The compute path is the C-ABI library ``libgb`` (hand-written CUDA for sm_103a,
declared in ``include/gb.h``); ``api`` is its thin Python binding.  Importing
this package does not load the library: ``api`` loads it on first use and
raises if it is missing.  ``workloads`` holds the seeded synthetic inputs.
"""
__all__ = ["api", "workloads", "build"]

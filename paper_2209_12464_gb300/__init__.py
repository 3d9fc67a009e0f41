"""RU-QLP (arXiv 2209.12464) on GB300: CUDA kernels behind a C ABI.

``paper_2209_12464_gb300.ruqlp`` is the thin ctypes binding of the C-ABI
library ``libruqlp.so`` (built from ``csrc/`` for sm_103a); ``workloads``
draws the seeded synthetic inputs.  Importing the package loads nothing; the
library is loaded on first use and a missing library is an error, never a
fallback.
"""
__all__ = ["ruqlp", "workloads"]

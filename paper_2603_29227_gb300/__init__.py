"""Kernel-SDF back-end query on GB300: local-GP signed distance, gradient and variance (arXiv 2603.29227).

The compute path is the CUDA library ``libksdf.so`` behind the C ABI declared in ``include/ksdf.h``;
``paper_2603_29227_gb300.ksdf`` is its thin ctypes binding (same function names) plus a
``torch.autograd.Function``.  Importing this package loads nothing: the library is opened on first use
and a missing build raises an error instead of falling back to any CPU code.
"""
__all__ = ["scenes"]

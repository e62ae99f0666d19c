"""Horizontal fusion of independent GPU kernels for GB300 (sm_103a).

The compute path is the C-ABI library ``libhfuse.so`` built from ``csrc/``;
``hfuse`` is its thin ctypes binding.  Importing the package does not load
the library; the first call into ``hfuse`` does, and fails loudly when it has
not been built.
"""
__all__ = ["hfuse", "workloads"]

"""GB300-native real-space exact exchange (arXiv 2405.01522 hot path).

The compute path is the C-ABI library ``librsx.so`` built from ``csrc/`` for sm_103a;
``rsx`` is its thin ctypes binding.  Importing this package loads nothing: the
library is opened on first use and the binding raises if it is missing.
"""
__all__ = ["inputs", "rsx"]

"""GB300-native parallel parser for regular expressions (arXiv 2503.06763).

The package holds the native library (``csrc/``: the host RE compiler and the
sm_103a CUDA kernels behind the C ABI of ``include/slpf_parser.h``), its build
script and a thin ctypes binding.  ``Regex(pattern).parse(text)`` returns the
clean SLPF of a device-resident text.
"""
from .native import KINDS, RE_OK, RE_REJECTED, STATUS_NAMES, Batch, Regex, ReError, load  # noqa: F401

__all__ = ["Regex", "Batch", "ReError", "load", "KINDS", "RE_OK", "RE_REJECTED", "STATUS_NAMES"]

"""GB300-native i-DEQ: inertial deep-equilibrium image restoration on sm_103a.

The compute path is the C-ABI library libideq.so (include/ideq.h) built from
csrc/; ``binding`` is its thin ctypes binding.  Importing ``binding`` without the
built library raises ImportError: there is no CPU fallback.
"""
__all__ = ["binding", "build"]

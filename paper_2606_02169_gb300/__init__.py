"""GB300-native matrix-free spin / truncated-boson Hamiltonian action.

y = H x on the full tensor-product basis with mixed-radix indexing ("Spin
Hamiltonian as Matrix-Free Linear Map"), in hand-written sm_103a CUDA behind
the C ABI of include/hm.h. This package is the thin Python binding.
"""
from ._capi import HmError, load  # noqa: F401
from .autograd import HamApply, LanczosE0, hamiltonian_apply, lanczos_e0  # noqa: F401
from .hamiltonian import Batch, Hamiltonian  # noqa: F401

__all__ = ["Hamiltonian", "Batch", "HamApply", "LanczosE0", "hamiltonian_apply", "lanczos_e0",
           "HmError", "load"]

"""GB300-native force of the Abacus N-body method (Garrison et al.): the
near-field pair sums, their adjoint, and the multipole/Taylor far field.

The hot path is libnf (CUDA, sm_103a) behind a C ABI (``include/nf.h``);
this package is its Python binding.  Importing it loads the library and
fails if it cannot: there is no CPU path.
"""
from . import _lib
from ._lib import NFError, nf_version
from .nearfield import (
    BatchedNearField,
    FarField,
    NearField,
    bin_particles,
    forces,
    forces_adjoint,
    forces_density,
    multipoles,
    near_field,
    stats,
    status,
    workspace,
)

_lib.load()

__all__ = [
    "_lib",
    "NFError",
    "nf_version",
    "BatchedNearField",
    "FarField",
    "NearField",
    "bin_particles",
    "forces",
    "forces_adjoint",
    "forces_density",
    "multipoles",
    "near_field",
    "stats",
    "status",
    "workspace",
]

"""GB300-native near-field force of the Abacus N-body method (Garrison et al.).

The hot path is libnf (CUDA, sm_103a) behind a C ABI (``include/nf.h``);
this package is its Python binding.  Importing it loads the library and
fails if it cannot: there is no CPU path.
"""
from . import _lib
from ._lib import NFError, nf_version
from .nearfield import (
    BatchedNearField,
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

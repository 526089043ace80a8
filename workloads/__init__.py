"""Seeded synthetic particle sets for the near-field force.

This package only draws inputs.  It holds none of the near-field method's
arithmetic, so both the CUDA path and the CPU oracle can take their inputs from
it without sharing any of the computation they are checked on.
"""
from .recipes import (
    Workload,
    uniform_positions,
    clustered_positions,
    plummer_eps,
    config_plain,
    config_clustered,
    config_large,
    config_adjoint,
    config_batched,
    upstream_gradient,
    fd_sample,
    named_config,
)

__all__ = [
    "Workload",
    "uniform_positions",
    "clustered_positions",
    "plummer_eps",
    "config_plain",
    "config_clustered",
    "config_large",
    "config_adjoint",
    "config_batched",
    "upstream_gradient",
    "fd_sample",
    "named_config",
]

"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package draws random numbers and lays out point sets, targets and initial
parameters. It holds none of the PINN method's arithmetic (no jets, residuals,
losses or gradients), so both sides may import it without sharing any of the
computation they are compared on.
"""
from .workloads import (  # noqa: F401
    SplitMix64, NetSpec, Problem, Batch, WORKLOADS, make_workload, layer_dims,
    param_count, init_params, ff_matrix, make_batch, family_specs, make_family,
    PDE_BURGERS, PDE_NS, PDE_MAXWELL, PDE_ADVECTION, PDE_ALLEN_CAHN,
)

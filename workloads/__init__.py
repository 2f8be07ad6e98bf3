"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only *generates* inputs: circuit topologies, Trotter-initialised
gates with seeded noise, raw random HVP directions and model parameters.  It
holds none of the arithmetic of the method itself (no cost, gradient, Hessian,
target unitary or state-vector contraction); both the CUDA path and the oracle
receive the same arrays from here and compute everything else independently.
"""
from .fermi_hubbard import (  # noqa: F401
    Problem,
    brickwall_layers,
    layer_pattern,
    trotter_times,
    trotter4_times,
    trotter_gate,
    parity_mask,
    make_problem,
    random_directions,
    random_unitary,
    config_problem,
    batch_problems,
    make_spinless_problem,
    spinless_gate,
)

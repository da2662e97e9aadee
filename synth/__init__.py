"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only draws random numbers and lays them out as problem inputs
(network widths, parameter vector, inputs X, one-hot labels Y).  It contains
none of the curvature arithmetic, so the oracle and the CUDA path can both
consume the same host buffers without sharing any method code.
"""

from .inputs import (  # noqa: F401
    Problem,
    SplitMix64Stream,
    make_problem,
    make_mlp,
    make_random_mlp,
    named_config,
    NAMED_CONFIGS,
)

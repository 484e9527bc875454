"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package holds only input generation: random regular graphs and QAOA
angles drawn from a counter-free SplitMix64 stream.  It contains none of the
method's arithmetic (no circuit, network, contraction or expectation value),
so the oracle and the CUDA path can both use it without sharing any code of
the method.
"""

from .rng import SplitMix64
from .graphs import random_regular_graph, ring_plus_pairs_graph, is_connected
from .workloads import WORKLOADS, Workload, workload, qaoa_angles

__all__ = [
    "SplitMix64",
    "random_regular_graph",
    "ring_plus_pairs_graph",
    "is_connected",
    "WORKLOADS",
    "Workload",
    "workload",
    "qaoa_angles",
]

"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random numbers and nothing else: it holds none of the
search method's arithmetic (no quantisation, no distances, no graph logic).
Both the CPU oracle and the CUDA library take what it produces as plain
input arrays.
"""

from .generators import (  # noqa: F401
    WORKLOADS,
    Mixture,
    density_sample,
    level_uniforms,
    make_mixture,
    sample_mixture,
    workload,
)

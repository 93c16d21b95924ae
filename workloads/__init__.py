"""Seeded synthetic workloads for the FINGER search path.

This package only draws random numbers: base vectors and queries with the
shapes and value distributions of the five benchmark configurations.  It holds
none of the search or table arithmetic, so the FP64 oracle and the CUDA path
can both take their inputs from it without sharing any method code.
"""
from .gen import (CONFIGS, WorkloadConfig, base_vectors, config, query_vectors,  # noqa: F401
                  training_queries, uneven_batches)

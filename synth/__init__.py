"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This package holds workload descriptors (sizes, physical constants, seeds) and
the seeded random draws of the KL coefficient vectors xi.  It contains none of
the method's arithmetic: no operator, no propagator, no surrogate, no
transform.  Both the CPU oracle and the CUDA path read their inputs from here,
so the two sides never share code beyond these draws.
"""
from .workloads import WORKLOADS, Workload, draw_train, draw_uneven_shapes, draw_xi, workload

__all__ = ["WORKLOADS", "Workload", "draw_xi", "draw_train", "draw_uneven_shapes", "workload"]

"""Seeded synthetic inputs (Plummer spheres, subsamples, ragged ensembles).

Shared by the oracle tests and the GPU path; holds no force, potential or
integrator arithmetic.
"""
from .plummer import (PLUMMER_A, Workload, adjoint_case, gaussian, plummer, plummer_offset, precision_offset,
                      ragged_batch, ragged_sizes, small_plain, subsample, throughput_plain)

__all__ = ["PLUMMER_A", "Workload", "adjoint_case", "gaussian", "plummer", "plummer_offset", "precision_offset",
           "ragged_batch", "ragged_sizes", "small_plain", "subsample", "throughput_plain"]

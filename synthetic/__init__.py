"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method itself: it only draws blob
positions, reaction rates and source fields. Every array it returns is a plain
NumPy FP64 array, so the same bytes reach the GPU (after a host-to-device copy)
and the CPU oracle.

Workloads follow the shapes used in the paper's experiments: a periodic cubic
grid of spacing h, a uniform source, and blobs that are either on a cubic
lattice (Sec. III.E, Sec. IV.B) or at random non-overlapping centres, here
placed by random sequential addition in place of the external hard-sphere
packings of Sec. IV.C.
"""
from .placement import (rsa_positions, lattice_positions, single_blob_position,
                        loguniform_rates, uniform_source, Workload, workload, batch_workloads)

__all__ = ["rsa_positions", "lattice_positions", "single_blob_position",
           "loguniform_rates", "uniform_source", "Workload", "workload", "batch_workloads"]

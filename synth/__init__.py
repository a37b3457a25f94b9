"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This package produces inputs only: analytically rendered depth frames,
camera-to-world poses, pinhole intrinsics and the tabulated sensor-noise
model.  It contains none of the mapping method's arithmetic (no voxel
traversal, no sensor likelihood, no message passing), so the oracle and the
GPU path can both consume it without sharing any of the method's code.
"""
from .scenes import (  # noqa: F401
    Grid, Camera, NoiseTable, Frame, Workload,
    sigma_gen, make_workload, WORKLOADS,
)

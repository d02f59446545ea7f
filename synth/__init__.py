"""Seeded synthetic video streams for background subtraction.

This package only produces input data (frames, ground-truth masks, a planted
subspace).  It holds none of pROST's arithmetic, so both the FP64 oracle tests
and the CUDA path read their inputs from here without sharing method code.
"""

from .video import SyntheticVideo, WORKLOADS, make_workload, batched_workload, window_workload, random_orthonormal

__all__ = ["SyntheticVideo", "WORKLOADS", "make_workload", "batched_workload", "window_workload", "random_orthonormal"]

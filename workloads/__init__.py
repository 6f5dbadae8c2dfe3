"""Seeded synthetic inputs shared by the oracle and the CUDA library.

Meshes come as face lists, cameras as per-frame FP64/FP32 parameters; no part
of the method (halfedge ingest, bisection, CBT) lives here.
"""
from . import cameras, configs, meshes  # noqa: F401

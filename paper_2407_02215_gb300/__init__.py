"""GB300-native (sm_103a) adaptive bisection with a concurrent binary tree.

The per-frame update of Benyoub & Dupuy, "Concurrent Binary Trees for
Large-Scale Game Components" (2024), as a C-ABI CUDA library (libcbt.so,
include/cbt.h) with a thin Python binding. Import fails loudly when the CUDA
library has not been built.
"""
from .build import build as build_library  # noqa: F401
from .cbt import (CBT, CBT_NULL, Batch, CBTError, Server, halfedges_from_faces, load,  # noqa: F401
                  sum_reduce, compact, update_many, vertices_to_host_async, workspace_bytes)

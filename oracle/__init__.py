"""CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It never imports the CUDA package.
"""
from .oracle import Oracle, OracleError, cbt_compact, cbt_one_to_bit, cbt_sum_reduction, cbt_zero_to_bit  # noqa: F401
from .oracle import decode_weights, fbm, halfedges_from_faces, lod_test, lowbias32, splitmix64  # noqa: F401

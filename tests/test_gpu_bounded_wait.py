"""Failure detection without a GPU fault: a grid barrier whose last arrival
never comes gives up after its poll limit, the kernel returns, the host
reads the timeout status, and the same context then runs frames that still
match the oracle."""
import pytest

import workloads as W
from oracle import Oracle
from tests.gpu_helpers import run_pair

pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_context_survives():
    import ctypes

    import torch

    import paper_2407_02215_gb300 as P
    P.build_library()
    lib = P.load()
    scratch = torch.zeros(64, dtype=torch.int32, device="cuda")  # 256 bytes, allocator-aligned
    rc = lib.cbt_selftest_bounded_wait(ctypes.c_void_p(scratch.data_ptr()), 4, 1 << 12, None)
    assert rc == 7  # CBT_ETIMEOUT
    torch.cuda.synchronize()
    # the context is intact: a fused instance still matches the oracle
    spec = W.configs.config1(n_frames=6)
    run_pair(spec.mesh, spec.D, spec.max_depth, spec.frames, P.CBT, Oracle)

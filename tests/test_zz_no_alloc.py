"""The no-allocation entry point cbt_reduce_compact_static.

It serves callers that cannot allocate device memory: real-time frame loops
where cudaMalloc/cudaFree would synchronize the device, or applications whose
device memory all comes from their own allocator. Its scratch is a static
device array, so it must give the same CBT sums and live-slot list as the
update path (cbt_cbt / cbt_leaves, whose scratch lives in the caller's
workspace), call after call. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from workloads.cameras import MODE_RANDOM, forced_params

pytestmark = pytest.mark.gpu


def _setup():
    import torch

    import paper_2407_02215_gb300 as P
    P.build_library()
    lib = P.load()
    lib.cbt_reduce_compact_static.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.cbt_reduce_compact_static.restype = ctypes.c_int
    return torch, P, lib


def _check_against_update_path(torch, P, lib, mesh, D, max_depth, frames, calls=2):
    g = P.CBT(mesh, D, max_depth)
    words = max(1, (1 << D) // 32)
    sums2 = torch.zeros(2 * words, dtype=torch.int32, device="cuda")
    live2 = torch.zeros(1 << D, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    per = len(frames) // calls
    for c in range(calls):
        for fp in frames[c * per:(c + 1) * per]:
            g.update(fp)
        bits, sums = g.cbt()
        slots, _, _ = g.leaves()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = lib.cbt_reduce_compact_static(ctypes.c_void_p(bits.data_ptr()), D,
                                           ctypes.c_void_p(sums2.data_ptr()),
                                           ctypes.c_void_p(live2.data_ptr()),
                                           ctypes.c_void_p(count.data_ptr()), stream)
        assert rc == 0
        torch.cuda.synchronize()
        n = int(count.item())
        assert n == slots.numel(), f"call {c}: count {n} vs {slots.numel()}"
        assert torch.equal(live2[:n], slots), f"call {c}: live slots differ"
        assert torch.equal(sums2[1:], sums[1:]), f"call {c}: sums differ"


def test_static_scratch_multi_tile_pool():
    """A 2^20 pool (32 tiles of 1024 words) after 6 and after 12 frames."""
    torch, P, lib = _setup()
    mesh = W.meshes.grid_mesh(40, 40, 0.1, seed=9)
    cams = W.cameras.flythrough_path(12, seed=9, alt_lo=0.03)
    frames = [W.cameras.frame_params(c, 2.0) for c in cams]
    _check_against_update_path(torch, P, lib, mesh, 20, 22, frames)


def test_static_scratch_pool_smaller_than_a_word():
    """A 2^4 pool (16 slots, part of one word), two calls in a row."""
    torch, P, lib = _setup()
    frames = [forced_params(MODE_RANDOM, seed=3) for _ in range(8)]
    _check_against_update_path(torch, P, lib, W.meshes.fig1_mesh(), 4, 6, frames)


def test_static_scratch_rejects_oversized_pools():
    torch, P, lib = _setup()
    z = ctypes.c_void_p(1)
    assert lib.cbt_reduce_compact_static(z, 28, z, z, z, None) == 2  # CBT_ECAPACITY
    assert lib.cbt_reduce_compact_static(None, 10, z, z, z, None) == 1  # CBT_EINVAL

"""The no-allocation entry point cbt_reduce_compact_static.

It serves callers that cannot allocate device memory: real-time frame loops
in which cudaMalloc/cudaFree would synchronize the device, and applications
whose device memory all comes from their own allocator. Its scratch is a
static device array, so what is checked here is that it gives what the rest
of the library and the oracle give, call after call on the same array:
  - on seeded random bitfields (pool sizes 2^1 .. 2^22, densities 0 to 1),
    every node of the sum tree and the whole live-slot list against the
    oracle's SumReduction and CachePointers (Sec. 3.1, Alg. 7), and against
    the allocating entry points cbt_sum_reduce and cbt_compact;
  - at 2^27 slots (all 4096 tiles of its scratch) against those entry points;
  - after frames of the update, against cbt_cbt and cbt_leaves;
  - a status word of 0 in sums[0] and the set-bit count in count.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O
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


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _static(torch, lib, bits, D):
    """One call; returns (sums, live, count) on the host."""
    words = max(1, (1 << D) // 32)
    sums = torch.full((2 * words,), -1, dtype=torch.int32, device="cuda")
    live = torch.full((1 << D,), -1, dtype=torch.int32, device="cuda")
    count = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.cbt_reduce_compact_static(_p(bits), D, _p(sums), _p(live), _p(count), stream) == 0
    torch.cuda.synchronize()
    return (sums.cpu().numpy().view(np.uint32), live.cpu().numpy().view(np.uint32),
            int(count.cpu().numpy().view(np.uint32)[0]))


def _oracle(words_host, D):
    """The oracle's CBT (2^(D+1) nodes, leaves = the bits) and live list."""
    cap = 1 << D
    bits = np.unpackbits(words_host.view(np.uint8), bitorder="little")[:cap].astype(np.uint32)
    cbt = np.zeros(2 * cap, np.uint32)
    cbt[cap:] = bits
    cbt = O.cbt_sum_reduction(D, cbt)
    return cbt, O.cbt_compact(D, cbt)


def _bitfield(rng, D, density):
    words = max(1, (1 << D) // 32)
    bits = rng.random(words * 32) < density
    return np.packbits(bits, bitorder="little").view(np.uint32)[:words].copy()


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6, 7, 8, 12, 15, 20, 22])
def test_static_against_oracle_and_entry_points(D):
    torch, P, lib = _setup()
    rng = np.random.default_rng(100 + D)
    words = max(1, (1 << D) // 32)
    for density in (0.0, 0.03, 0.5, 0.97, 1.0):
        results = []
        for call in range(2):  # two calls in a row on the same static scratch
            host = _bitfield(rng, D, density)
            bits = torch.from_numpy(host.view(np.int32)).cuda()
            sums, live, count = _static(torch, lib, bits, D)
            cbt, ref_live = _oracle(host, D)
            n = int(cbt[1])
            assert sums[0] == 0, f"D={D} call {call}: status {sums[0]:#x}"
            assert count == n
            assert np.array_equal(sums[1:2 * words], cbt[1:2 * words]), f"D={D} d={density} call {call}: sums"
            assert np.array_equal(live[:n], ref_live), f"D={D} d={density} call {call}: live"
            if D >= 5:  # the allocating entry points take D >= 5
                s2 = torch.zeros(2 * words, dtype=torch.int32, device="cuda")
                l2 = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
                P.sum_reduce(bits, D, s2)
                P.compact(bits, s2, D, l2)
                torch.cuda.synchronize()
                assert np.array_equal(s2.cpu().numpy().view(np.uint32)[1:], sums[1:])
                assert np.array_equal(l2.cpu().numpy().view(np.uint32)[:n], live[:n])
            results.append(count)
        assert len(results) == 2


def test_static_at_its_largest_pool():
    """2^27 slots, half of the bits set: every tile of the static scratch;
    equal to cbt_sum_reduce and cbt_compact, twice."""
    torch, P, lib = _setup()
    D = 27
    words = 1 << (D - 5)
    g = torch.Generator(device="cuda").manual_seed(27)
    for call in range(2):
        bits = torch.randint(-2**31, 2**31 - 1, (words,), dtype=torch.int32, device="cuda", generator=g)
        sums, live, count = _static(torch, lib, bits, D)
        s2 = torch.zeros(2 * words, dtype=torch.int32, device="cuda")
        P.sum_reduce(bits, D, s2)
        torch.cuda.synchronize()
        n = int(s2[1].item())
        l2 = torch.zeros(n, dtype=torch.int32, device="cuda")
        P.compact(bits, s2, D, l2)
        torch.cuda.synchronize()
        assert sums[0] == 0 and count == n
        assert np.array_equal(s2.cpu().numpy().view(np.uint32)[1:], sums[1:])
        assert np.array_equal(l2.cpu().numpy().view(np.uint32), live[:n])
        del bits, s2, l2


def _check_against_update_path(torch, P, lib, mesh, D, max_depth, frames, calls=2):
    g = P.CBT(mesh, D, max_depth)
    per = len(frames) // calls
    for c in range(calls):
        for fp in frames[c * per:(c + 1) * per]:
            g.update(fp)
        bits, sums = g.cbt()
        slots, _, _ = g.leaves()
        sums2, live2, n = _static(torch, lib, bits, D)
        assert sums2[0] == 0
        assert n == slots.numel(), f"call {c}: count {n} vs {slots.numel()}"
        assert np.array_equal(live2[:n], slots.cpu().numpy().view(np.uint32)), f"call {c}: live slots differ"
        assert np.array_equal(sums2[1:], sums.cpu().numpy().view(np.uint32)[1:]), f"call {c}: sums differ"


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

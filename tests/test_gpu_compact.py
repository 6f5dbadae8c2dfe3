"""CachePointers (Alg. 7 for every index) over a caller's bitfield
(cbt_compact after cbt_sum_reduce): the live list equals the oracle's
OneToBitID(i) for every i at sizes it finishes quickly, in both kernels
(one warp below 4096 words, chunks above); at 2^27 slots (the size the paper
times the prior method at) the list is checked by what determines it at any
size: strictly increasing, every listed bit set, as many entries as set bits."""
import numpy as np
import pytest

from oracle import cbt_compact, cbt_sum_reduction

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2407_02215_gb300 as P
    P.build_library()
    return P


def _bits(D, density, seed):
    rng = np.random.default_rng(seed)
    b = (rng.random(1 << D) < density).astype(np.uint8)
    return b, np.packbits(b, bitorder="little").view(np.uint32)


def _gpu_compact(P, words, D, cap=None):
    import torch
    bits = torch.from_numpy(words.view(np.int32).copy()).cuda()
    sums = torch.zeros(2 * words.size, dtype=torch.int32, device="cuda")
    P.sum_reduce(bits, D, sums)
    n = int(sums[1].item())
    live = torch.full((n + 64 if cap is None else cap,), -1, dtype=torch.int32, device="cuda")
    P.compact(bits, sums, D, live)
    torch.cuda.synchronize()
    return n, live.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("D,density", [(5, 0.5), (9, 0.0), (11, 1.0), (16, 0.3), (17, 0.5), (18, 0.02),
                                       (20, 0.5), (22, 0.97)])
def test_matches_oracle(P, D, density):
    b, words = _bits(D, density, seed=100 + D)
    cbt = np.zeros(2 << D, np.uint32)
    cbt[1 << D:] = b
    want = cbt_compact(D, cbt_sum_reduction(D, cbt))
    n, got = _gpu_compact(P, words, D)
    assert n == want.size
    assert np.array_equal(got[:n], want)
    assert np.all(got[n:] == 0xFFFFFFFF)  # nothing written past the count


@pytest.mark.parametrize("D", [10, 19])
def test_capacity_bound(P, D):
    """Positions at index >= cap are dropped; the first cap are exact."""
    b, words = _bits(D, 0.5, seed=D)
    ones = np.flatnonzero(b).astype(np.uint32)
    cap = ones.size // 3
    _, got = _gpu_compact(P, words, D, cap=cap)
    assert np.array_equal(got, ones[:cap])


def test_full_size_properties(P):
    D = 27
    b, words = _bits(D, 0.5, seed=27)
    del b
    n, got = _gpu_compact(P, words, D)
    live = got[:n].astype(np.int64)
    pc = int(np.unpackbits(words.view(np.uint8)).sum())
    assert n == pc
    assert np.all(np.diff(live) > 0)
    assert live[0] >= 0 and live[-1] < (1 << D)
    assert np.all((words[live >> 5] >> (live & 31).astype(np.uint32)) & 1)
    assert np.all(got[n:] == 0xFFFFFFFF)


def test_rejects_bad_arguments(P):
    import ctypes
    lib = P.load()
    z = ctypes.c_void_p(0)
    assert lib.cbt_compact(z, z, 20, z, 0, None) == 1  # CBT_EINVAL: NULL
    import torch
    t = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    assert lib.cbt_compact(p, p, 4, p, 16, None) == 1    # D < 5
    assert lib.cbt_compact(p, p, 29, p, 16, None) == 2   # CBT_ECAPACITY

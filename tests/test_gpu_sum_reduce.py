"""SumReduction (Sec. 3.1) over a caller's bitfield (cbt_sum_reduce): every
node of the sum tree equals the oracle's at sizes it finishes quickly; at
2^27 slots (the size the paper times the prior method's reduction at) the
tree is checked by properties that hold at any size: the word level is the
popcount of the words, every node is the sum of its children, the root is
the number of set bits."""
import numpy as np
import pytest

from oracle import cbt_sum_reduction

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2407_02215_gb300 as P
    P.build_library()
    return P


def _bits(D, density, seed):
    rng = np.random.default_rng(seed)
    n = 1 << D
    b = (rng.random(n) < density).astype(np.uint8)
    return b, np.packbits(b, bitorder="little").view(np.uint32)


def _gpu_sums(P, words, D):
    import torch
    bits = torch.from_numpy(words.view(np.int32).copy()).cuda()
    sums = torch.zeros(2 * words.size, dtype=torch.int32, device="cuda")
    P.sum_reduce(bits, D, sums)
    torch.cuda.synchronize()
    return sums.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("D,density", [(5, 0.5), (8, 0.0), (15, 1.0), (16, 0.3), (17, 0.7), (18, 0.2),
                                       (20, 0.5), (22, 0.9)])
def test_matches_oracle(P, D, density):
    b, words = _bits(D, density, seed=D)
    cbt = np.zeros(2 << D, np.uint32)
    cbt[1 << D:] = b
    want = cbt_sum_reduction(D, cbt)
    got = _gpu_sums(P, words, D)
    W = words.size
    assert np.array_equal(got[1:2 * W], want[1:2 * W])


def test_full_size_properties(P):
    D = 27
    _, words = _bits(D, 0.37, seed=27)
    got = _gpu_sums(P, words, D).astype(np.int64)
    assert got[0] == 0  # the finished-chunk counter is left at 0
    W = words.size
    pc = np.unpackbits(words.view(np.uint8)).reshape(W, 32).sum(axis=1)
    assert np.array_equal(got[W:2 * W], pc)
    assert np.array_equal(got[1:W], got[2:2 * W:2] + got[3:2 * W:2])
    assert got[1] == int(pc.sum())


def test_rejects_bad_arguments(P):
    import ctypes
    lib = P.load()
    z = ctypes.c_void_p(0)
    assert lib.cbt_sum_reduce(z, 20, z, None) == 1   # CBT_EINVAL: NULL
    import torch
    t = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    assert lib.cbt_sum_reduce(p, 4, p, None) == 1     # D < 5
    assert lib.cbt_sum_reduce(p, 29, p, None) == 2    # CBT_ECAPACITY
    q = ctypes.c_void_p(t.data_ptr() + 4)
    assert lib.cbt_sum_reduce(q, 10, p, None) == 1    # misaligned

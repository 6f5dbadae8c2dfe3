"""Pin of the oracle's gate and allocation order, by an independent
restatement on tiny pools.

The test recomputes, from the frame-start state alone (the CBT, heap IDs and
links the oracle exports before the frame), which requests the gate grants
and which slot every new bisector takes, then checks the oracle's frame
against it. It never calls the oracle's update to predict: the restatement
below is written from the paper and the readings it needs.

- Wishes: the geometry-free modes only (RANDOM, from the published SplitMix64
  of Steele, Lea & Flood 2014; LIST; FORCE_SPLIT; FORCE_MERGE), so that no
  vertex arithmetic is involved.
- Split cost: the compatibility chain (Alg. 3, command form R5) on the
  frame-start links: 2 for the requester, 3 for every coarser member, 2 for a
  diamond partner; or 3d + 4 under the paper's gate (Sec. 3.3 kernel 4).
- Merge requests: the Alg. 4 group on the frame-start links, charged at the
  member with the smallest heap ID with its parent count (2 under the paper's
  gate), when every member wishes to merge.
- Gate (R6 reading of the allocation counter of Sec. 3.3 kernels 4-5): merge
  requests in ascending slot of their charged member, granted while the
  running total (granted or not) stays within the free slots F; then split
  requests in ascending slot, granted while the granted merge total plus
  their running total stays within F. A request past the first one that does
  not fit is denied even if it would fit on its own.
- Fates: granted chains mark their members; a group merges when its charged
  member was granted, every member wishes to merge and none was marked.
- Slots (R7 reading of Alg. 8 and ReserveBlocks, Sec. 3.2-3.3): the new
  bisectors in ascending slot of the bisector they come from, a split
  family's leaves depth first (child 0's subtree before child 1's), a
  merge's parents in ascending heap ID; the k-th takes the k-th zero bit of
  the frame-start bitfield, found here by brute force.
"""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from workloads.cameras import (GATE_CHAIN, GATE_PAPER, MODE_FORCE_MERGE, MODE_FORCE_SPLIT, MODE_LIST,
                               MODE_RANDOM, forced_params)

NULL = 0xFFFFFFFF
M64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64's output function on the counter x (Steele et al. 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_restatement_matches_published_vector():
    """The first outputs of SplitMix64 from state 0 and from state 1234567
    (published sequences): the state advances by the golden gamma and each
    output is the mix of the advanced state."""
    gamma = 0x9E3779B97F4A7C15
    for seed, want in ((0, [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]),
                       (1234567, [6457827717110365317, 3203168211198807973, 9817491932198370423])):
        out = [splitmix64((seed + k * gamma) & M64) for k in range(3)]
        assert out == want


class Start:
    """The frame-start state, from the oracle's export."""

    def __init__(self, o):
        e = o.export()
        self.cap = o.cap
        self.bits = e["cbt"][self.cap:].astype(bool)
        self.heap = [int(x) for x in e["heap"]]
        self.twin = [int(x) for x in e["twin"]]
        self.next = [int(x) for x in e["next"]]
        self.prev = [int(x) for x in e["prev"]]
        self.ch = o.ch
        self.max_depth = o.max_depth
        self.live = [int(s) for s in np.flatnonzero(self.bits)]

    def depth(self, s):
        return self.heap[s].bit_length() - 1 - self.ch


def wishes(st, fp, frame):
    split, merge = {}, {}
    key = splitmix64(((fp.seed & 0xFFFFFFFF) << 32) | frame)
    slist = set(int(x) for x in fp.split_list)
    mlist = set(int(x) for x in fp.merge_list)
    for s in st.live:
        j, d = st.heap[s], st.depth(s)
        can_split = d < st.max_depth
        if fp.mode == MODE_FORCE_SPLIT:
            sw, mw = can_split, False
        elif fp.mode == MODE_FORCE_MERGE:
            sw, mw = False, d >= 1
        elif fp.mode == MODE_RANDOM:
            sw = can_split and (splitmix64(j ^ key) & 7) == 0
            mw = (not sw) and d >= 1 and (splitmix64((j >> 1) ^ key) & 1) == 1
        else:
            sw = can_split and j in slist
            mw = (not sw) and d >= 1 and j in mlist
        split[s], merge[s] = sw, mw
    return split, merge


R, N, P = 1, 2, 4


def chain(st, b):
    """Members after b of b's compatibility chain with their split bits, and
    whether it ends at a diamond partner (Alg. 3 on the frame-start links)."""
    members, cur = [], b
    while True:
        t = st.twin[cur]
        if t == NULL:
            return members, False
        if st.twin[t] == cur:
            members.append((t, R))
            return members, True
        if st.next[t] == cur:
            members.append((t, R | N))
        elif st.prev[t] == cur:
            members.append((t, R | P))
        else:
            raise AssertionError("non-conforming chain")
        assert st.depth(t) + 1 == st.depth(cur)
        cur = t


def group(st, s1):
    """Alg. 4: the members (s1, sibling, then the two across the outer half of
    the refinement edge, if any) and the parents' heap IDs, or None."""
    j1 = st.heap[s1]
    if st.depth(s1) < 1:
        return None
    odd = j1 & 1
    s2 = st.prev[s1] if odd else st.next[s1]
    s3 = st.next[s1] if odd else st.prev[s1]
    if s2 == NULL or st.heap[s2] >> 1 != j1 >> 1:
        return None
    if s3 == NULL:
        return [s1, s2], [j1 >> 1]
    j3 = st.heap[s3]
    if j3.bit_length() != j1.bit_length() or j3 >> 1 == j1 >> 1:
        return None
    s4 = st.next[s3] if odd else st.prev[s3]
    if s4 == NULL or st.heap[s4] >> 1 != j3 >> 1:
        return None
    return [s1, s2, s3, s4], sorted([j1 >> 1, j3 >> 1])


def family(j, bits):
    """Leaves of a split with these bits, child 0's subtree first."""
    c0 = [4 * j, 4 * j + 1] if bits & P else [2 * j]
    c1 = [4 * j + 2, 4 * j + 3] if bits & N else [2 * j + 1]
    return c0 + c1


def predict(st, fp, frame):
    F = st.cap - len(st.live)
    split, merge = wishes(st, fp, frame)
    paper = fp.gate == GATE_PAPER
    scost, chains, mcost, groups = {}, {}, {}, {}
    for s in st.live:
        if split[s]:
            members, diamond = chain(st, s)
            chains[s] = members
            scost[s] = 3 * st.depth(s) + 4 if paper else 2 + 3 * (len(members) - int(diamond)) + 2 * int(diamond)
        if merge[s]:
            g = group(st, s)
            if g is None:
                continue
            mem, parents = g
            charged = min(mem, key=lambda m: st.heap[m])
            if charged == s and all(merge[m] for m in mem):
                mcost[s] = 2 if paper else len(parents)
                groups[s] = (mem, parents)
    # gate: merges, then splits, each a prefix over ascending slots
    mgrant, run, mg = set(), 0, 0
    for s in st.live:
        if s in mcost:
            run += mcost[s]
            if run <= F:
                mgrant.add(s)
                mg = run
    sgrant, run = set(), 0
    for s in st.live:
        if s in scost:
            run += scost[s]
            if mg + run <= F:
                sgrant.add(s)
    # fates
    bits = {}
    for s in st.live:
        if s in sgrant:
            bits[s] = bits.get(s, 0) | R
            for t, b in chains[s]:
                bits[t] = bits.get(t, 0) | b
    valid = [s for s in st.live if s in groups and s in mgrant
             and all(merge[m] and not bits.get(m, 0) for m in groups[s][0])]
    # new records in canonical order, the k-th on the k-th free bit
    new, gone = [], set()
    for s in st.live:
        if bits.get(s, 0):
            new += family(st.heap[s], bits[s])
            gone.add(s)
        elif s in valid:
            new += groups[s][1]
            gone.update(groups[s][0])
    free = np.flatnonzero(~st.bits)
    assert len(new) <= F
    placed = {int(free[k]): j for k, j in enumerate(new)}
    return dict(F=F, split_wishes=sum(split.values()), merge_candidates=len(mcost),
                split_granted=len(sgrant), merge_granted=len(mgrant), merge_groups=len(valid),
                allocated=len(new), placed=placed, gone=gone, denied=len(scost) - len(sgrant) +
                len(mcost) - len(mgrant))


def check_frame(o, fp, frame):
    st = Start(o)
    want = predict(st, fp, frame)
    got = o.update(fp)
    assert got["frame"] == frame
    for k in ("split_wishes", "merge_candidates", "split_granted", "merge_granted", "merge_groups",
              "allocated"):
        assert got[k] == want[k], (k, got[k], want[k])
    after = o.export()
    bits_after = after["cbt"][o.cap:].astype(bool)
    expect_bits = st.bits.copy()
    for s in want["gone"]:
        expect_bits[s] = False
    for s in want["placed"]:
        assert not st.bits[s]
        expect_bits[s] = True
    assert np.array_equal(bits_after, expect_bits)
    for s, j in want["placed"].items():
        assert int(after["heap"][s]) == j, (s, int(after["heap"][s]), j)
    for s in st.live:
        if s not in want["gone"]:
            assert int(after["heap"][s]) == st.heap[s]
    return want


MESHES = [
    ("fig1", lambda: W.meshes.fig1_mesh()),
    ("tetra", lambda: W.meshes.tetra_mesh()),
    ("grid2", lambda: W.meshes.grid_mesh(2, 2, 0.5, seed=7)),
    ("cube", lambda: W.meshes.cube_mesh()),
]


def _frames(seed):
    rng = np.random.default_rng(seed)
    out = [forced_params(MODE_FORCE_SPLIT)] * 3
    for k in range(24):
        r = k % 6
        if r == 3:
            out.append(forced_params(MODE_FORCE_MERGE, gate=GATE_PAPER if k % 12 == 9 else GATE_CHAIN))
        elif r == 5:
            out.append(forced_params(MODE_FORCE_SPLIT, gate=GATE_PAPER if k % 12 == 5 else GATE_CHAIN))
        else:
            out.append(forced_params(MODE_RANDOM, seed=int(rng.integers(1, 1 << 31)),
                                     gate=GATE_PAPER if k % 4 == 1 else GATE_CHAIN))
    return out


@pytest.mark.parametrize("name,make", MESHES)
@pytest.mark.parametrize("D", [4, 5, 6, 7])
def test_gate_and_slots_match_restatement(name, make, D):
    mesh = make()
    H = mesh.H
    if (1 << D) < H:
        pytest.skip("pool smaller than the roots")
    o = Oracle(mesh, D=D, max_depth=9)
    denied = allocated = 0
    for frame, fp in enumerate(_frames(D * 31 + H)):
        want = check_frame(o, fp, frame)
        denied += want["denied"]
        allocated += want["allocated"]
    assert allocated > 0


def test_gate_binds_in_the_pinned_runs():
    """The tiny pools do exercise the prefix cutoff: requests are denied while
    others are granted in the same frame, for merges and for splits."""
    o = Oracle(W.meshes.cube_mesh(), D=6, max_depth=9)
    seen_split_cut = seen_merge_cut = False
    for frame, fp in enumerate(_frames(6 * 31 + 24)):
        want = check_frame(o, fp, frame)
        if 0 < want["split_granted"] < want["split_wishes"]:
            seen_split_cut = True
        if 0 < want["merge_granted"] < want["merge_candidates"]:
            seen_merge_cut = True
    assert seen_split_cut and seen_merge_cut


def test_list_frames_with_chains_and_quads():
    """Requests named by heap ID on a 2x2 grid: splits whose chains cross
    roots and end in diamonds, then merges of quads and border pairs, with a
    pool that cannot hold every request."""
    mesh = W.meshes.grid_mesh(2, 2, 0.0, seed=3)
    o = Oracle(mesh, D=7, max_depth=9)
    frame = 0
    rng = np.random.default_rng(11)
    for _ in range(3):
        check_frame(o, forced_params(MODE_FORCE_SPLIT), frame)
        frame += 1
    for k in range(30):
        st = Start(o)
        heaps = np.array([st.heap[s] for s in st.live], np.uint64)
        pick = rng.random(heaps.size)
        fp = forced_params(MODE_LIST, split_list=np.sort(heaps[pick < 0.2]),
                           merge_list=np.sort(np.concatenate([heaps[pick > 0.4], heaps[pick > 0.4] ^ 1]).astype(np.uint64)),
                           gate=GATE_PAPER if k % 5 == 4 else GATE_CHAIN)
        check_frame(o, fp, frame)
        frame += 1


def test_split_cost_lower_bounds():
    """The bounds the single-instance frame skips chain walks with: a split
    wish under a root whose halfedge has a Twin has a Twin itself (its
    refinement edge lies inside the root triangle, on an edge to the face's
    centroid, or on that halfedge) and costs at least 4 under the chain gate
    (its own pair, plus the Twin's pair when they form a diamond, else at
    least 3 for a coarser Twin and more down the chain); under a boundary
    halfedge it can cost 2. On the pinned runs every split wish keeps to
    these bounds (the restated chain, which the frames above match against
    the oracle), the Twin exists wherever the root's does, and both kinds of
    root occur."""
    seen = {2: 0, 4: 0}
    for name, make in MESHES:
        mesh = make()
        o = Oracle(mesh, D=7, max_depth=9)
        root_twin = o.halfedges["twin"]
        for frame, fp in enumerate(_frames(7 * 31 + mesh.H)):
            st = Start(o)
            split, _ = wishes(st, fp, frame)
            for s in st.live:
                if not split[s]:
                    continue
                h = (st.heap[s] >> st.depth(s)) - (1 << st.ch)
                members, diamond = chain(st, s)
                cost = 2 + 3 * (len(members) - int(diamond)) + 2 * int(diamond)
                bound = 4 if root_twin[h] >= 0 else 2
                if bound == 4:
                    assert st.twin[s] != NULL, (name, frame, s)
                assert cost >= bound, (name, frame, s, cost)
                seen[bound] += 1
            o.update(fp)
    assert seen[2] > 0 and seen[4] > 0

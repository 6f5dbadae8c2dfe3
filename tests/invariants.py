"""Exact invariant checks of a bisector state, independent of both
implementations.

Vertices are rebuilt symbolically, top-down, with the per-level bisection rule
of Eq. 1 (child 0 = (v0, v2, m), child 1 = (v2, v1, m), m = (v0 + v1) / 2)
starting from the root bisector (Vert(h), Vert(Next h), centroid of the face)
of Sec. 2.2. A point is a rational combination of mesh vertices and face
centroids, so equality is exact and the checks do not depend on floating point.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

NULL = 0xFFFFFFFF


def bitlen(x: int) -> int:
    return int(x).bit_length()


def depth_of(j: int, ch: int) -> int:
    return bitlen(j) - 1 - ch


def root_of(j: int, ch: int) -> int:
    return (j >> depth_of(j, ch)) - (1 << ch)


def _mid(a, b):
    out = dict(a)
    for k, v in b.items():
        out[k] = out.get(k, 0) + v
    return {k: v / 2 for k, v in out.items() if v != 0}


def _key(p):
    return tuple(sorted(p.items()))


def symbolic_vertices(j: int, ch: int, he) -> tuple:
    """The three vertices of bisector j as hashable exact combinations."""
    d = depth_of(j, ch)
    h = root_of(j, ch)
    v = [{("v", int(he["vert"][h])): Fraction(1)},
         {("v", int(he["vert"][he["next"][h]])): Fraction(1)},
         {("c", int(he["face"][h])): Fraction(1)}]
    for lvl in range(d - 1, -1, -1):
        b = (j >> lvl) & 1
        m = _mid(v[0], v[1])
        v = [v[0], v[2], m] if b == 0 else [v[2], v[1], m]
    return tuple(_key(p) for p in v)


def check_state(slots, heap, links, he, ch: int, max_depth: int, cbt=None, pos=None,
                root_table=None):
    """Raises AssertionError unless the leaves form a conforming, edge-matched
    triangulation covering every root bisector exactly once.

    slots/heap/links: the live bisectors (ascending slots), links [N][3] as
    (Twin, Next, Prev) slots. he: halfedge arrays of the mesh.
    """
    slots = [int(s) for s in slots]
    heap = [int(j) for j in heap]
    links = np.asarray(links, np.int64)
    H = len(he["twin"])
    assert slots == sorted(slots)
    slot_index = {s: i for i, s in enumerate(slots)}
    # Partition: every root covered exactly once (integer measure 2^-d).
    cover = [0] * H
    for j in heap:
        d = depth_of(j, ch)
        assert 0 <= d <= max_depth, (j, d)
        cover[root_of(j, ch)] += 1 << (max_depth - d)
    assert all(c == 1 << max_depth for c in cover), "leaves do not partition the roots"
    assert len(set(heap)) == len(heap)
    # Border segments of the mesh, as vertex-index pairs.
    border = set()
    for h in range(H):
        if he["twin"][h] == -1:
            a, b = int(he["vert"][h]), int(he["vert"][he["next"][h]])
            border.add(frozenset((("v", a), ("v", b))))
    edges = {}
    for i, j in enumerate(heap):
        v = symbolic_vertices(j, ch, he)
        for e, (a, b) in enumerate(((0, 1), (1, 2), (2, 0))):
            k = frozenset((v[a], v[b]))
            edges.setdefault(k, []).append((i, e))
    for k, users in edges.items():
        assert len(users) in (1, 2), f"edge shared by {len(users)} bisectors"
        if len(users) == 1:
            i, e = users[0]
            assert links[i, e] == NULL, "unmatched edge with a neighbour link"
            keys = set()
            for p in k:
                keys |= {name for name, _ in p}
            assert any(keys <= set(bk) for bk in border), "hanging edge not on the mesh border"
        else:
            (i, e), (i2, e2) = users
            assert links[i, e] == slots[i2], "link does not name the bisector across the edge"
            assert links[i2, e2] == slots[i], "link does not name the bisector across the edge"
    for i in range(len(slots)):
        for e in range(3):
            t = int(links[i, e])
            assert t == NULL or t in slot_index, "link to a dead slot"
    if cbt is not None:
        cbt = np.asarray(cbt, np.int64)
        cap = cbt.shape[0] // 2
        assert int(cbt[1]) == len(slots)
        live = np.nonzero(cbt[cap:])[0].tolist()
        assert live == slots
        for k in range(1, cap):
            assert cbt[k] == cbt[2 * k] + cbt[2 * k + 1]
    if pos is not None and root_table is not None:
        area = np.zeros(H)
        for j in heap:
            d = depth_of(j, ch)
            area[root_of(j, ch)] += 0.5 ** d
        rt = np.asarray(root_table)
        root_area = 0.5 * np.linalg.norm(np.cross(rt[:, 1] - rt[:, 0], rt[:, 2] - rt[:, 0]), axis=1)
        assert np.allclose(area * root_area, root_area, rtol=1e-12)
    return True


def state_from_oracle(o):
    slots, heap, links = o.leaves()
    return slots, heap, links

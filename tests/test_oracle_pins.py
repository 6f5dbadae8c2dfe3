"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows. None of them compares the oracle
with itself: they use values printed in the paper, closed forms, exact
rational geometry and brute force.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import (Oracle, cbt_compact, cbt_one_to_bit, cbt_sum_reduction, cbt_zero_to_bit, decode_weights, fbm,
                    halfedges_from_faces, lod_test, lowbias32, splitmix64)
from workloads.cameras import (MODE_FORCE_MERGE, MODE_FORCE_SPLIT, MODE_LIST, MODE_RANDOM,
                               forced_params)
from tests.invariants import check_state, depth_of, symbolic_vertices

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- Fig. 1

def test_fig1_halfedge_table():
    """Sec. 2.1, Fig. 1: ingest of the three faces gives the printed table."""
    g = gold("fig1_halfedges.json")
    he = halfedges_from_faces(W.meshes.fig1_mesh())
    for k in ("twin", "next", "prev", "vert", "face"):
        assert he[k].tolist() == g[k], k


def test_root_bisector_example():
    """Sec. 2.2: b7's neighbours are b8 / b11 / b1 and its v2 is the average
    of Vert(h7..h11); v0 = Vert(h7), v1 = Vert(Next(h7))."""
    g = gold("worked_examples.json")
    m = W.meshes.fig1_mesh()
    o = Oracle(m, D=6, max_depth=4)
    slots, heap, links = o.leaves()
    assert slots.tolist() == list(range(12))
    assert links[7].tolist() == [g["root_neighbours_b7"]["twin"], g["root_neighbours_b7"]["next"],
                                 g["root_neighbours_b7"]["prev"]]
    rt = o.root_table()
    verts = [int(v) for v in np.asarray(o.halfedges["vert"])[g["pentagon_halfedges"]]]
    s = [0.0, 0.0, 0.0]
    for v in verts:  # Alg. 1 order: Vert(h7), Vert(h8), ..., Vert(h11)
        s = [s[c] + m.pos[v][c] for c in range(3)]
    assert rt[7, 2].tolist() == [x / 5 for x in s]
    assert rt[7, 0].tolist() == m.pos[1].tolist() and rt[7, 1].tolist() == m.pos[2].tolist()


# ---------------------------------------------------------------- CBT

def _cbt_from_bits(D, bits):
    cbt = np.zeros(2 << D, np.uint32)
    cbt[1 << D:] = bits
    return cbt_sum_reduction(D, cbt)


def test_cbt_figure_sums_and_search():
    """Sec. 3.1 CBT figure (D = 4): the printed sum-reduction tree, and Alg. 7
    returning 0, 3, 10 for the first three set bits (Sec. 3.2)."""
    g = gold("cbt_figure.json")
    D = g["D"]
    cbt = _cbt_from_bits(D, g["bitfield"])
    k = 1
    for level in g["levels_root_first"]:
        assert cbt[k:k + len(level)].tolist() == level
        k += len(level)
    ones = [cbt_one_to_bit(D, cbt, i) for i in range(int(cbt[1]))]
    assert ones[:3] == g["one_to_bit_first_three"]
    assert ones == [i for i, b in enumerate(g["bitfield"]) if b]
    zeros = [cbt_zero_to_bit(D, cbt, i) for i in range((1 << D) - int(cbt[1]))]
    assert zeros == [i for i, b in enumerate(g["bitfield"]) if not b]


@pytest.mark.parametrize("D", [1, 2, 5, 9, 12])
def test_cbt_search_brute_force(D):
    """Alg. 7/8 against a plain scan of random bitfields."""
    rng = np.random.default_rng(D)
    for p in (0.05, 0.5, 0.95):
        bits = (rng.random(1 << D) < p).astype(np.uint32)
        cbt = _cbt_from_bits(D, bits)
        ones = np.nonzero(bits)[0]
        zeros = np.nonzero(bits == 0)[0]
        assert int(cbt[1]) == ones.size
        for i in rng.choice(max(1, ones.size), size=min(50, ones.size), replace=False) if ones.size else []:
            assert cbt_one_to_bit(D, cbt, int(i)) == ones[i]
        for i in rng.choice(max(1, zeros.size), size=min(50, zeros.size), replace=False) if zeros.size else []:
            assert cbt_zero_to_bit(D, cbt, int(i)) == zeros[i]
        assert np.array_equal(cbt_compact(D, cbt), ones)


def test_memory_formula_d17():
    """Sec. 4 'Memory Consumption' with Table 2: D = 17, a pool of 2^D x 9
    ints, a CBT of 2^(D+1) ints and a pointer buffer of 2^D x 2 ints come to
    6.5 MiB; the paper rounds the total (with the input buffers) to 7 MiB."""
    D = 17
    total = (1 << D) * 9 * 4 + (1 << (D + 1)) * 4 + (1 << D) * 2 * 4 + 4
    assert total == 6815748
    assert round(total / 2**20) == 7


# --------------------------------------------------------- Eq. 1, Alg. 2

def test_decode_matches_per_level_bisection():
    """Alg. 2's matrix product (bits read from the low end) against the
    top-down per-level rule of Eq. 1, in exact rationals."""
    he = halfedges_from_faces(W.meshes.fig1_mesh())
    ch = 4
    rng = np.random.default_rng(0)
    for _ in range(200):
        h = int(rng.integers(12))
        d = int(rng.integers(0, 20))
        path = int(rng.integers(0, 1 << d)) if d else 0
        j = ((16 + h) << d) + path
        Wm = decode_weights(j, ch)
        assert (Wm.sum(axis=1) == 1 << d).all()  # barycentric rows
        sym = symbolic_vertices(j, ch, he)
        names = [("v", int(he["vert"][h])), ("v", int(he["vert"][he["next"][h]])), ("c", int(he["face"][h]))]
        for r in range(3):
            want = {}
            for k in range(3):
                if Wm[r, k]:
                    want[names[k]] = want.get(names[k], 0) + Fraction(int(Wm[r, k]), 1 << d)
            assert tuple(sorted(want.items())) == sym[r]


def test_decode_eq1_first_level():
    """Eq. 1 printed: 2 M0 and 2 M1 for the two children of a root."""
    assert decode_weights(2 * 16, 4).tolist() == [[2, 0, 0], [0, 0, 2], [1, 1, 0]]
    assert decode_weights(2 * 16 + 1, 4).tolist() == [[0, 0, 2], [0, 2, 0], [1, 1, 0]]


def test_decode_deep_exact():
    """Depth 60 with a known path: all-zero path keeps v0 as vertex 0 and
    alternating halvings give exact dyadic weights."""
    ch = 2
    j = 4 << 60
    Wm = decode_weights(j, ch)
    assert int(Wm[0, 0]) == 1 << 60 and int(Wm[0, 1]) == 0 and int(Wm[0, 2]) == 0
    assert (Wm.astype(object).sum(axis=1) == 1 << 60).all()


def test_root_corners_follow_the_path_bits():
    """Brute force over every path to depth 10: a corner's row has a single
    nonzero weight (the corner is a root corner) exactly when Eq. 1 carried
    it down unchanged: corner 0 when the bits below the first are all 0,
    corner 1 when they are all 1 (the first bit picking root corner 0 / 2,
    or 1 / 2), corner 2 only at depth 0."""
    ch = 2
    for d in range(0, 11):
        for path in range(1 << d):
            j = (4 << d) + path
            Wm = decode_weights(j, ch).astype(np.int64)
            for v in range(3):
                nz = np.flatnonzero(Wm[v])
                if d == 0:
                    want = v
                elif v == 2:
                    want = None
                else:
                    low = path & ((1 << (d - 1)) - 1)
                    first = (path >> (d - 1)) & 1
                    if v == 0:
                        want = (2 if first else 0) if low == 0 else None
                    else:
                        want = (1 if first else 2) if low == (1 << (d - 1)) - 1 else None
                if want is None:
                    assert nz.size >= 2, (d, path, v)
                else:
                    assert nz.tolist() == [want], (d, path, v)


def test_split_turns_the_vertex_order_over():
    """Each split halves the area and reverses the vertex order: the weight
    matrix of a depth-d bisector has determinant (-1)^d 4^d."""
    rng = np.random.default_rng(3)
    ch = 2
    for d in list(range(0, 8)) + [int(x) for x in rng.integers(8, 21, 30)]:
        path = int(rng.integers(0, 1 << d)) if d else 0
        m = [[int(x) for x in row] for row in decode_weights((4 << d) + path, ch)]
        det = (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
               + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))
        assert det == (-1) ** d * 4 ** d, (d, path, det)


@pytest.mark.parametrize("mesh_name", ["cube", "grid"])
def test_edge_kinds_give_the_depth_parity(mesh_name):
    """In the conforming bisection a refinement edge (Twin) at depth d is
    shared with a refinement edge at depth d or a Next / Prev edge at depth
    d - 1: across every link of a randomly refined state the two depths
    differ by at most one, and their parities agree exactly when both edges
    are refinement edges or both are not."""
    m = W.meshes.cube_mesh() if mesh_name == "cube" else W.meshes.grid_mesh(5, 4, tri_frac=0.3, seed=8)
    o = Oracle(m, 14, 13)
    _random_refine(o, 6, 11)
    slots, heap, links = o.leaves()
    row = {int(s): i for i, s in enumerate(slots)}
    depth = [int(j).bit_length() - 1 - o.ch for j in heap]
    seen = 0
    for i, s in enumerate(slots):
        for x in range(3):
            u = int(links[i, x])
            if u == 0xFFFFFFFF:
                continue
            k = row[u]
            back = [e for e in range(3) if int(links[k, e]) == int(s)]
            assert len(back) == 1
            e = back[0]
            assert abs(depth[i] - depth[k]) <= 1
            assert ((depth[i] - depth[k]) % 2 == 0) == ((x == 0) == (e == 0))
            seen += 1
    assert seen > 250


# ------------------------------------------------------- hash and LOD

def test_splitmix64_published_vector():
    """SplitMix64 (Steele, Lea & Flood 2014) from state 0: its first three
    outputs are the published values."""
    g = 0x9E3779B97F4A7C15
    outs = [splitmix64((k * g) & 0xFFFFFFFFFFFFFFFF) for k in range(3)]
    assert outs == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_lod_special_cases():
    """The LOD reading (split when the projected refinement edge exceeds the
    threshold, cull when all vertices are behind one plane)."""
    planes = np.array([[0, 0, 1]], np.float32)  # keep z >= 0
    tri = np.array([[-1, 0, 10], [1, 0, 10], [0, 1, 10]], np.float32)
    # |e| = 2 at distance 10: big iff 4 q > 100
    assert lod_test(tri, planes, 1, 26.0) == 3
    assert lod_test(tri, planes, 1, 24.0) == 1
    behind = tri * np.array([1, 1, -1], np.float32)
    assert lod_test(behind, planes, 1, 26.0) & 1 == 0
    straddle = tri.copy()
    straddle[2, 2] = -5.0
    assert lod_test(straddle, planes, 1, 26.0) & 1 == 1
    assert lod_test(behind, planes, 0, 26.0) & 1 == 1  # no planes: visible


# -------------------------------------------------- worked examples

def _heap(jp, d, ch):
    return jp + (1 << (ch + d))


def _leafset(o):
    _, heap, _ = o.leaves()
    return sorted(int(j) for j in heap)


def _list_frame(split=(), merge=()):
    return forced_params(MODE_LIST, split_list=np.array(split, np.uint64),
                         merge_list=np.array(merge, np.uint64))


def test_compatibility_chain_and_decimation_examples():
    """Fig. 3 / Sec. 2.3 / Sec. 3.3: with b7 split (paired with b1), refining
    b14 splits b11 into b22, b46, b47; merging the quad b28, b29, b46, b47
    gives back b14, b23; then b22, b23 merge into b11 and the quad b14, b15,
    b2, b3 into b7, b1."""
    g = gold("worked_examples.json")
    m = W.meshes.fig1_mesh()
    o = Oracle(m, D=8, max_depth=6)
    ch = o.ch
    he = o.halfedges

    def want(key):
        return sorted(_heap(jp, d, ch) for jp, d in g[key])

    o.update(_list_frame(split=[_heap(7, 0, ch)]))
    assert _leafset(o) == want("after_split_b7")
    b14 = _heap(14, 1, ch)
    assert [2 * b14, 2 * b14 + 1] == [_heap(jp, d, ch) for jp, d in g["children_of_b14"]]
    slot = {int(j): int(s) for s, j in zip(*o.leaves()[:2])}
    assert o.chain_cost(slot[b14]) == 2 + 3  # b14 itself, b11 one level up, border end
    st = o.update(_list_frame(split=[b14]))
    assert st["split_bisectors"] == 2 and st["allocated"] == 5
    assert _leafset(o) == want("after_split_b14")
    for key in ("after_first_merge", "after_second_merge"):
        st = o.update(forced_params(MODE_FORCE_MERGE))
        assert st["ab_mismatch"] == 0
        assert _leafset(o) == want(key)
        slots, heap, links = o.leaves()
        check_state(slots, heap, links, he, ch, 6, cbt=o.export()["cbt"])


def test_uniform_refinement_closed_form():
    """Uniform refinement to depth d gives H 2^d leaves, every heap ID
    (2^ceil(log2 H) + h) 2^d + p, p < 2^d; forced merging returns the roots."""
    m = W.meshes.cube_mesh()
    o = Oracle(m, D=16, max_depth=14)
    for d in range(1, 11):
        st = o.update(forced_params(MODE_FORCE_SPLIT))
        assert st["ab_mismatch"] == 0
        leaves = _leafset(o)
        assert len(leaves) == 24 * 2**d
        assert leaves == sorted(((32 + h) << d) + p for h in range(24) for p in range(1 << d))
    for d in range(9, -1, -1):
        o.update(forced_params(MODE_FORCE_MERGE))
        assert o.live_count == 24 * 2**d
    assert _leafset(o) == [32 + h for h in range(24)]
    # the merged roots are linked as the halfedges were (slots may differ)
    slots, heap, links = o.leaves()
    root_of = {int(s): int(j) - 32 for s, j in zip(slots, heap)}
    he = o.halfedges
    for s, j, ln in zip(slots, heap, links):
        h = int(j) - 32
        assert [root_of[int(x)] for x in ln] == [int(he["twin"][h]), int(he["next"][h]), int(he["prev"][h])]


@pytest.mark.parametrize("mesh_name", ["fig1", "grid"])
def test_split_then_merge_restores_the_root_links(mesh_name):
    """Open meshes (border halfedges have no Twin): uniform refinement to
    depth 6 and forced merging back leave the H roots linked exactly as the
    halfedge operators, border links null."""
    m = W.meshes.fig1_mesh() if mesh_name == "fig1" else W.meshes.grid_mesh(3, 2, tri_frac=0.3, seed=1)
    o = Oracle(m, D=14, max_depth=8)
    H, base = m.H, 1 << o.ch
    for _ in range(6):
        o.update(forced_params(MODE_FORCE_SPLIT))
    assert o.live_count == H * 64
    for _ in range(6):
        o.update(forced_params(MODE_FORCE_MERGE))
    slots, heap, links = o.leaves()
    assert sorted(int(j) for j in heap) == [base + h for h in range(H)]
    root_of = {int(s): int(j) - base for s, j in zip(slots, heap)}
    root_of[0xFFFFFFFF] = -1
    he = o.halfedges
    for j, ln in zip(heap, links):
        h = int(j) - base
        assert [root_of[int(x)] for x in ln] == [int(he["twin"][h]), int(he["next"][h]), int(he["prev"][h])]


def test_max_allocation_bound():
    """Sec. 3.3 kernel 4: a split never needs more than 3d + 4 allocations;
    brute force over every live bisector of random states."""
    for mesh in (W.meshes.fig1_mesh(), W.meshes.tetra_mesh(), W.meshes.grid_mesh(2, 2, 0.5, seed=7)):
        o = Oracle(mesh, D=10, max_depth=8)
        worst = 0
        for f in range(60):
            o.update(forced_params(MODE_RANDOM, seed=11))
            slots, heap, _ = o.leaves()
            for s, j in zip(slots, heap):
                c = o.chain_cost(int(s))
                d = depth_of(int(j), o.ch)
                assert c <= 3 * d + 4
                worst = max(worst, c - (3 * d + 4))
        assert worst == 0  # the bound is reached


def test_textbook_order_independence():
    """The union of compatibility chains does not depend on the order in which
    the requests are applied: two request orders give the same state."""
    for mesh in (W.meshes.fig1_mesh(), W.meshes.cube_mesh(), W.meshes.grid_mesh(2, 2, 0.5, seed=7)):
        a = Oracle(mesh, D=10, max_depth=8)
        b = Oracle(mesh, D=10, max_depth=8)
        b.set_order_seed(12345)
        for f in range(40):
            sa = a.update(forced_params(MODE_RANDOM, seed=3))
            sb = b.update(forced_params(MODE_RANDOM, seed=3))
            assert sa == sb
            for x, y in zip(a.leaves(), b.leaves()):
                assert np.array_equal(x, y)


def test_dodecahedron_mesh():
    """The planet base of the paper's scenes (Sec. 4, H = 60): 12 planar
    pentagons, every directed edge twinned once, outward orientation, every
    vertex on the sphere."""
    R = 6.371e6
    m = W.meshes.dodecahedron_mesh(R)
    assert m.F == 12 and list(m.face_sizes) == [5] * 12 and m.H == 60
    assert np.allclose(np.linalg.norm(m.pos, axis=1), R, rtol=1e-15, atol=0)
    edges = set()
    off = 0
    for f in range(m.F):
        idx = list(m.face_verts[off:off + 5])
        off += 5
        P = m.pos[idx]
        c = P.mean(0)
        n = np.cross(P[1] - P[0], P[2] - P[0])
        assert np.dot(n, c) > 0  # outward, counter-clockwise seen from outside
        assert np.abs((P - c) @ (n / np.linalg.norm(n))).max() < 1e-9 * R  # planar
        for k in range(5):
            edges.add((idx[k], idx[(k + 1) % 5]))
    assert len(edges) == 60 and all((b, a) in edges for a, b in edges)


def test_sphere_projection_properties():
    """PREC_SPHERE (R13 reading): after four uniform levels on the
    dodecahedron, every exported vertex plus the eye lies on the sphere to
    FP32 rounding of the camera-relative coordinate, and points the same way
    from the centre as the flat FP64 vertex it comes from (radial move); the
    mesh vertices themselves stay put."""
    R = 6.371e6
    m = W.meshes.dodecahedron_mesh(R)
    o = Oracle(m, 12, 8)
    for _ in range(4):
        o.update(forced_params(MODE_FORCE_SPLIT))
    eye = np.array([0.1 * R, -0.2 * R, 1.05 * R])
    v = o.vertices(eye, 3, 20, R).reshape(-1, 3).astype(np.float64)
    flat = o.vertices_f64().reshape(-1, 3)
    on = v + eye
    ulp = np.spacing(np.abs(v).max(axis=1).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(np.linalg.norm(on, axis=1) - R) <= 2.0 * ulp + 1e-9 * R)
    cross = np.linalg.norm(np.cross(on, flat), axis=1) / (np.linalg.norm(on, axis=1) * np.linalg.norm(flat, axis=1))
    assert cross.max() < 1e-6
    assert np.all(np.einsum("ij,ij->i", on, flat) > 0)
    corner = np.isclose(np.linalg.norm(flat, axis=1), R, rtol=1e-12)
    assert corner.any() and np.allclose(on[corner], flat[corner], rtol=0, atol=2.0 * ulp[corner].max())


# ------------------------------------------------- displacement (R14 reading)

def _xorshift_inverse(y, k):
    x = y
    for _ in range(32 // k + 1):
        x = y ^ (x >> k)
    return x


def test_lowbias32_is_a_bijection_of_its_published_steps():
    """lowbias32 (Wellons 2018) is x ^= x >> 16; x *= 0x7feb352d; x ^= x >> 15;
    x *= 0x846ca68b; x ^= x >> 16. Each step is invertible on 32-bit words
    (odd multipliers have modular inverses), so undoing the five steps in
    reverse order must give back every input; a dropped, reordered or
    mistyped step does not invert."""
    M = 1 << 32
    inv1, inv2 = pow(0x7FEB352D, -1, M), pow(0x846CA68B, -1, M)
    rng = np.random.default_rng(14)
    xs = [0, 1, 2, 0xFFFFFFFF, 0x80000000] + [int(v) for v in rng.integers(0, M, 2000, dtype=np.uint64)]
    for x in xs:
        y = lowbias32(x)
        y = _xorshift_inverse(y, 16)
        y = (y * inv2) % M
        y = _xorshift_inverse(y, 15)
        y = (y * inv1) % M
        y = _xorshift_inverse(y, 16)
        assert y == x
    assert lowbias32(0) == 0  # every step fixes 0


def test_value_noise_cell_is_a_smoothstep_bilinear_blend():
    """One octave of the 2-D value noise inside a cell is the bilinear blend
    of its four corner values with the smoothstep weight 3t^2 - 2t^3 per
    axis, the corner values being the noise at the integer points
    themselves (closed form in FP64, against the oracle's FP32)."""
    rng = np.random.default_rng(15)
    for _ in range(200):
        i, j = (int(v) for v in rng.integers(-50, 50, 2))
        tx, ty = (float(np.float32(v)) for v in rng.uniform(0, 1, 2))
        c00 = fbm([i, j], 1.0, 1, 7)
        c10 = fbm([i + 1, j], 1.0, 1, 7)
        c01 = fbm([i, j + 1], 1.0, 1, 7)
        c11 = fbm([i + 1, j + 1], 1.0, 1, 7)
        x = np.float32(i + tx)
        y = np.float32(j + ty)
        ux, uy = (3 * t * t - 2 * t ** 3 for t in (float(x) - i, float(y) - j))
        want = (1 - ux) * (1 - uy) * c00 + ux * (1 - uy) * c10 + (1 - ux) * uy * c01 + ux * uy * c11
        assert abs(fbm([x, y], 1.0, 1, 7) - want) <= 4e-6
        assert -1.0 <= c00 < 1.0


def test_value_noise_is_continuous_with_flat_lattice_points():
    """The smoothstep blend is C1: crossing a cell face changes the 3-D noise
    only by O(step), and at a lattice point the slope vanishes, so a step
    of 2^-12 away changes it by O(2^-24)."""
    rng = np.random.default_rng(16)
    for _ in range(100):
        p = rng.integers(-20, 20, 3).astype(np.float64)
        k = int(rng.integers(0, 3))
        at = fbm(p, 1.0, 1, 3)
        for s in (-1, 1):
            q = p.copy()
            q[k] += s * 2.0 ** -12
            assert abs(fbm(q, 1.0, 1, 3) - at) <= 2.0 ** -18
        r = p.copy()
        r[(k + 1) % 3] += 0.37
        lo, hi = r.copy(), r.copy()
        lo[k] -= 2.0 ** -16
        hi[k] += 2.0 ** -16
        assert abs(fbm(hi, 1.0, 1, 3) - fbm(lo, 1.0, 1, 3)) <= 2.0 ** -12


def test_fbm_is_the_weighted_sum_of_its_octaves():
    """Octave o of the fractal sum is one octave at frequency f 2^o, weight
    2^-o, lattice seeded with seed ^ o: the K-octave value equals that sum
    of single-octave values (to FP32 rounding of the sum)."""
    rng = np.random.default_rng(17)
    for _ in range(100):
        x = rng.uniform(-3, 3, 3).astype(np.float32)
        f = float(np.float32(rng.uniform(0.5, 4)))
        seed = int(rng.integers(0, 1 << 32))
        want = sum(2.0 ** -o * fbm(x, f * 2 ** o, 1, seed ^ o) for o in range(5))
        assert abs(fbm(x, f, 5, seed) - want) <= 1e-5
        assert abs(fbm(x, f, 5, seed)) <= 2.0 - 2.0 ** -4


def test_value_noise_statistics():
    """Lattice values are uniform on [-1, 1): mean 0 and variance 1/3 over
    many integer points."""
    rng = np.random.default_rng(18)
    v = np.array([fbm(p, 1.0, 1, 11) for p in rng.integers(-10 ** 6, 10 ** 6, (4000, 2)).astype(np.float32)])
    assert abs(v.mean()) < 0.04 and abs(v.var() - 1.0 / 3.0) < 0.03


def _disp_frame(eye, precision, radius=0.0, amp=0.05, freq=4.0, octaves=4, seed=9):
    fp = forced_params(MODE_FORCE_SPLIT)
    fp.eye = np.asarray(eye, np.float64)
    fp.precision = precision
    fp.sphere_radius = radius
    fp.disp_amplitude, fp.disp_frequency, fp.disp_octaves, fp.disp_seed = amp, freq, octaves, seed
    return fp


def test_displacement_plain_moves_z_only_and_ignores_the_camera():
    """FP32 form: the displaced vertices differ from the plain ones in z
    only; the world height (z + eye) is a function of the world position,
    so two cameras agree on it to FP32 rounding; amplitude 0 is the
    undisplaced form bit for bit."""
    m = W.meshes.grid_mesh(6, 6, tri_frac=0.2, seed=3, height_sigma=0.05)
    o = Oracle(m, 14, 12)
    for _ in range(3):
        o.update(forced_params(MODE_FORCE_SPLIT))
    eyes = [np.array([0.3, 0.6, 0.4]), np.array([0.9, 0.1, 0.25])]
    plain = [o.vertices(e, 0) for e in eyes]
    disp = [o.vertices(e, 0, frame=_disp_frame(e, 0)) for e in eyes]
    zero = o.vertices(eyes[0], 0, frame=_disp_frame(eyes[0], 0, amp=0.0))
    assert np.array_equal(zero, plain[0])
    for p, d in zip(plain, disp):
        assert np.array_equal(p[..., :2], d[..., :2])
        assert np.abs(d[..., 2] - p[..., 2]).max() > 1e-3
        assert np.abs(d[..., 2] - p[..., 2]).max() <= 0.05 * (2 - 2 ** -3) + 1e-6
    # the height added is +amplitude * fbm(world x, y), read back through fbm
    e32 = eyes[0].astype(np.float32)
    pts = plain[0].reshape(-1, 3)
    hgt = np.array([0.05 * fbm([x + e32[0], y + e32[1]], 4.0, 4, 9) for x, y, _ in pts])
    dz = (disp[0].reshape(-1, 3)[:, 2].astype(np.float64) - pts[:, 2])
    assert np.abs(dz - hgt).max() <= 1e-6
    w0 = disp[0].astype(np.float64) + eyes[0]
    w1 = disp[1].astype(np.float64) + eyes[1]
    # the noise reads world x, y rounded through FP32: positions agree to a few
    # ulps, and the noise's slope (<= 0.05 * 1.5 * 4 * 2^4 per unit) maps them
    assert np.abs(w0 - w1).max() <= 1e-5


def test_displacement_sphere_is_radial():
    """Sphere form: each displaced vertex plus the eye lies on the ray of
    its flat FP64 vertex, at distance R + amplitude * fbm(u) from the
    centre, u the unit direction (the noise read back through the oracle's
    own fbm at u, in FP64 to FP32 rounding of the coordinates)."""
    R = 6.371e6
    m = W.meshes.dodecahedron_mesh(R)
    o = Oracle(m, 12, 8)
    for _ in range(3):
        o.update(forced_params(MODE_FORCE_SPLIT))
    eye = np.array([0.2 * R, 0.1 * R, 1.1 * R])
    fp = _disp_frame(eye, 3, R, amp=2.0e4, freq=8.0, octaves=3, seed=5)
    v = o.vertices(eye, 3, 20, R, frame=fp).reshape(-1, 3).astype(np.float64) + eye
    flat = o.vertices_f64().reshape(-1, 3)
    u = flat / np.linalg.norm(flat, axis=1, keepdims=True)
    hgt = np.array([2.0e4 * fbm(x.astype(np.float32), 8.0, 3, 5) for x in u])
    ulp = np.spacing(np.float32(2 * R)).astype(np.float64)
    assert np.abs(np.linalg.norm(v, axis=1) - (R + hgt)).max() <= 4 * ulp + 2.0e4 * 2 * 8 * 8 * 1e-7
    cross = np.linalg.norm(np.cross(v, flat), axis=1) / (np.linalg.norm(v, axis=1) * np.linalg.norm(flat, axis=1))
    assert cross.max() < 1e-6
    assert np.abs(hgt).max() > 1e3


# ------------------------------------------------ indexed export (R15 reading)

def _random_refine(o, frames, seed):
    from workloads.cameras import forced_params as fp_
    for k in range(frames):
        o.update(fp_(MODE_RANDOM, seed=seed + k))


@pytest.mark.parametrize("mesh_name", ["cube", "dodeca"])
def test_indexed_export_euler_closed(mesh_name):
    """A closed surface (sphere topology) keeps Euler characteristic 2 under
    conforming bisection: with F triangles and E = 3F/2 edges the indexed
    form must have exactly V = 2 + F/2 vertices (a missed merge of two
    corners, or a wrong one, changes V); each triangle has three distinct
    vertices; vertices are numbered in order of first appearance."""
    m = W.meshes.cube_mesh() if mesh_name == "cube" else W.meshes.dodecahedron_mesh(1.0)
    o = Oracle(m, 13, 12)
    for k in range(6):
        _random_refine(o, 2, 40 + 3 * k)
        _, idx, ids = o.export_indexed()
        F = idx.shape[0]
        assert idx.max() + 1 == 2 + F // 2
        assert np.all((idx[:, 0] != idx[:, 1]) & (idx[:, 1] != idx[:, 2]) & (idx[:, 0] != idx[:, 2]))
        flat = idx.reshape(-1).astype(np.int64)
        assert np.all(np.diff(np.maximum.accumulate(flat)) <= 1) and flat[0] == 0
        assert np.array_equal(ids, o.leaves()[1])


def test_indexed_export_euler_open_and_geometry():
    """An open grid (disk topology): V - E + F = 1 with E = (3F + B) / 2, B
    the border edges (null links of the leaves). And geometry decides
    identity: corners given one index have the same FP64 position, and
    different indices are different points."""
    m = W.meshes.grid_mesh(5, 4, tri_frac=0.3, seed=8, height_sigma=0.05)
    o = Oracle(m, 14, 14)
    for k in range(5):
        _random_refine(o, 2, 70 + 5 * k)
        _, idx, _ = o.export_indexed()
        F = idx.shape[0]
        B = int((o.leaves()[2] == 0xFFFFFFFF).sum())
        assert (3 * F + B) % 2 == 0
        E = (3 * F + B) // 2
        V = int(idx.max()) + 1
        assert V - E + F == 1
    pos = o.vertices_f64().reshape(-1, 3)
    flat = idx.reshape(-1)
    first = np.zeros((V, 3))
    first[flat[::-1]] = pos[::-1]  # the first occurrence's position per index
    assert np.abs(pos - first[flat]).max() <= 1e-12
    q = np.round(first * 2 ** 30).astype(np.int64)
    assert np.unique(q, axis=0).shape[0] == V


def test_indexed_export_pinched_vertex():
    """Two triangles that meet only at a vertex (a bowtie: no edge shared):
    the shared mesh vertex stays one index however far either side is
    refined, so V - E + F stays 1 (E = (3F + B) / 2, every root edge a
    border), and that index's corners lie on both triangles' sides."""
    m = W.meshes._mesh("bowtie", [[0, 1, 2], [0, 3, 4]],
                       [(0, 0, 0), (1, 0, 0), (1, 1, 0), (-1, 0, 0), (-1, -1, 0)])
    o = Oracle(m, 12, 10)
    for k in range(4):
        _random_refine(o, 2, 90 + 3 * k)
        _, idx, _ = o.export_indexed()
        F = idx.shape[0]
        B = int((o.leaves()[2] == 0xFFFFFFFF).sum())
        V = int(idx.max()) + 1
        assert V - (3 * F + B) // 2 + F == 1
    pos = o.vertices_f64().reshape(-1, 3)
    flat = idx.reshape(-1)
    at0 = np.flatnonzero(np.abs(pos).max(axis=1) == 0.0)
    assert at0.size >= 2 and np.unique(flat[at0]).size == 1
    side = np.sign(o.vertices_f64().sum(axis=1)[at0 // 3, 0])
    assert (side > 0).any() and (side < 0).any()


@pytest.mark.parametrize("form", ["plain", "sphere"])
def test_zero_amplitude_displacement_is_the_plain_update(form):
    """R14 reduces to the undisplaced update when the amplitude is zero (the
    other displacement parameters set): the frames give the same leaves and
    links as the plain configuration, for the FP32 and the sphere forms."""
    if form == "plain":
        a = W.configs.config_terrain(n_frames=12, nx=10, D=14, amp=0.0)
        b = W.configs.config2(n_frames=12, nx=10)
        D, frames_a, frames_b = 14, a.frames, b.frames
    else:
        a = W.configs.config_waves(n_frames=300, D=13, amp=0.0)
        b = W.configs.config_dodeca(n_frames=300, D=13)
        D, frames_a, frames_b = 13, a.frames[60:300:12], b.frames[60:300:12]
    assert frames_a[0].disp_octaves > 0 and frames_a[0].disp_amplitude == 0.0
    oa, ob = Oracle(a.mesh, D, a.max_depth), Oracle(b.mesh, D, b.max_depth)
    for fa, fb in zip(frames_a, frames_b):
        oa.update(fa)
        ob.update(fb)
    for x, y in zip(oa.leaves(), ob.leaves()):
        assert np.array_equal(x, y)
    assert oa.live_count > len(a.mesh.face_sizes)

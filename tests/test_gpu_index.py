"""Indexed export (cbt_index, R15 reading): the vertex buffer, index buffer
and triangle heap IDs equal the oracle's indexed form of the same state,
bit for bit (plain grid, displaced terrain, sphere-form planet with depths
beyond 31, closed cube, two triangles sharing only a vertex); at full size
the index buffer obeys the Euler characteristic of the surface and numbers
vertices by first occurrence."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from workloads.cameras import MODE_FORCE_SPLIT, forced_params
from tests.gpu_helpers import run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2407_02215_gb300 as P
    P.build_library()
    return P


def _index_pair(g, o, fp, D):
    import torch
    vbuf = torch.empty((1 << D, 3, 3), dtype=torch.float32, device="cuda")
    g.update(fp, vertices_out=vbuf)
    o.update(fp)
    torch.cuda.synchronize()
    n = o.live_count
    assert g.live_count() == n and g.stats()["error"] == 0
    vg, ig, hg = g.index(vbuf[:n])
    tri = o.vertices(fp.eye, fp.precision, fp.fixed_shift, fp.sphere_radius, frame=fp)
    vo, io, ho = o.export_indexed(tri)
    assert np.array_equal(ig.cpu().numpy().view(np.uint32), io)
    assert np.array_equal(hg.cpu().numpy().view(np.uint64), ho)
    assert np.array_equal(vg.cpu().numpy().view(np.uint32), vo.view(np.uint32))
    return vo, io


@pytest.mark.parametrize("terrain", [False, True], ids=["grid", "terrain"])
def test_grid_flythrough_indexed(P, terrain):
    spec = (W.configs.config_terrain(n_frames=31, nx=24, D=16) if terrain
            else W.configs.config2(n_frames=31, nx=24))
    g, o = run_pair(spec.mesh, 16, spec.max_depth, spec.frames[:-1], P.CBT, Oracle, check_every=10)
    v, idx = _index_pair(g, o, spec.frames[-1], 16)
    assert v.shape[0] == idx.max() + 1


def test_planet_indexed_deep(P):
    """Sphere form on the dodecahedron planet under a camera that descends
    looking straight down with a 2 degree view, so that refinement goes
    deeper than 31 levels (64-bit weights in the oracle's identities, path
    bits past 32 in the root-corner test)."""
    from workloads.cameras import PREC_SPHERE, frame_params, sphere_descent_path
    R = 6.371e6
    mesh = W.meshes.dodecahedron_mesh(R)
    cams = sphere_descent_path(mesh, R, 60, seed=5, alt_lo=1.0)
    for c in cams:
        c.target = c.eye / np.linalg.norm(c.eye) * R
        c.fovy_rad = np.radians(2.0)
        c.aspect = 1.0
    frames = [frame_params(c, 14.0, precision=PREC_SPHERE, sphere_radius=R) for c in cams]
    g, o = run_pair(mesh, 15, 50, frames[:-1], P.CBT, Oracle, check_every=20)
    _, heap, _ = o.leaves()
    depth = np.array([int(j).bit_length() - 1 - o.ch for j in heap])
    assert depth.max() > 31
    _index_pair(g, o, frames[-1], 15)


def test_closed_cube_indexed(P):
    """Uniform refinement of the cube: 24 2^d triangles and 2 + 12 2^d
    vertices (Euler characteristic 2), equal to the oracle's."""
    m = W.meshes.cube_mesh()
    g, o = run_pair(m, 16, 14, [forced_params(MODE_FORCE_SPLIT)] * 9, P.CBT, Oracle, check_every=9)
    fp = forced_params(MODE_FORCE_SPLIT)
    fp.eye = np.array([2.0, 1.0, 0.5])
    v, idx = _index_pair(g, o, fp, 16)
    assert idx.shape[0] == 24 * 2 ** 10 and v.shape[0] == 2 + 12 * 2 ** 10


def test_pinched_vertex_indexed(P):
    """Two triangles meeting only at a vertex (no shared edge): the corners
    at that vertex are matched by their global point although no neighbour
    link joins the two sides; the indexed form equals the oracle's after
    random refinement of both sides."""
    from workloads.cameras import MODE_RANDOM
    m = W.meshes._mesh("bowtie", [[0, 1, 2], [0, 3, 4]],
                       [(0, 0, 0), (1, 0, 0), (1, 1, 0), (-1, 0, 0), (-1, -1, 0)])
    frames = [forced_params(MODE_RANDOM, seed=90 + k) for k in range(8)]
    g, o = run_pair(m, 12, 10, frames[:-1], P.CBT, Oracle, check_every=7)
    fp = frames[-1]
    fp.eye = np.array([0.3, -0.2, 1.0])
    v, idx = _index_pair(g, o, fp, 12)
    assert v.shape[0] == idx.max() + 1


def test_full_size_grid_index_properties(P):
    """The 100 x 100 grid flythrough on a 2^20 pool at its lowest point:
    V - E + F = 1 (a disk) with E = (3F + B) / 2 and B the border edges; each
    triangle's corners distinct; vertices numbered by first occurrence; each
    vertex's position is one of its occurrences' exported vertices."""
    import torch
    spec = W.configs.config2()
    g = P.CBT(spec.mesh, spec.D, spec.max_depth)
    vbuf = torch.empty((1 << spec.D, 3, 3), dtype=torch.float32, device="cuda")
    for fp in spec.frames[:60]:
        g.update(fp)
    g.update(spec.frames[60], vertices_out=vbuf)
    n = g.live_count()
    v, idx, heap = g.index(vbuf[:n])
    idx = idx.cpu().numpy().astype(np.int64)
    F = idx.shape[0]
    links = g.leaves()[2].cpu().numpy().view(np.uint32)
    B = int((links == 0xFFFFFFFF).sum())
    V = int(idx.max()) + 1
    assert v.shape[0] == V and F == n > 100000
    assert V - (3 * F + B) // 2 + F == 1
    assert np.all((idx[:, 0] != idx[:, 1]) & (idx[:, 1] != idx[:, 2]) & (idx[:, 0] != idx[:, 2]))
    flat = idx.reshape(-1)
    assert flat[0] == 0 and np.all(np.diff(np.maximum.accumulate(flat)) <= 1)
    tri = vbuf[:n].cpu().numpy().reshape(-1, 3)
    first = np.full(V, -1, np.int64)
    first[flat[::-1]] = np.arange(flat.size)[::-1]
    assert np.array_equal(v.cpu().numpy(), tri[first])


def test_index_errors(P):
    import ctypes
    import torch
    spec = W.configs.config1(n_frames=2)
    g = P.CBT(spec.mesh, 14, 14)
    lib = P.load()
    ws = g.index_workspace(64)
    idx = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    nv, nt = ctypes.c_uint32(), ctypes.c_uint32()
    p = ctypes.c_void_p
    # vertices without the per-bisector vertices
    assert lib.cbt_index(g._h, None, p(ws.data_ptr()), ws.numel(), p(idx.data_ptr()), 4, p(idx.data_ptr()), 4,
                         None, ctypes.byref(nv), ctypes.byref(nt), None) == 1
    # 24 live triangles into room for 4
    assert lib.cbt_index(g._h, None, p(ws.data_ptr()), ws.numel(), None, 0, p(idx.data_ptr()), 4, None,
                         ctypes.byref(nv), ctypes.byref(nt), None) == 4
    assert nt.value == 24
    # a workspace off its 256-byte alignment
    assert lib.cbt_index(g._h, None, p(ws.data_ptr() + 8), ws.numel() - 8, None, 0, p(idx.data_ptr()), 4, None,
                         ctypes.byref(nv), ctypes.byref(nt), None) == 1
    # a workspace sized for fewer live bisectors
    small = g.index_workspace(2)
    big = torch.empty((24, 3), dtype=torch.int32, device="cuda")
    assert lib.cbt_index(g._h, None, p(small.data_ptr()), small.numel(), None, 0, p(big.data_ptr()), 24, None,
                         ctypes.byref(nv), ctypes.byref(nt), None) == 4

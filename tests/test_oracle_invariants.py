"""The oracle's states satisfy the invariants the method guarantees: a
conforming triangulation with mutual, edge-matched links; leaves that
partition the roots; a CBT whose root is the live count (Sec. 2.3, Sec. 3)."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from workloads.cameras import MODE_RANDOM, PREC_FIXED, PREC_FP32, PREC_FP64, forced_params
from tests.invariants import check_state, depth_of

TINY = [
    ("fig1", lambda: W.meshes.fig1_mesh()),
    ("tetra", lambda: W.meshes.tetra_mesh()),
    ("cube", lambda: W.meshes.cube_mesh()),
    ("grid2", lambda: W.meshes.grid_mesh(2, 2, 0.5, seed=7)),
]


@pytest.mark.parametrize("name,make", TINY)
def test_random_frames_keep_invariants(name, make):
    mesh = make()
    o = Oracle(mesh, D=9, max_depth=7)
    rt = o.root_table()
    for f in range(60):
        st = o.update(forced_params(MODE_RANDOM, seed=17))
        assert st["ab_mismatch"] == 0
        assert st["allocated"] <= st["free_before"]
        slots, heap, links = o.leaves()
        check_state(slots, heap, links, o.halfedges, o.ch, 7, cbt=o.export()["cbt"],
                    pos=mesh.pos, root_table=rt)


def test_pool_exhaustion_is_gated():
    """A tiny pool: the gate keeps allocations within the free bits and the
    state stays valid while requests are denied."""
    mesh = W.meshes.cube_mesh()
    o = Oracle(mesh, D=7, max_depth=10)
    denied = 0
    for f in range(40):
        st = o.update(forced_params(MODE_RANDOM, seed=5))
        assert st["allocated"] <= st["free_before"]
        denied += st["split_wishes"] - st["split_granted"]
        slots, heap, links = o.leaves()
        check_state(slots, heap, links, o.halfedges, o.ch, 10, cbt=o.export()["cbt"])
    assert denied > 0


def test_cube_lod_path_invariants():
    spec = W.configs.config1()
    o = Oracle(spec.mesh, spec.D, spec.max_depth)
    for fp in spec.frames[:7]:
        st = o.update(fp)
        assert st["ab_mismatch"] == 0
    slots, heap, links = o.leaves()
    check_state(slots, heap, links, o.halfedges, o.ch, spec.max_depth, cbt=o.export()["cbt"])


def _gamma(n, u):
    return n * u / (1 - n * u)


def test_vertex_error_bounds():
    """FP32 vertices (R9 reading) against FP64: per coordinate within
    Higham's dot-product bound gamma_3 sum |w||V| (with |V| already rounded to
    FP32) plus the rounding of the root offsets; fixed point (R10 reading)
    within 2^-shift + 1/2 ulp."""
    spec = W.configs.config1()
    o = Oracle(spec.mesh, spec.D, spec.max_depth)
    for fp in spec.frames[:6]:
        o.update(fp)
    eye = spec.frames[5].eye
    exact = o.vertices_f64() - eye[None, None, :]
    v32 = o.vertices(eye, PREC_FP32).astype(np.float64)
    u = 2.0**-24
    mag = np.abs(o.root_table() - eye).max()
    bound = _gamma(3, u) * 3 * mag + 3 * u * mag + u * np.abs(exact)
    assert (np.abs(v32 - exact) <= bound).all()
    vf = o.vertices(eye, PREC_FIXED, 20).astype(np.float64)
    assert (np.abs(vf - exact) <= 2.0**-20 * 2 + u * np.abs(exact) + 1e-12).all()
    v64 = o.vertices(eye, PREC_FP64).astype(np.float64)
    assert (np.abs(v64 - exact) <= u * np.abs(exact) + 1e-12).all()


def test_planet_fixed_point_precision():
    """Planet scale (R = 6.371e6 m): fixed-point vertices stay within a
    micrometre of FP64 next to a camera 2 m above the surface, where FP32
    offsets of the roots would be off by decimetres."""
    spec = W.configs.config3(n_frames=600)
    o = Oracle(spec.mesh, D=12, max_depth=48)
    slots, heap, _ = o.leaves()
    eye = spec.frames[-1].eye
    exact = o.vertices_f64() - eye[None, None, :]
    vf = o.vertices(eye, PREC_FIXED, 20).astype(np.float64)
    err_fixed = np.abs(vf - exact) - 2.0**-24 * np.abs(exact)
    assert err_fixed.max() <= 2.0**-19
    v32 = o.vertices(eye, PREC_FP32).astype(np.float64)
    assert np.abs(v32 - exact).max() > 1e-2

"""Parity of the CUDA library with the CPU oracle, frame by frame: the live
slots, heap IDs, neighbour links, CBT bitfield and every CBT sum must be
identical (integer state, bit-exact), and so must the per-frame counters."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from workloads.cameras import (GATE_PAPER, MODE_FORCE_MERGE, MODE_FORCE_SPLIT, MODE_LIST,
                               MODE_RANDOM, PREC_FIXED, PREC_FP32, PREC_FP64, forced_params)
from tests.gpu_helpers import assert_same_state, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["fused", "per_step"])
def CBT(request):
    """Instances in either execution form: one cooperative launch per frame,
    or one launch per step."""
    import paper_2407_02215_gb300 as P
    P.build_library()
    fused = request.param == "fused"

    def make(*args, **kw):
        g = P.CBT(*args, **kw)
        g.set_fused(fused)
        assert g.fused == fused
        return g
    return make


TINY = [
    ("fig1", W.meshes.fig1_mesh, 8, 6),
    ("tetra", W.meshes.tetra_mesh, 9, 7),
    ("cube", W.meshes.cube_mesh, 10, 8),
    ("grid2", lambda: W.meshes.grid_mesh(2, 2, 0.5, seed=7), 9, 7),
]


@pytest.mark.parametrize("name,make,D,md", TINY)
def test_create(CBT, name, make, D, md):
    m = make()
    g, o = CBT(m, D, md), Oracle(m, D, md)
    assert_same_state(g, o, "create")


@pytest.mark.parametrize("name,make,D,md", TINY)
def test_random_frames(CBT, name, make, D, md):
    frames = [forced_params(MODE_RANDOM, seed=21) for _ in range(50)]
    run_pair(make(), D, md, frames, CBT, Oracle)


def test_small_pools_and_ragged_words(CBT):
    """Pools of 2^3..2^6 slots (less than one or a few bitfield words) under
    random requests: the gate keeps allocations within the free bits."""
    for D in (4, 5, 6, 7):
        frames = [forced_params(MODE_RANDOM, seed=D) for _ in range(40)]
        run_pair(W.meshes.fig1_mesh(), D, 8, frames, CBT, Oracle)


def test_merge_requests_beyond_free_slots(CBT):
    """A saturated pool of 8 tiles asked to merge everything: the merge
    requests need more parents than there are free slots, so the gate grants
    them in slot order only while their running total fits."""
    frames = [forced_params(MODE_FORCE_SPLIT) for _ in range(10)]
    frames += [forced_params(MODE_FORCE_MERGE) for _ in range(6)]
    frames += [forced_params(MODE_RANDOM, seed=31) for _ in range(10)]
    g, o = run_pair(W.meshes.cube_mesh(), 13, 12, frames, CBT, Oracle, check_every=2)


def test_paper_gate(CBT):
    frames = [forced_params(MODE_RANDOM, seed=4, gate=GATE_PAPER) for _ in range(40)]
    run_pair(W.meshes.cube_mesh(), 9, 8, frames, CBT, Oracle)


def test_worked_example_frames(CBT):
    """The paper's compatibility-chain and decimation example (Fig. 3)."""
    m = W.meshes.fig1_mesh()
    ch = 4
    b7 = 16 + 7
    b14 = (16 + 7) * 2
    frames = [forced_params(MODE_LIST, split_list=np.array([b7], np.uint64)),
              forced_params(MODE_LIST, split_list=np.array([b14], np.uint64)),
              forced_params(MODE_FORCE_MERGE), forced_params(MODE_FORCE_MERGE)]
    g, o = run_pair(m, 8, 6, frames, CBT, Oracle)
    assert g.live_count() == 12


def test_uniform_closed_form(CBT):
    spec = W.configs.config1_uniform(10)
    g, o = run_pair(spec.mesh, spec.D, spec.max_depth, spec.frames[:10], CBT, Oracle)
    assert g.live_count() == 24 * 2**10
    _, heap, _ = g.leaves()
    want = sorted(((32 + h) << 10) + p for h in range(24) for p in range(1 << 10))
    assert sorted(heap.cpu().numpy().tolist()) == want
    for fp in spec.frames[10:]:
        g.update(fp)
    assert g.live_count() == 24


def test_cube_lod_path(CBT):
    spec = W.configs.config1()
    run_pair(spec.mesh, spec.D, spec.max_depth, spec.frames, CBT, Oracle)


@pytest.mark.parametrize("prec", [PREC_FP32, PREC_FIXED, PREC_FP64])
def test_grid_lod_precisions(CBT, prec):
    """A 24x24 grid flythrough under each vertex-evaluation form."""
    mesh = W.meshes.grid_mesh(24, 24, 0.1, seed=9)
    cams = W.cameras.flythrough_path(30, seed=9, alt_lo=0.02)
    frames = [W.cameras.frame_params(c, 2.0, precision=prec) for c in cams]
    run_pair(mesh, 17, 22, frames, CBT, Oracle, check_every=5)


@pytest.mark.parametrize("prec", [PREC_FP32, PREC_FIXED, PREC_FP64])
def test_vertices_bit_exact(CBT, prec):
    spec = W.configs.config1()
    g, o = run_pair(spec.mesh, spec.D, spec.max_depth, spec.frames[:8], CBT, Oracle, check_every=8)
    eye = spec.frames[7].eye
    vg = g.vertices(eye, prec, 20).cpu().numpy()
    vo = o.vertices(eye, prec, 20)
    assert vg.shape == vo.shape
    assert np.array_equal(vg.view(np.uint32), vo.view(np.uint32))


def test_single_triangle_all_border(CBT):
    """The smallest mesh: one triangle (3 halfedges, every edge on the
    border, so every chain ends at a null twin), split, merged and randomly
    requested on pools of 2^3 and 2^10."""
    m = W.meshes._mesh("triangle", [[0, 1, 2]], [(0, 0, 0), (1, 0, 0), (0.2, 0.9, 0)])
    frames = ([forced_params(MODE_FORCE_SPLIT)] * 6 + [forced_params(MODE_FORCE_MERGE)] * 7 +
              [forced_params(MODE_RANDOM, seed=5)] * 30)
    for D in (3, 10):
        run_pair(m, D, 12, frames, CBT, Oracle)


def test_deepest_heap_ids(CBT):
    """The longest heap IDs the index width allows (Sec. 3.3: ceil(log2 H) +
    1 + max depth <= 63): the cube (H = 24) with max depth 57, refined under a
    2-degree view descending to 1e-11 above a face in the FP64 form, reaches
    depth 57 (63-bit heap IDs) with the oracle's states every 10 frames, and
    the FP64-form vertices of the deepest bisectors are bit-identical."""
    from workloads.cameras import Camera, frame_params
    target = np.array([0.1037, 0.2981, 0.5])
    frames = []
    for k in range(70):
        alt = np.exp(np.log(2.0) + (np.log(1e-11) - np.log(2.0)) * k / 69)
        cam = Camera(eye=target + np.array([0, 0, alt]), target=target, up=np.array([0.0, 1.0, 0.0]),
                     fovy_rad=np.radians(2.0), aspect=1.0)
        frames.append(frame_params(cam, 14.0, precision=PREC_FP64))
    g, o = run_pair(W.meshes.cube_mesh(), 16, 57, frames, CBT, Oracle, check_every=10)
    heap = o.leaves()[1]
    assert max(int(j).bit_length() for j in heap) == 63
    eye = frames[-1].eye
    vg = g.vertices(eye, PREC_FP64, 20).cpu().numpy()
    vo = o.vertices(eye, PREC_FP64, 20)
    assert np.array_equal(vg.view(np.uint32), vo.view(np.uint32))


@pytest.mark.parametrize("D", [5, 9, 12])
def test_forms_alternating_frame_by_frame(D):
    """One instance whose execution form changes between frames (one launch,
    one launch per step, one launch again ...): each form takes over the
    state the other left, including what the one-launch frame carries from
    one frame to the next (the cleared chain marks and the free list of every
    zero bit), and every frame matches the oracle."""
    import paper_2407_02215_gb300 as P
    P.build_library()
    forms = [True, True, False, True, False, False, True, True, True, False]

    def make(*args, **kw):
        return P.CBT(*args, **kw)
    frames = [forced_params(MODE_RANDOM, seed=40 + D) for _ in range(3 * len(forms))]
    m = W.meshes.cube_mesh()
    g, o = make(m, D, D - 1), Oracle(m, D, D - 1)
    for k, fp in enumerate(frames):
        g.set_fused(forms[k % len(forms)])
        g.update(fp)
        so = o.update(fp)
        sg = g.stats()
        assert sg["error"] == 0, f"frame {k}: device error {sg['error']:#x}"
        assert sg["allocated"] == so["allocated"], f"frame {k}"
        assert_same_state(g, o, f"frame {k} ({'fused' if forms[k % len(forms)] else 'per step'})")


def test_single_instance_above_the_one_launch_tables():
    """A single instance whose pool (2^23 slots) exceeds the single-instance
    frame's tables runs the batch frame (its phase names say so), and every
    frame equals the oracle: forced splits to depth 9, random requests, then
    merges."""
    import paper_2407_02215_gb300 as P
    P.build_library()
    m = W.meshes.cube_mesh()
    D, md = 23, 12
    g, o = P.CBT(m, D, md), Oracle(m, D, md)
    g.set_fused(True)
    g.set_timing(True)
    frames = [forced_params(MODE_FORCE_SPLIT) for _ in range(9)]
    frames += [forced_params(MODE_RANDOM, seed=23) for _ in range(6)]
    frames += [forced_params(MODE_FORCE_MERGE) for _ in range(3)]
    for k, fp in enumerate(frames):
        g.update(fp)
        so = o.update(fp)
        sg = g.stats()
        assert sg["error"] == 0, f"frame {k}: device error {sg['error']:#x}"
        for key in ("live_after", "split_granted", "merge_granted", "allocated"):
            assert sg[key] == so[key], f"frame {k}: {key} gpu {sg[key]} oracle {so[key]}"
        if k % 3 == 2 or k == len(frames) - 1:
            assert_same_state(g, o, f"frame {k}")
    assert "gate_sum" in g.kernel_times()  # a phase of the batch frame

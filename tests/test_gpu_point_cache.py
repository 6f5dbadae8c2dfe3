"""The sphere form's optional per-slot point cache (cbt_attach_point_cache:
classify keeps each bisector's FP64 points and scales, tagged with its heap
ID and a cache generation, and evaluates only the eye-relative rounding while
the tag matches). The cache must never change a result: a new generation is
made whenever the radius or the displacement changes, frames of another form
or mode leave it as it is, and cache memory that held another instance's
points starts with no tag matching. Every case is compared with the oracle
frame by frame; the same frames without a cache take the uncached path."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from workloads.cameras import PREC_FP32, forced_params
from tests.gpu_helpers import assert_same_state, run_pair

FORMS = pytest.mark.parametrize("fused", [True, False], ids=["fused", "per_step"])
EINVAL, ENOMEM = 1, 4  # CBT_EINVAL, CBT_ENOMEM


@pytest.fixture(scope="module")
def P():
    import paper_2407_02215_gb300 as P
    P.build_library()
    return P


def _maker(P, fused, cache=True):
    def make(mesh, D, max_depth):
        g = P.CBT(mesh, D, max_depth, point_cache=cache)
        g.set_fused(fused)
        return g
    return make


def _shape_frames():
    """Every 3rd frame of a displaced planet descent on a 2^15 pool, the
    shape changing every second frame: amplitude off and halved, the radius
    0.1% larger, another seed, frequency and octave count; an FP32-form
    frame and a random-mode frame in between."""
    spec = W.configs.config_waves(D=15, amp=3.0e4, freq=16.0, octaves=4, seed=31)
    base = spec.frames[::3][:64]
    R = base[0].sphere_radius
    shapes = [dict(), dict(disp_amplitude=0.0), dict(sphere_radius=R * 1.001), dict(disp_amplitude=1.5e4),
              dict(disp_seed=32), dict(disp_frequency=8.0), dict(disp_octaves=3)]
    frames = []
    for k, fp in enumerate(base):
        frames.append(dataclasses.replace(fp, **shapes[(k // 2) % len(shapes)]))
        if k == 20:
            frames.append(dataclasses.replace(fp, precision=PREC_FP32, sphere_radius=0.0, disp_amplitude=0.0))
        if k == 40:
            frames.append(forced_params(3, seed=5))
    return spec, frames


def _export_check(g, o, fp, D):
    import torch
    vbuf = torch.empty((1 << D, 3, 3), dtype=torch.float32, device="cuda")
    g.update(fp, vertices_out=vbuf)
    o.update(fp)
    torch.cuda.synchronize()
    n = o.live_count
    assert g.live_count() == n and g.stats()["error"] == 0
    vo = o.vertices(fp.eye, fp.precision, fp.fixed_shift, fp.sphere_radius, frame=fp)
    assert np.array_equal(vbuf[:n].cpu().numpy().view(np.uint32), vo.view(np.uint32))


@pytest.mark.gpu
@pytest.mark.parametrize("cache", [True, False], ids=["cache", "no_cache"])
@FORMS
def test_shape_changes_make_new_generations(P, fused, cache):
    """States equal the oracle's after every frame of the shape-changing
    sequence (a stale cached point would change an LOD decision); then two
    more frames with the exported vertices compared bit for bit, the first
    with a new shape, the second with the same one (cached points)."""
    spec, frames = _shape_frames()
    g, o = run_pair(spec.mesh, 15, spec.max_depth, frames, _maker(P, fused, cache), Oracle, check_every=1)
    last = frames[-1]
    _export_check(g, o, dataclasses.replace(last, disp_amplitude=2.0e4), 15)
    _export_check(g, o, dataclasses.replace(last, disp_amplitude=2.0e4), 15)


def test_the_shape_changes_decide_something():
    """The shape changes of the sequence above matter: the oracle run with
    one fixed shape ends in another state (so a cache that ignored them
    could not pass the test above)."""
    spec, frames = _shape_frames()
    fixed = [dataclasses.replace(f, disp_amplitude=spec.frames[0].disp_amplitude,
                                 sphere_radius=spec.frames[0].sphere_radius,
                                 disp_seed=spec.frames[0].disp_seed, disp_frequency=spec.frames[0].disp_frequency,
                                 disp_octaves=spec.frames[0].disp_octaves)
             if f.precision != PREC_FP32 and f.mode == 0 else f for f in frames]
    a, b = Oracle(spec.mesh, 15, spec.max_depth), Oracle(spec.mesh, 15, spec.max_depth)
    for fa, fb in zip(frames, fixed):
        a.update(fa)
        b.update(fb)
    assert a.live_count != b.live_count or not np.array_equal(a.leaves()[1], b.leaves()[1])


@pytest.mark.gpu
@FORMS
def test_reused_cache_memory_starts_without_tags(P, fused):
    """An instance (in the workspace of another one) attached to the other
    one's point-cache memory, with the same mesh and pool, the same heap IDs
    early in the descent and another radius, equals the oracle: none of the
    old instance's cached points is taken."""
    import torch
    spec = W.configs.config_dodeca(n_frames=300, D=15)
    frames = spec.frames[::10][:20]
    R = frames[0].sphere_radius
    g1 = P.CBT(spec.mesh, 15, spec.max_depth, point_cache=True)
    g1.set_fused(fused)
    for fp in frames:
        g1.update(fp)
    torch.cuda.synchronize()
    ws, pcm = g1.workspace, g1.point_cache
    del g1
    g2 = P.CBT(spec.mesh, 15, spec.max_depth, workspace=ws, point_cache=pcm)
    g2.set_fused(fused)
    o = Oracle(spec.mesh, 15, spec.max_depth)
    for k, fp in enumerate(frames[:-1]):
        fq = dataclasses.replace(fp, sphere_radius=R * 1.002)
        g2.update(fq)
        o.update(fq)
        torch.cuda.synchronize()
        assert g2.stats()["error"] == 0
        assert_same_state(g2, o, f"frame {k}")
    _export_check(g2, o, dataclasses.replace(frames[-1], sphere_radius=R * 1.002), 15)


@pytest.mark.gpu
def test_attach_errors(P):
    """cbt_attach_point_cache refuses memory that is not 16-byte aligned or
    too short, and a second cache; the state still updates afterwards."""
    import ctypes as C
    import torch
    lib = P.load()
    spec = W.configs.config_dodeca(n_frames=300, D=14)
    g = P.CBT(spec.mesh, 14, spec.max_depth)
    need = lib.cbt_point_cache_bytes(14)
    buf = torch.empty(need + 64, dtype=torch.uint8, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.cbt_attach_point_cache(g.handle, C.c_void_p(buf.data_ptr() + 8), need, s) == EINVAL
    assert lib.cbt_attach_point_cache(g.handle, C.c_void_p(buf.data_ptr()), need - 16, s) == ENOMEM
    assert lib.cbt_attach_point_cache(g.handle, None, need, s) == EINVAL
    assert lib.cbt_attach_point_cache(g.handle, C.c_void_p(buf.data_ptr()), need, s) == 0
    assert lib.cbt_attach_point_cache(g.handle, C.c_void_p(buf.data_ptr()), need, s) == EINVAL
    o = Oracle(spec.mesh, 14, spec.max_depth)
    for fp in spec.frames[::30]:
        g.update(fp)
        o.update(fp)
    torch.cuda.synchronize()
    assert g.stats()["error"] == 0
    assert_same_state(g, o, "after the attach calls")


def test_point_cache_bytes():
    """144 bytes per pool slot (16 FP64 values and a 16-byte tag), 0 for a
    pool exponent outside 1..30; a host call, no GPU needed."""
    import paper_2407_02215_gb300 as P
    P.build_library()
    lib = P.load()
    assert lib.cbt_point_cache_bytes(17) == 144 << 17
    assert lib.cbt_point_cache_bytes(1) == 288
    assert lib.cbt_point_cache_bytes(0) == 0 and lib.cbt_point_cache_bytes(31) == 0
    assert lib.cbt_attach_point_cache(None, None, 0, None) == EINVAL  # NULL state: refused before any CUDA call


def test_python_arguments_are_checked_before_any_device_work():
    """The binding refuses a host tensor (or a wrong type) as workspace or
    point-cache memory before it allocates or launches anything."""
    import torch
    import paper_2407_02215_gb300 as P
    P.build_library()
    mesh = W.meshes.cube_mesh()
    with pytest.raises(ValueError, match="point_cache"):
        P.CBT(mesh, 12, 8, point_cache=torch.empty(144 << 12, dtype=torch.uint8))
    for bad in ("yes", 1):
        with pytest.raises(ValueError, match="point_cache"):
            P.CBT(mesh, 12, 8, point_cache=bad)
    with pytest.raises(ValueError, match="workspace"):
        P.CBT(mesh, 12, 8, workspace=torch.empty(1 << 24, dtype=torch.uint8))

"""Displaced surfaces (R14 reading of Sec. 4's wave layers and elevation
data): the LOD test and the vertex export see vertices displaced by seeded
fractal value noise, in the FP32 form (terrain: +z) and the sphere form
(planet: radial). The CUDA path must give the oracle's states frame by
frame and its displaced vertices bit for bit, in the one-launch and the
per-step forms and in a batch."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from workloads.cameras import PREC_FIXED
from tests.gpu_helpers import assert_same_state, run_pair

pytestmark = pytest.mark.gpu
FORMS = pytest.mark.parametrize("fused", [True, False], ids=["fused", "per_step"])


@pytest.fixture(scope="module")
def P():
    import paper_2407_02215_gb300 as P
    P.build_library()
    return P


def _maker(P, fused):
    def make(mesh, D, max_depth):
        g = P.CBT(mesh, D, max_depth)
        g.set_fused(fused)
        return g
    return make


def _export_check(g, o, fp, D):
    import torch
    vbuf = torch.empty((1 << D, 3, 3), dtype=torch.float32, device="cuda")
    g.update(fp, vertices_out=vbuf)
    o.update(fp)
    torch.cuda.synchronize()
    n = o.live_count
    assert g.live_count() == n and g.stats()["error"] == 0
    vo = o.vertices(fp.eye, fp.precision, fp.fixed_shift, fp.sphere_radius, frame=fp)
    vg = vbuf[:n].cpu().numpy()
    assert np.array_equal(vg.view(np.uint32), vo.view(np.uint32))
    return vg


@FORMS
def test_terrain_flythrough(P, fused):
    """A 30 x 30 grid flythrough with a 6-octave displacement on a 2^17
    pool: same states as the oracle every 5 frames, then one more frame's
    exported vertices bit-identical; the displacement changed the result
    (the undisplaced run ends elsewhere)."""
    spec = W.configs.config_terrain(n_frames=41, nx=30, D=17)
    g, o = run_pair(spec.mesh, 17, spec.max_depth, spec.frames[:-1], _maker(P, fused), Oracle, check_every=5)
    v = _export_check(g, o, spec.frames[-1], 17)
    flat = W.configs.config2(n_frames=41, nx=30)
    of = Oracle(flat.mesh, 17, flat.max_depth)
    for fp in flat.frames:
        of.update(fp)
    assert of.live_count != o.live_count or not np.array_equal(of.leaves()[1], o.leaves()[1])
    assert np.isfinite(v).all()


@FORMS
def test_displaced_planet(P, fused):
    """The dodecahedron planet with 30 km relief (4 octaves over the unit
    direction) on a 2^15 pool, every 3rd frame of the descent: same states as
    the oracle; then the exported sphere-form vertices of one more frame are
    bit-identical (the one-launch form copies them from its classify cache)."""
    spec = W.configs.config_waves(D=15, amp=3.0e4, freq=16.0, octaves=4, seed=31)
    frames = spec.frames[::3]
    g, o = run_pair(spec.mesh, 15, spec.max_depth, frames[:-1], _maker(P, fused), Oracle, check_every=10)
    _export_check(g, o, frames[-1], 15)


def test_wave_planet_end_of_descent(P):
    """The wave-planet workload as benchmarked (2 m waves, 1 km to 125 m
    cells, pool 2^17): the last 30 frames of the descent, on which the
    waves decide splits near the camera, equal the oracle's states."""
    spec = W.configs.config_waves()
    frames = spec.frames[:1] + spec.frames[-30:]
    run_pair(spec.mesh, spec.D, spec.max_depth, frames, _maker(P, True), Oracle, check_every=10)


def test_batch_mixed_displacement(P):
    """A batch of a displaced terrain, an undisplaced grid and a displaced
    planet, one launch per frame and per-step kernels: every instance equals
    its oracle every frame."""
    import torch
    t = W.configs.config_terrain(n_frames=12, nx=16, D=15)
    f = W.configs.config2(n_frames=12, nx=16)
    p = W.configs.config_waves(n_frames=300, D=14, amp=3.0e4, freq=16.0, octaves=3)
    pop = [(t.mesh, 15, t.max_depth, t.frames), (f.mesh, 15, f.max_depth, f.frames),
           (p.mesh, 14, p.max_depth, p.frames[100:300:17])]
    for fused in (True, False):
        gs = [P.CBT(m, D, md) for m, D, md, _ in pop]
        os_ = [Oracle(m, D, md) for m, D, md, _ in pop]
        batch = P.Batch(gs)
        batch.set_fused(fused)
        for k in range(12):
            batch.update([fr[k] for _, _, _, fr in pop])
            for b, o in enumerate(os_):
                o.update(pop[b][3][k])
            torch.cuda.synchronize()
            for b, (g, o) in enumerate(zip(gs, os_)):
                assert g.stats()["error"] == 0
                assert_same_state(g, o, f"fused={fused} frame {k} instance {b}")


def test_displacement_needs_fp32_or_sphere_form(P):
    """The displacement is defined for the FP32 and sphere forms only, with 1
    to 8 octaves and a positive frequency: anything else is CBT_EINVAL."""
    spec = W.configs.config_terrain(n_frames=2, nx=8, D=12)
    g = P.CBT(spec.mesh, 12, spec.max_depth)
    bad = []
    fp = spec.frames[0]
    for field, value in (("precision", PREC_FIXED), ("disp_octaves", 0), ("disp_octaves", 9),
                         ("disp_frequency", 0.0), ("disp_frequency", float("inf"))):
        old = getattr(fp, field)
        setattr(fp, field, value)
        with pytest.raises(P.CBTError):
            g.update(fp)
        setattr(fp, field, old)
        bad.append(field)
    g.update(fp)
    assert g.stats()["error"] == 0 and len(bad) == 5

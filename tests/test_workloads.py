"""The seeded workload recipes: each configuration has the sizes its
description states, and two calls give identical inputs (the oracle and the
CUDA path are fed from the same generator, so a drift here would go
unnoticed by parity)."""
import numpy as np
import pytest

import workloads as W
from oracle import halfedges_from_faces
from workloads.cameras import PREC_FIXED, PREC_FP32, PREC_SPHERE


def _H(mesh):
    return int(halfedges_from_faces(mesh)["twin"].shape[0])


def _same_frames(a, b):
    assert len(a) == len(b)
    for fa, fb in zip(a, b):
        for k, va in vars(fa).items():
            vb = getattr(fb, k)
            if isinstance(va, np.ndarray):
                assert np.array_equal(va, vb), k
            else:
                assert va == vb, k


@pytest.mark.parametrize("make", [
    lambda: W.configs.config1(), lambda: W.configs.config2(n_frames=12, nx=20),
    lambda: W.configs.config3(n_frames=20, D=16), lambda: W.configs.config_dodeca(n_frames=30),
    lambda: W.configs.config_waves(n_frames=30), lambda: W.configs.config_terrain(n_frames=12, nx=20)],
    ids=["cube", "grid", "cube_sphere", "dodeca", "waves", "terrain"])
def test_recipes_are_deterministic(make):
    a, b = make(), make()
    assert np.array_equal(a.mesh.pos, b.mesh.pos)
    assert np.array_equal(a.mesh.face_verts, b.mesh.face_verts)
    _same_frames(a.frames, b.frames)


def test_grid_flythrough_sizes():
    s = W.configs.config2()
    assert _H(s.mesh) == 42034 and s.D == 20 and s.max_depth == 26 and len(s.frames) == 120
    assert all(f.precision == PREC_FP32 and f.disp_amplitude == 0.0 for f in s.frames)


def test_planet_sizes():
    s = W.configs.config3()
    assert _H(s.mesh) == 1536 and s.D == 22 and s.max_depth == 48 and len(s.frames) == 600
    assert all(f.precision == PREC_FIXED for f in s.frames)
    r = np.linalg.norm(s.mesh.pos, axis=1)
    assert np.allclose(r, 6.371e6, rtol=1e-12)


def test_dodeca_and_wave_planet_sizes():
    d = W.configs.config_dodeca()
    assert _H(d.mesh) == 60 and d.D == 17 and d.max_depth == 50 and len(d.frames) == 300
    assert all(f.precision == PREC_SPHERE and f.sphere_radius == 6.371e6 and f.disp_amplitude == 0.0
               for f in d.frames)
    alt = [np.linalg.norm(f.eye) - 6.371e6 for f in d.frames]
    assert alt[0] == pytest.approx(2e7, rel=1e-6) and alt[-1] == pytest.approx(2.0, rel=1e-6)
    w = W.configs.config_waves()
    assert _H(w.mesh) == 60 and w.D == 17 and len(w.frames) == 300
    assert all((f.disp_amplitude, f.disp_frequency, f.disp_octaves, f.disp_seed) == (2.0, 6371.0, 4, 29)
               for f in w.frames)


def test_terrain_sizes():
    t = W.configs.config_terrain()
    assert _H(t.mesh) == 42034 and t.D == 20 and len(t.frames) == 120
    assert all((f.precision, f.disp_amplitude, f.disp_frequency, f.disp_octaves) == (PREC_FP32, 0.02, 4.0, 6)
               for f in t.frames)


def test_batch_population():
    """256 instances, halfedge counts log-uniform from 24 to 40k, pools from
    2^14 to 2^20, 64 frames each."""
    specs = W.configs.config4()
    assert len(specs) == 256
    Hs = np.array([_H(s.mesh) for s in specs])
    Ds = np.array([s.D for s in specs])
    assert Hs.max() <= 40000 and Hs.min() >= 24
    assert Ds.min() >= 14 and Ds.max() <= 20
    assert all(len(s.frames) == 64 for s in specs)
    assert all((1 << s.D) >= _H(s.mesh) for s in specs)

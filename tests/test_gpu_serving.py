"""Served form: requests arriving while other ticks run are admitted into
the next tick (continuous batching over resident instances), ticks overlap on
two streams, and every instance ends in exactly the state it reaches when its
frames run alone through cbt_update."""
import numpy as np
import pytest

import workloads as W
from workloads.cameras import MODE_RANDOM, forced_params
from workloads.configs import InstanceSpec

pytestmark = pytest.mark.gpu


def _population():
    specs = [InstanceSpec("fig1", W.meshes.fig1_mesh(), 7, 6,
                          [forced_params(MODE_RANDOM, seed=11) for _ in range(10)]),
             InstanceSpec("tetra", W.meshes.tetra_mesh(), 9, 7,
                          [forced_params(MODE_RANDOM, seed=12) for _ in range(10)])]
    c1 = W.configs.config1(n_frames=12)
    specs.append(InstanceSpec("cube", c1.mesh, 15, 12, c1.frames))
    for k, (nx, D) in enumerate(((10, 15), (16, 16), (24, 17))):
        m = W.meshes.grid_mesh(nx, nx, 0.15, seed=20 + k)
        cams = W.cameras.flythrough_path(12, seed=20 + k, alt_lo=0.03)
        specs.append(InstanceSpec(f"grid{nx}", m, D, 20, [W.cameras.frame_params(c, 2.5) for c in cams]))
    return specs


@pytest.mark.parametrize("fused", [False, True], ids=["per_step", "fused"])
def test_served_results_equal_alone(fused):
    import torch

    import paper_2407_02215_gb300 as P
    from paper_2407_02215_gb300.serving import ServeLoop, ping_pong
    P.build_library()
    loop = ServeLoop(_population(), hbm_budget_bytes=1 << 36, inflight=2, max_batch=4, fused=fused)
    stats = loop.run(rate_hz=4000.0, duration_s=5.0, seed=7, max_requests=240)
    assert stats["requests"] == 240
    assert stats["p99_ms"] >= stats["p50_ms"] > 0.0
    assert 1.0 <= stats["mean_batch"] <= 4.0
    torch.cuda.synchronize()
    for b, spec in enumerate(loop.specs):
        alone = P.CBT(spec.mesh, spec.D, spec.max_depth)
        for k in range(loop.served[b]):
            alone.update(ping_pong(spec.frames, k))
        mixed = loop.instances[b]
        assert mixed.stats()["error"] == 0
        for x, y in zip(mixed.leaves(), alone.leaves()):
            assert torch.equal(x, y), spec.name
        for x, y in zip(mixed.cbt(), alone.cbt()):
            assert torch.equal(x[1:], y[1:]), spec.name
    assert sum(loop.served) == 240


def test_hbm_budget_admission():
    import paper_2407_02215_gb300 as P
    from paper_2407_02215_gb300.serving import ServeLoop
    P.build_library()
    specs = _population()
    need = [P.workspace_bytes(s.mesh.H, s.D) for s in specs]
    budget = sum(need[:3])
    loop = ServeLoop(specs, hbm_budget_bytes=budget, inflight=2)
    assert [s.name for s in loop.specs] == [s.name for s in specs[:3]]
    assert loop.rejected == [s.name for s in specs[3:]]


def _forms_population():
    """Every vertex form: displaced FP32 terrain, the sphere-projected
    dodecahedron planet (plain and displaced) and the fixed-point cube
    sphere, each a short stretch of its own path."""
    t = W.configs.config_terrain(n_frames=10, nx=14, D=15)
    d = W.configs.config_dodeca(n_frames=300, D=14)
    w = W.configs.config_waves(n_frames=300, D=14, amp=3.0e4, freq=16.0, octaves=3)
    p = W.configs.config3(n_frames=600, D=15)
    return [InstanceSpec("terrain", t.mesh, 15, t.max_depth, t.frames),
            InstanceSpec("dodeca", d.mesh, 14, d.max_depth, d.frames[100:300:20]),
            InstanceSpec("waves", w.mesh, 14, w.max_depth, w.frames[100:300:20]),
            InstanceSpec("planet", p.mesh, 15, p.max_depth, p.frames[200:600:40])]


@pytest.mark.parametrize("fused", [False, True], ids=["per_step", "fused"])
def test_served_vertex_forms_equal_alone(fused):
    """Served ticks that mix the FP32, displaced, sphere and fixed-point
    forms leave every instance in the state its frames give alone."""
    import torch

    import paper_2407_02215_gb300 as P
    from paper_2407_02215_gb300.serving import ServeLoop, ping_pong
    P.build_library()
    loop = ServeLoop(_forms_population(), hbm_budget_bytes=1 << 36, inflight=2, max_batch=4, fused=fused)
    stats = loop.run(rate_hz=3000.0, duration_s=5.0, seed=9, max_requests=80)
    assert stats["requests"] == 80
    torch.cuda.synchronize()
    for b, spec in enumerate(loop.specs):
        alone = P.CBT(spec.mesh, spec.D, spec.max_depth)
        for k in range(loop.served[b]):
            alone.update(ping_pong(spec.frames, k))
        mixed = loop.instances[b]
        assert mixed.stats()["error"] == 0
        for x, y in zip(mixed.leaves(), alone.leaves()):
            assert torch.equal(x, y), spec.name

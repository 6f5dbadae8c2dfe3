"""Batched form: many uneven instances updated by one launch per kernel give,
instance by instance and frame by frame, exactly the oracle's states; so do
CUDA-graph replay, the online autotuner's changing tile and grid sizes, and a
single instance replayed as a graph."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from workloads.cameras import MODE_RANDOM, PREC_FIXED, forced_params
from tests.gpu_helpers import assert_same_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2407_02215_gb300 as P
    P.build_library()
    return P


def _population():
    """Instances of very different sizes and modes, each with its frames."""
    pop = []
    pop.append((W.meshes.fig1_mesh(), 6, 6, [forced_params(MODE_RANDOM, seed=1) for _ in range(24)]))
    pop.append((W.meshes.tetra_mesh(), 9, 7, [forced_params(MODE_RANDOM, seed=2) for _ in range(24)]))
    spec = W.configs.config1(n_frames=24)
    pop.append((spec.mesh, 14, 14, spec.frames))
    g = W.meshes.grid_mesh(12, 12, 0.2, seed=5)
    cams = W.cameras.flythrough_path(24, seed=5, alt_lo=0.02)
    pop.append((g, 16, 22, [W.cameras.frame_params(c, 2.0) for c in cams]))
    g2 = W.meshes.grid_mesh(30, 20, 0.1, seed=6)
    cams2 = W.cameras.flythrough_path(24, seed=6, alt_lo=0.05)
    pop.append((g2, 18, 22, [W.cameras.frame_params(c, 3.0, precision=PREC_FIXED) for c in cams2]))
    pop.append((W.meshes.cube_mesh(), 5, 10, [forced_params(MODE_RANDOM, seed=3) for _ in range(24)]))
    return pop


def _run_batch(P, graph=False, autotune=0, vertices=False, fused=True):
    import torch
    pop = _population()
    gs = [P.CBT(m, D, md) for m, D, md, _ in pop]
    os_ = [Oracle(m, D, md) for m, D, md, _ in pop]
    batch = P.Batch(gs)
    batch.set_fused(fused)
    if graph:
        batch.set_graph(True)
    if autotune:
        batch.autotune(autotune)
    vbufs = [torch.empty((1 << D, 3, 3), dtype=torch.float32, device="cuda") for _, D, _, _ in pop] if vertices else None
    nf = len(pop[0][3])
    for k in range(nf):
        batch.update([fr[k] for _, _, _, fr in pop], vertices_out=vbufs)
        for b, o in enumerate(os_):
            o.update(pop[b][3][k])
        torch.cuda.synchronize()
        for b, (g, o) in enumerate(zip(gs, os_)):
            st = g.stats()
            assert st["error"] == 0
            if k % 6 == 5 or k == nf - 1:
                assert_same_state(g, o, f"instance {b} frame {k}")
                if vertices:
                    fp = pop[b][3][k]
                    n = o.live_count
                    vo = o.vertices(fp.eye, fp.precision, fp.fixed_shift)
                    vg = vbufs[b][:n].cpu().numpy()
                    assert np.array_equal(vg.view(np.uint32), vo.view(np.uint32)), f"instance {b} vertices"
    return batch


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "per_step"])
def test_batch_matches_oracle_per_instance(P, fused):
    b = _run_batch(P, vertices=True, fused=fused)
    assert b.last_launch_count == (1 if fused else 11)


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "per_step"])
def test_batch_graph_replay(P, fused):
    _run_batch(P, graph=True, fused=fused)


def test_batch_autotune_keeps_results(P):
    b = _run_batch(P, autotune=2)
    cfg = b.config()
    assert not cfg["tuning"] and cfg["tile_words"] in (64, 128, 256)


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "per_step"])
def test_single_instance_graph_mode(P, fused):
    spec = W.configs.config1()
    g = P.CBT(spec.mesh, spec.D, spec.max_depth)
    g.set_fused(fused)
    g.set_graph(True)
    o = Oracle(spec.mesh, spec.D, spec.max_depth)
    for k, fp in enumerate(spec.frames):
        g.update(fp)
        o.update(fp)
    assert_same_state(g, o, "graph")

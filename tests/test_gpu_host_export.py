"""The frame's vertex export written straight into pinned host memory (its
mapped device address, cbt_host_device_pointer) equals the export into
device memory bit for bit, in the one-launch and per-step forms; so does
cbt_vertices_to_host's copy of the device export; an unpinned host tensor
is refused."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2407_02215_gb300 as P
    P.build_library()
    return P


@pytest.mark.parametrize("fused", [True, False], ids=["fused", "per_step"])
def test_pinned_host_export_matches_device(P, fused):
    import torch
    spec = W.configs.config2(n_frames=16, nx=30)
    a = P.CBT(spec.mesh, 17, spec.max_depth)
    b = P.CBT(spec.mesh, 17, spec.max_depth)
    a.set_fused(fused)
    b.set_fused(fused)
    dv = torch.empty((1 << 17, 3, 3), dtype=torch.float32, device="cuda")
    hv = torch.empty((1 << 17, 3, 3), dtype=torch.float32, pin_memory=True)
    for fp in spec.frames:
        a.update(fp, vertices_out=dv)
        b.update(fp, vertices_out=hv)
        n = b.live_count()
        assert a.live_count() == n
        assert np.array_equal(dv[:n].cpu().numpy().view(np.uint32), hv[:n].numpy().view(np.uint32))


def test_unpinned_host_tensor_refused(P):
    import torch
    spec = W.configs.config1(n_frames=2)
    g = P.CBT(spec.mesh, 14, 14)
    with pytest.raises(P.CBTError):
        g.update(spec.frames[0], vertices_out=torch.empty((1 << 14, 3, 3), dtype=torch.float32))


def test_vertices_to_host(P):
    import torch
    spec = W.configs.config2(n_frames=8, nx=30)
    g = P.CBT(spec.mesh, 17, spec.max_depth)
    dv = torch.empty((1 << 17, 3, 3), dtype=torch.float32, device="cuda")
    hv = torch.full((1 << 17, 3, 3), -1.0, dtype=torch.float32, pin_memory=True)
    hn = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    for fp in spec.frames:
        g.update(fp, vertices_out=dv)
        n = g.vertices_to_host(dv, hv, hn)
        assert n == g.live_count()
        assert np.array_equal(dv[:n].cpu().numpy().view(np.uint32), hv[:n].numpy().view(np.uint32))
    small = torch.empty((16, 3, 3), dtype=torch.float32, pin_memory=True)
    with pytest.raises(P.CBTError):
        g.vertices_to_host(dv, small, hn)
    assert int(hn[0]) == g.live_count()
    assert np.array_equal(dv[:16].cpu().numpy().view(np.uint32), small.numpy().view(np.uint32))


def test_live_count_async_into_pinned_and_device_memory(P):
    """cbt_live_count_async enqueues the count behind the frame on the same
    stream: after a stream synchronisation the pinned word and the device
    word hold the count cbt_live_count returns, frame after frame; and the
    rows cbt_vertices_to_host_async then copies out on a second stream equal
    the device export."""
    import torch
    spec = W.configs.config2(n_frames=12, nx=30)
    g = P.CBT(spec.mesh, 17, spec.max_depth)
    s, side = torch.cuda.Stream(), torch.cuda.Stream()
    dv = torch.empty((1 << 17, 3, 3), dtype=torch.float32, device="cuda")
    hv = torch.empty((1 << 17, 3, 3), dtype=torch.float32, pin_memory=True)
    hn = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    dn = torch.zeros(1, dtype=torch.int32, device="cuda")
    for fp in spec.frames:
        with torch.cuda.stream(s):
            g.update(fp, stream=s, vertices_out=dv)
            g.live_count_async(hn, stream=s)
            g.live_count_async(dn, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        ev.synchronize()
        n = int(hn[0])
        side.wait_event(ev)
        hv.fill_(float("nan"))
        P.vertices_to_host_async(dv, hv, n, stream=side)  # cbt_vertices_to_host_async
        side.synchronize()
        assert n == g.live_count() == int(dn.cpu()[0])
        assert np.array_equal(dv[:n].cpu().numpy().view(np.uint32), hv[:n].numpy().view(np.uint32))
    with pytest.raises(ValueError):
        g.live_count_async(torch.zeros(1, dtype=torch.int32))  # neither CUDA nor pinned

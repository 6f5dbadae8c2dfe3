"""Host logic of the continuous-batching serving loop, on the CPU: the
device instances, the tick server and the streams are replaced by fakes, so
the admission by memory budget and the scheduling (one tick in flight per
instance, each instance's frames in order, oldest request first, at most
max_batch per tick, every request answered) are checked without a GPU."""
import types

import pytest

import paper_2407_02215_gb300.serving as S


class FakeCBT:
    def __init__(self, mesh, D, max_depth, device=None):
        self.mesh, self.D = mesh, D


class FakeServer:
    """Ticks complete after `delay` polls; a tick reports one live count per
    instance in it (the instance's index times 10 plus its frame number)."""

    def __init__(self, instances, inflight, delay=2):
        self.instances, self.inflight, self.delay = instances, inflight, delay
        self.workspace = types.SimpleNamespace(numel=lambda: 1000)
        self.pending, self.log, self.next_tk, self.fused = {}, [], 0, False

    def set_fused(self, on):
        self.fused = on

    def next_slot_free(self):
        return len(self.pending) < self.inflight

    def submit(self, pick, fps, stream=None):
        tk = self.next_tk
        self.next_tk += 1
        self.pending[tk] = [self.delay, list(pick), list(fps)]
        self.log.append((tk, list(pick), list(fps)))
        return tk

    def poll(self, tk):
        p = self.pending[tk]
        p[0] -= 1
        if p[0] > 0:
            return None
        del self.pending[tk]
        return [10 * b + f for b, f in zip(p[1], p[2])]


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(S, "CBT", FakeCBT)
    monkeypatch.setattr(S, "Server", FakeServer)
    monkeypatch.setattr(S, "workspace_bytes", lambda H, D: H * (1 << D))
    monkeypatch.setattr(S.torch.cuda, "Stream", lambda device=None: object())
    return S


def _spec(name, H, D, n_frames=5):
    return types.SimpleNamespace(name=name, mesh=types.SimpleNamespace(H=H), D=D, max_depth=8,
                                 frames=list(range(n_frames)))


def test_admission_by_budget(fakes):
    specs = [_spec("a", 10, 4), _spec("b", 10, 6), _spec("c", 10, 4), _spec("d", 10, 5)]
    loop = fakes.ServeLoop(specs, hbm_budget_bytes=160 + 160 + 320, device="cpu")
    # a (160) fits, b (640) does not, c (160) fits, d (320) fits exactly
    assert [s.name for s in loop.specs] == ["a", "c", "d"]
    assert loop.rejected == ["b"]
    assert loop.hbm_used == 640 + 1000  # instances plus the server's own workspace


@pytest.mark.parametrize("max_batch", [1, 2, 64])
def test_saturated_server_schedule(fakes, max_batch):
    specs = [_spec(f"i{k}", 8, 4, n_frames=3) for k in range(5)]
    loop = fakes.ServeLoop(specs, hbm_budget_bytes=10 ** 9, inflight=2, max_batch=max_batch, device="cpu")
    per = 7
    out = loop.run(rate_hz=1.0, duration_s=60.0, per_instance=per)
    assert out["requests"] == 5 * per
    log = loop.server.log
    assert all(len(pick) <= max_batch for _, pick, _ in log)
    # each instance's frames follow its camera path played back and forth
    seen = {b: [] for b in range(5)}
    for _, pick, fps in log:
        assert len(set(pick)) == len(pick)
        for b, f in zip(pick, fps):
            seen[b].append(f)
    for b in range(5):
        assert seen[b] == [S.ping_pong(specs[b].frames, k) for k in range(per)]
    assert loop.served == [per] * 5


def test_one_tick_in_flight_per_instance(fakes):
    """An instance joins no tick while one of its ticks is still running."""
    specs = [_spec(f"i{k}", 8, 4) for k in range(3)]
    loop = fakes.ServeLoop(specs, hbm_budget_bytes=10 ** 9, inflight=3, device="cpu")
    loop.server.delay = 3
    running = {}
    submit = loop.server.submit
    poll = loop.server.poll

    def submit_checked(pick, fps, stream=None):
        for b in pick:
            assert b not in running.values(), f"instance {b} submitted twice"
        tk = submit(pick, fps, stream)
        for b in pick:
            running[(tk, b)] = b
        return tk

    def poll_checked(tk):
        res = poll(tk)
        if res is not None:
            for key in [k for k in running if k[0] == tk]:
                del running[key]
        return res

    loop.server.submit, loop.server.poll = submit_checked, poll_checked
    out = loop.run(rate_hz=1.0, duration_s=60.0, per_instance=4)
    assert out["requests"] == 12 and not running


def test_oldest_request_first(fakes, monkeypatch):
    """Six requests arrive at once, for instances 2, 0, 1, 2, 0, 1 in that
    order; with one tick of one instance at a time, the ticks take them in
    arrival order (each tick the instance whose queued request is oldest)."""
    order = iter([2, 0, 1, 2, 0, 1])

    class ScriptedRng:
        def __init__(self, seed=None):
            pass

        def exponential(self, scale):
            return 1e-9

        def integers(self, n):
            return next(order)

    monkeypatch.setattr(S.np.random, "default_rng", ScriptedRng)
    specs = [_spec(f"i{k}", 8, 4) for k in range(3)]
    loop = fakes.ServeLoop(specs, hbm_budget_bytes=10 ** 9, inflight=1, max_batch=1, device="cpu")
    loop.server.delay = 1
    out = loop.run(rate_hz=1.0, duration_s=60.0, max_requests=6)
    assert out["requests"] == 6
    assert [pick[0] for _, pick, _ in loop.server.log] == [2, 0, 1, 2, 0, 1]


def test_poisson_arrivals_all_answered(fakes):
    specs = [_spec(f"i{k}", 8, 4) for k in range(4)]
    loop = fakes.ServeLoop(specs, hbm_budget_bytes=10 ** 9, inflight=2, device="cpu")
    out = loop.run(rate_hz=20000.0, duration_s=5.0, seed=3, max_requests=300)
    assert out["requests"] == 300
    assert sum(loop.served) == 300
    assert out["p99_ms"] >= out["p50_ms"] >= 0.0

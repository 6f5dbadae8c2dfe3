"""Continuous-batching serving loop over resident CBT instances.

Requests (an instance and its next camera) arrive as a seeded Poisson
process into per-instance FIFO queues. Instances are admitted at start-up
while their workspaces fit the HBM budget and stay resident. Whenever a tick
slot is free, every admitted instance with a queued request and no tick in
flight joins the next tick (oldest request first, up to max_batch); ticks go
to alternating streams, so a tick that starts while another runs overlaps it
on the device. A request's latency runs from its arrival to the host seeing
its tick complete. Each instance's frames are applied in order, so its
result is exactly the one it would get alone.
"""
from __future__ import annotations

import gc
import time
from collections import deque

import numpy as np
import torch

from .cbt import CBT, Server, workspace_bytes


def ping_pong(frames, k):
    """The k-th frame of a camera path played back and forth."""
    n = len(frames)
    cyc, pos = divmod(k, n)
    return frames[pos] if cyc % 2 == 0 else frames[n - 1 - pos]


class ServeLoop:
    def __init__(self, specs, hbm_budget_bytes: int, inflight: int = 2, max_batch: int = 512,
                 device="cuda", fused: bool = False):
        self.device = torch.device(device)
        self.specs, self.instances, self.rejected = [], [], []
        used = 0
        for spec in specs:
            need = workspace_bytes(spec.mesh.H, spec.D)
            if used + need > hbm_budget_bytes:
                self.rejected.append(spec.name)
                continue
            used += need
            self.instances.append(CBT(spec.mesh, spec.D, spec.max_depth, device=self.device))
            self.specs.append(spec)
        self.hbm_used = used
        self.server = Server(self.instances, inflight)
        if fused:
            self.server.set_fused(True)
        self.hbm_used += self.server.workspace.numel()
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(inflight)]
        self.max_batch = max_batch
        self.served = [0] * len(self.instances)  # frames applied per instance

    def run(self, rate_hz: float, duration_s: float, seed: int = 0, max_requests: int | None = None,
            per_instance: int | None = None):
        """Serves Poisson arrivals at rate_hz for duration_s (or until
        max_requests arrived); with per_instance, every instance instead has
        that many requests queued at the start (a saturated server, equal work
        per instance). Python's garbage collector is paused meanwhile (a
        collection over the loop's objects stalls the host for milliseconds)."""
        gc_was = gc.isenabled()
        gc.disable()
        try:
            return self._run(rate_hz, duration_s, seed, max_requests, per_instance)
        finally:
            if gc_was:
                gc.enable()

    def _run(self, rate_hz, duration_s, seed, max_requests, per_instance):
        rng = np.random.default_rng(seed)
        n = len(self.instances)
        queues = [deque() for _ in range(n)]
        ready = set()  # instances with a queued request and no tick in flight
        busy = set()
        inflight = {}
        lat, bis, completed, ticks, batch_sizes = [], 0, 0, 0, []
        arrivals = 0
        t0 = time.perf_counter()
        next_arr = t0 + rng.exponential(1.0 / rate_hz)
        if per_instance is not None:
            for b in range(n):
                queues[b].extend([t0] * per_instance)
                ready.add(b)
            arrivals = max_requests = n * per_instance
            next_arr = float("inf")
        stream_i = 0
        while True:
            now = time.perf_counter()
            open_ = now - t0 <= duration_s and (max_requests is None or arrivals < max_requests)
            while open_ and next_arr <= now:
                b = int(rng.integers(n))
                queues[b].append(next_arr)
                arrivals += 1
                if b not in busy:
                    ready.add(b)
                next_arr += rng.exponential(1.0 / rate_hz)
                if max_requests is not None and arrivals >= max_requests:
                    break
            for tk in list(inflight):
                res = self.server.poll(tk)
                if res is None:
                    continue
                done_t = time.perf_counter()
                idx, arr = inflight.pop(tk)
                for b, a, live in zip(idx, arr, res):
                    lat.append(done_t - a)
                    bis += live
                    completed += 1
                    busy.discard(b)
                    if queues[b]:
                        ready.add(b)
            if ready and self.server.next_slot_free():
                pick = sorted(ready, key=lambda b: queues[b][0])[: self.max_batch]
                fps, arr = [], []
                for b in pick:
                    arr.append(queues[b].popleft())
                    fps.append(ping_pong(self.specs[b].frames, self.served[b]))
                    self.served[b] += 1
                    ready.discard(b)
                    busy.add(b)
                tk = self.server.submit(pick, fps, stream=self.streams[stream_i])
                stream_i = (stream_i + 1) % len(self.streams)
                inflight[tk] = (pick, arr)
                ticks += 1
                batch_sizes.append(len(pick))
            if not open_ and not inflight and not ready:
                break
        wall = time.perf_counter() - t0
        lat_ms = np.array(lat) * 1e3 if lat else np.zeros(1)
        return {
            "rate_hz": rate_hz, "requests": completed, "ticks": ticks, "wall_s": wall,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "requests_per_s": completed / wall, "bisectors_per_s": bis / wall,
            "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else 0.0,
        }

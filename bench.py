#!/usr/bin/env python
"""Benchmark of the per-frame CBT adaptive-bisection update on GB300.

One step = one frame of the whole update (classify, chain gate, chain
scatter, allocation, free-slot decode, fill/relink, CBT reduction + live-slot
compaction, vertex export) over the grid workload: a 100 x 100 mixed
quad/triangle mesh (42,034 halfedges), a pool of 2^20 bisectors, max depth
26, a 120-frame seeded flythrough, LOD threshold 2 px at 1920x1080.

Frames are stateful: the timed run starts from the root bisectors and plays
frames 0..K-1; the W warm-up frames run on a separate, discarded instance.
The pool (about 55 MB) fits in L2, so L2 is flushed (a 256 MiB write) before
every timed frame, outside the frame's CUDA-event interval.

value = bisectors updated per second = sum over frames of the live count at
frame start / sum of frame times (device time, CUDA events). With --gpus N
(torchrun) every rank runs its own replica of the workload (the update of one
instance does not shard); value sums the ranks' bisectors over the slowest
rank's time.

--impl reference times the CPU oracle (sequential C, one core) on the same
workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "bisectors updated/sec (per-frame CBT bisection update)"
UNIT = "bisectors/s"
L2_FLUSH_BYTES = 256 << 20


def frames_for(spec, K):
    """K stateful frames: the camera path, continued back and forth."""
    fr = list(spec.frames)
    out = []
    while len(out) < K:
        out.extend(fr if (len(out) // len(fr)) % 2 == 0 else fr[::-1])
    return out[:K]


def workload_config(spec, K):
    return {"workload": f"{spec.name}: {spec.mesh.name} ({spec.mesh.H} halfedges), pool 2^{spec.D}, "
                        f"max depth {spec.max_depth}, {K}-frame flythrough, LOD 2 px at 1920x1080",
            "halfedges": spec.mesh.H, "pool_log2": spec.D, "max_depth": spec.max_depth,
            "frames": K, "l2": "flushed before every timed frame (256 MiB write)"}


# ------------------------------------------------------------ algorithmic bytes

STEP_KERNELS = ("prep", "classify", "walk", "gate", "scatter", "alloc", "free", "fill", "cbt", "vertices")

# DRAM traffic of the one-launch frame from one ncu capture (dram__bytes_read
# + dram__bytes_write, L2 flushed before each pass), per live bisector at
# frame start, valid only for the kernel code it was taken on: the hash below
# is over the sources' code lines with their // comments removed, so that an
# edit of comments alone keeps the capture.
FRAME_TRAFFIC = {"code_sha256_16": "d4cbf5a756f0205c", "bytes_per_live": 70.4,
                 "capture": "k_frame1, frames 8 and 9 of the flythrough: 50.9 MB at 712,190 live, "
                            "52.0 MB at 748,560 live"}
FRAME_SOURCES = ("cbt_fused.cu", "cbt_phases.cuh", "cbt_device.cuh")


def frame_code_hash():
    """SHA-256 (first 16 hex digits) of the frame kernel's code lines."""
    import hashlib
    h = hashlib.sha256()
    for f in FRAME_SOURCES:
        with open(os.path.join(ROOT, "paper_2407_02215_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def frame_traffic(mean_live):
    """Measured DRAM bytes per launch scaled to the mean live count, or None
    once the kernel code differs from the code the capture was taken on."""
    if frame_code_hash() != FRAME_TRAFFIC["code_sha256_16"]:
        return None
    return FRAME_TRAFFIC["bytes_per_live"] * mean_live


def frame_bytes(st: dict, cap: int, export: bool = True) -> float:
    """The bytes one frame must move, from the frame's counters: per live
    bisector at frame start (N) its record read once (8 B heap ID, 4 B root
    slot, 12 B links), its 4 B command word written and about 8 B of scan
    words; 24 B per new record (A); 12 B per rewritten link of an unchanged
    neighbour (U); the bitfield read and written (2^D / 8 B each) and the
    sum tree written (8 B per bitfield word); with the export, 36 B per live
    bisector after the frame (N')."""
    N, A, U, N2 = st["live_before"], st["allocated"], st["relinked"], st["live_after"]
    W = max(1, cap // 32)
    b = N * (8 + 4 + 12) + N * 4 + N * 8 + A * 24 + U * 12 + 2 * cap / 8 + 8 * W
    return float(b + (36 * N2 if export else 0))


def algorithmic_bytes(kernel: str, st: dict, cap: int) -> float:
    """Bytes each kernel must move per frame at minimum, from the frame's
    counters: N live at frame start, S split and M merged bisectors, A new
    records, U relinked unchanged neighbours, SW split wishes, MC merge
    candidates, Wd bitfield words."""
    N, A, U = st["live_before"], st["allocated"], st["relinked"]
    S, M = st["split_bisectors"], st["merged_bisectors"]
    SW, MC = st["split_wishes"], st["merge_candidates"]
    Wd = max(1, cap // 32)
    N2 = st["live_after"]
    return {
        # live slot, heap ID in; command word and cost out
        "classify": 20.0 * N,
        # live slot and command in; per split wish the twin record (links +
        # heap) and its cost out; per merge candidate three member records
        "walk": 8.0 * N + 28.0 * SW + 3 * 24.0 * MC,
        # live slot, command, cost in; running total out; the members'
        # command words per merge candidate
        "gate": 16.0 * N + 3 * 8.0 * MC,
        # live slot, command, running total; command OR on chain members
        "scatter": 12.0 * N + 28.0 * SW,
        # live slot and command in, destination out for changed bisectors
        "alloc": 8.0 * N + 4.0 * (S + M),
        # bitfield words up to the A-th zero (at most all) and A slots out
        "free": 4.0 * Wd + 4.0 * A,
        # live slot + command/destination per live; changed records in; new
        # records (heap 8 + links 16) out; one neighbour command/destination
        # and free-list entry per external edge (about 3 per new record);
        # 8 bytes per relinked neighbour
        "fill": 12.0 * N + 24.0 * (S + M) + 24.0 * A + 3 * 12.0 * A + 8.0 * U,
        # reduction: bitfield in, sum tree (2 x words) out; compaction:
        # bitfield in again, live list out
        "cbt": 4.0 * Wd + 8.0 * Wd + 4.0 * Wd + 4.0 * N2,
        # live slot, heap ID in; 9 floats out
        "vertices": (4.0 + 8.0 + 36.0) * N2,
        "prep": 0.0,
    }.get(kernel, 0.0)


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of this GPU's clocks during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        out_dir = os.environ.get("CBT_BENCH_OUT", os.path.join(tempfile.gettempdir(), "cbt_bench"))
        self.path = os.path.join(out_dir, f"clocks_rank{device_index}.csv")
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            self.sel = ["-i", uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"]
        except Exception:
            self.sel = []

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", *self.sel, f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# -------------------------------------------------------------- CPU oracle

def run_oracle(spec, frames, budget_s, lives=None):
    """Times the CPU oracle (one core) on frames until budget_s is spent;
    returns (bisectors, seconds, frames done); appends each frame's live
    count after the update to `lives` when given."""
    from oracle import Oracle
    o = Oracle(spec.mesh, spec.D, spec.max_depth)
    bis, secs, done = 0, 0.0, 0
    for fp in frames:
        t = time.perf_counter()
        st = o.update(fp)
        secs += time.perf_counter() - t
        bis += st["live_before"]
        done += 1
        if lives is not None:
            lives.append(st["live_after"])
        if secs >= budget_s:
            break
    return bis, secs, done


def cpu_baseline(spec, frames, budget_s=15.0, gpu_lives=None):
    """The oracle timed on a bounded sample of the frames; with the timed
    GPU run's per-frame live counts, also whether they equal the oracle's
    over that sample (the timed run doubles as a parity run)."""
    lives = []
    bis, secs, done = run_oracle(spec, frames, budget_s, lives)
    out = {"value": bis / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"first {done} frames of the same flythrough ({bis} bisector updates, "
                     f"{secs:.1f} s, sequential C oracle on one host core)"}
    if gpu_lives is not None:
        out["timed_run_live_counts_equal_oracle"] = list(gpu_lives[:done]) == lives
    return out


# -------------------------------------------------------------------- main

def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, world, op):
    """All-reduce of one number over the ranks (NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def reduce_max(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX) if world > 1 else x


def reduce_sum(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM) if world > 1 else x


def bench_ours(args):
    import torch

    from paper_2407_02215_gb300 import CBT

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    spec = W.configs.config2()
    frames = frames_for(spec, args.steps)
    warm = frames_for(spec, max(args.warmup, 0))

    # warm-up on a discarded instance
    g0 = CBT(spec.mesh, spec.D, spec.max_depth, device=dev)
    vbuf = torch.empty((1 << spec.D, 3, 3), dtype=torch.float32, device=dev)
    for fp in warm:
        g0.update(fp, vertices_out=vbuf)
    torch.cuda.synchronize()
    g0.stats()
    del g0

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # timed pass: one cooperative launch per frame (a single fused instance
    # launches directly even with graphs on), one event pair per frame
    g = CBT(spec.mesh, spec.D, spec.max_depth, device=dev)
    g.set_graph(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in frames]
    clocks = ClockSampler(dev.index or 0) if rank == 0 else None
    stats = []
    launches = 0
    if clocks:
        clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    for k, fp in enumerate(frames):
        flush.zero_()
        ev[k][0].record()
        g.update(fp, vertices_out=vbuf)
        ev[k][1].record()
        launches += g.last_launch_count
        stats.append(g.stats())
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if clocks else None
    ms = np.array([a.elapsed_time(b) for a, b in ev])
    bis = float(sum(s["live_before"] for s in stats))
    t_local = float(ms.sum()) / 1e3
    t_max = reduce_max(t_local, world)
    bis_all = reduce_sum(bis, world)
    value = bis_all / t_max

    # phase breakdown: the same frames again on a fresh instance; the one-launch
    # frame reads the device timer at its phase boundaries (block 0)
    gk = CBT(spec.mesh, spec.D, spec.max_depth, device=dev)
    gk.set_timing(True)
    ptimes, kbytes = {}, {}
    for fp in frames:
        flush.zero_()
        gk.update(fp, vertices_out=vbuf)
        for name, pms in gk.kernel_times().items():
            ptimes[name] = ptimes.get(name, 0.0) + pms
        st = gk.stats()
        for k in STEP_KERNELS:
            kbytes[k] = kbytes.get(k, 0.0) + algorithmic_bytes(k, st, 1 << spec.D)
    del gk
    fbytes = sum(frame_bytes(st, 1 << spec.D) for st in stats)

    # the per-step form (one launch per step, CUDA graph) on the same frames,
    # for comparison, and its per-kernel times (events between the launches)
    gs = CBT(spec.mesh, spec.D, spec.max_depth, device=dev)
    gs.set_fused(False)
    gs.set_graph(True)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in frames]
    for k, fp in enumerate(frames):
        flush.zero_()
        ev2[k][0].record()
        gs.update(fp, vertices_out=vbuf)
        ev2[k][1].record()
    torch.cuda.synchronize()
    ms_steps = np.array([a.elapsed_time(b) for a, b in ev2])
    gs.set_graph(False)
    del gs
    gt = CBT(spec.mesh, spec.D, spec.max_depth, device=dev)
    gt.set_fused(False)
    gt.set_timing(True)
    ktimes = {}
    for fp in frames:
        flush.zero_()
        gt.update(fp, vertices_out=vbuf)
        for name, kms in gt.kernel_times().items():
            ktimes[name] = ktimes.get(name, 0.0) + kms
    del gt

    # end to end through the C ABI with host buffers: the frame parameters go
    # host -> device as launch arguments; the frame exports its vertices to
    # device memory and cbt_vertices_to_host moves them, with the live count,
    # into pinned host memory under one synchronisation, every frame.
    g2 = CBT(spec.mesh, spec.D, spec.max_depth, device=dev)
    host_v = torch.empty((1 << spec.D, 3, 3), dtype=torch.float32, pin_memory=True)
    host_n = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    e2e_t, e2e_bis, d2h = 0.0, 0, 0
    barrier(world)
    for fp in frames:
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2.update(fp, vertices_out=vbuf)
        n = g2.vertices_to_host(vbuf, host_v, host_n)
        e2e_t += time.perf_counter() - t0
        d2h += 4 + 36 * n
    del g2
    # the same with cbt_live_count and a copy-engine copy after it (reported
    # beside it)
    g3 = CBT(spec.mesh, spec.D, spec.max_depth, device=dev)
    copy_t = 0.0
    for fp in frames:
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g3.update(fp, vertices_out=vbuf)
        n = g3.live_count()
        host_v[:n].copy_(vbuf[:n], non_blocking=True)
        torch.cuda.current_stream().synchronize()
        copy_t += time.perf_counter() - t0
    del g3
    copy_val = reduce_sum(float(sum(st["live_before"] for st in stats)), world) / reduce_max(copy_t, world)
    for st in stats:
        e2e_bis += st["live_before"]
    e2e_tmax = reduce_max(e2e_t, world)
    e2e_val = reduce_sum(float(e2e_bis), world) / e2e_tmax

    # end to end, pipelined (the e2e value): frame k runs on stream A while
    # the copy engine moves frame k-1's rows, their number enqueued by
    # cbt_live_count_async behind that frame, into pinned host memory on
    # stream B (cbt_vertices_to_host_async); two device and two host
    # buffers, and stream A waits for the copy out of a buffer before a frame
    # writes it again. Each frame's cbt_frame is built before the loop (a C
    # caller keeps its own), and the loop makes one library call per step.
    # The 256 MiB L2 flush runs before every frame on stream A, inside the
    # timed region.
    from paper_2407_02215_gb300 import cbt as CB
    from paper_2407_02215_gb300 import vertices_to_host_async
    gp = CBT(spec.mesh, spec.D, spec.max_depth, device=dev)
    h1 = CB.handles_of([gp])
    sA, sB = torch.cuda.Stream(), torch.cuda.Stream()
    vb = [vbuf, torch.empty_like(vbuf)]
    hv = [host_v, torch.empty(host_v.shape, dtype=host_v.dtype, pin_memory=True)]
    hn = torch.zeros(2, dtype=torch.int32, pin_memory=True)
    hn_np = hn.numpy()  # the same pinned words
    hn_v = [hn[0:1], hn[1:2]]
    K = len(frames)
    packed = [CB.pack_frames([fp], dev, [vb[k % 2]]) for k, fp in enumerate(frames)]
    evA = [torch.cuda.Event() for _ in range(K)]
    evB = [torch.cuda.Event() for _ in range(K)]

    def copy_out(k):
        evA[k].synchronize()
        n = int(hn_np[k % 2])
        sB.wait_event(evA[k])
        vertices_to_host_async(vb[k % 2], hv[k % 2], n, stream=sB)
        evB[k].record(sB)
        return n

    torch.cuda.synchronize()
    barrier(world)
    d2h_p = 0
    t0 = time.perf_counter()
    with torch.cuda.stream(sA):
        for k in range(K):
            if k >= 2:
                sA.wait_event(evB[k - 2])
            flush.zero_()
            CB.update_many_packed(h1, packed[k][0], 1, stream=sA)
            gp.live_count_async(hn_v[k % 2], stream=sA)
            evA[k].record(sA)
            if k >= 1:
                d2h_p += 4 + 36 * copy_out(k - 1)
    d2h_p += 4 + 36 * copy_out(K - 1)
    evB[K - 1].synchronize()
    pipe_t = time.perf_counter() - t0
    final_rows_ok = int(hn_np[(K - 1) % 2]) == stats[-1]["live_after"]
    del gp, vb, hv, packed
    pipe_val = reduce_sum(float(e2e_bis), world) / reduce_max(pipe_t, world)

    if rank != 0:
        return None
    frame_kernel = "k_frame1" if "final" in ptimes else "k_frame"
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    # the dominant (only) kernel of the timed region is the one-launch frame:
    # the frame's algorithmic bytes over its event-timed duration
    ach = fbytes / (float(ms.sum()) / 1e3) / 1e9
    phase_share = {k: round(v / sum(ptimes.values()), 4) for k, v in sorted(ptimes.items(), key=lambda x: -x[1])}
    cfg = workload_config(spec, len(frames))
    cfg["parallelism"] = f"replicas x{world}"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(frames),
        "warmup": args.warmup, "ms_per_step": float(ms.mean()), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64+fp32",
        "data": "synthetic (seeded grid mesh and camera path)", "config": cfg,
        "ms_per_frame_p50": float(np.percentile(ms, 50)), "ms_per_frame_p99": float(np.percentile(ms, 99)),
        "roofline": {"bound": "hbm", "kernel": f"{frame_kernel} (the whole frame, one cooperative launch)",
                     "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "peak_source": "measured" if peaks else "fallback",
                     "algorithmic_bytes_per_frame": fbytes / len(frames),
                     "bytes_model": "N(8+4+12) record read + 4N command + 8N scans + 24A new records + 12U "
                                    "relinks + bitfield read/write + sum tree + 36N' export, from the frame counters",
                     "traffic": frame_traffic(bis / len(frames)),
                     "traffic_note": "ncu DRAM bytes per launch scaled by live count; null if the kernel changed"},
        "per_kernel_bytes": {k: round(v / len(frames)) for k, v in kbytes.items()},
        "per_kernel_bytes_note": "per-step form's kernels, each reading its inputs again (L2 re-reads included)",
        "phase_ms_per_frame": {k: round(v / len(frames), 5) for k, v in ptimes.items()},
        "phase_share": phase_share,
        "phase_times_from": "second pass over the same frames, device timer at the phase boundaries",
        "per_step_form": {"value": bis_all / reduce_max(float(ms_steps.sum()) / 1e3, world),
                          "ms_per_frame": float(ms_steps.mean()),
                          "kernel_ms_per_frame": {k: round(v / len(frames), 5) for k, v in ktimes.items()},
                          "note": "one launch per step, CUDA graph, same frames"},
        "e2e": {"value": pipe_val, "unit": UNIT, "h2d_bytes_per_step": 168,
                "d2h_bytes_per_step": int(d2h_p / len(frames)),
                "how": "every frame: parameters in as launch arguments, its vertex rows and live count out to "
                       "pinned host memory (cbt_live_count_async, cbt_vertices_to_host_async); frame k+1 "
                       "computes while the copy engine moves frame k's rows (two buffers); one library call "
                       "per step, frames packed before the loop; the L2 flush before every frame is inside "
                       "the timed region",
                "last_count_equals_stats": final_rows_ok,
                "sequential_value": e2e_val,
                "sequential_how": "update, then cbt_vertices_to_host (a kernel copying rows and count into "
                                  "pinned memory) under one synchronisation, frame by frame, flush outside",
                "copy_form_value": copy_val},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, frames, args.cpu_budget, [st["live_after"] for st in stats])
    if not args.no_forms and world == 1:
        del g
        line.update(forms_summary(args))
    return line


def forms_summary(args):
    """The batched and served forms beside the plain per-instance launches
    (the 256-instance batch population over 64 frames, equal work, final
    states compared) and the served form's latency at one Poisson rate over
    the 1,032-instance served population."""
    import torch

    from paper_2407_02215_gb300.serving import ServeLoop
    specs4 = W.configs.config4()
    r = forms_compare(specs4, 64, args.hbm_budget_gb)
    batched = {"workload": "256 instances, H log-uniform 24..40k, pools 2^14..2^20, 64 frames",
               "unit": UNIT, "plain": r["plain"]["value"], "batched": r["batched"]["value"],
               "served_saturated": r["served_saturated"]["value"],
               "speedup_batched_vs_plain": r["speedup_batched_vs_plain"],
               "speedup_served_vs_plain": r["speedup_served_vs_plain"],
               "identical_final_states": r["identical_final_states"], "tuned": r["batched"]["tuned"],
               "plain_is": "one cbt_update per instance, one cbt_update_many call per frame"}
    del specs4
    specs5 = W.configs.config5()
    loop = ServeLoop(specs5, hbm_budget_bytes=int(args.hbm_budget_gb * 2**30), inflight=2, max_batch=4096)
    torch.cuda.synchronize()
    loop.run(args.serve_rate, 0.5, seed=99)  # warm-up
    s = loop.run(args.serve_rate, args.serve_seconds, seed=int(args.serve_rate))
    served = {"workload": f"{len(loop.specs)} resident instances (1024 batch-like + 8 planets), "
                          f"{loop.hbm_used / 2**30:.1f} GB of workspaces, Poisson arrivals",
              "rate_hz": args.serve_rate, "seconds": args.serve_seconds, "p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"],
              "requests_per_s": s["requests_per_s"], "bisectors_per_s": s["bisectors_per_s"],
              "mean_batch": s["mean_batch"], "tick_form": "per-step kernels, two overlapping streams"}
    del loop
    torch.cuda.synchronize()
    return {"batched": batched, "served": served}


def bench_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    spec = W.configs.config2()
    frames = frames_for(spec, args.steps)
    warm = frames_for(spec, max(args.warmup, 0))
    run_oracle(spec, warm, 1e9)
    bis, secs, done = run_oracle(spec, frames, args.ref_budget)
    value = bis / secs
    cfg = workload_config(spec, done)
    cfg["parallelism"] = "one host core"
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": done,
        "warmup": args.warmup, "ms_per_step": secs / done * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64+fp32", "impl": "reference",
        "data": "synthetic (seeded grid mesh and camera path)", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"frames 0..{done - 1} of the flythrough, sequential C oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def _final_states(insts):
    """Every instance's whole state: bitfield and sum tree, and the live
    bisectors' slots, heap IDs and links."""
    out = []
    for g in insts:
        bits, sums = g.cbt()
        slots, heap, links = g.leaves()
        out.append((bits, sums[1:], slots, heap, links))  # sums[0] is no node of the tree
    return out


def _same_states(a, b):
    import torch
    return len(a) == len(b) and all(all(torch.equal(x, y) for x, y in zip(sa, sb)) for sa, sb in zip(a, b))


def forms_compare(specs, n_frames, hbm_budget_gb=120.0, serve=True, tune_rounds=2):
    """The plain, batched and served forms on the same instances and frames,
    with equal work: plain = one cbt_update per instance, issued by one
    cbt_update_many call per frame; batched = the autotuned batch form
    (CUDA graph); served = a saturated server with every instance's frames
    queued at the start. Frames are packed beforehand and submitted back to
    back. Each form starts from fresh instances; the final states of every
    instance (bitfield, sum tree, live slots, heap IDs, links) are compared
    with those of a counting pass that reads the live counts per frame."""
    import torch

    from paper_2407_02215_gb300 import CBT, Batch
    from paper_2407_02215_gb300 import cbt as B
    from paper_2407_02215_gb300.serving import ServeLoop
    dev = torch.device("cuda")
    n = len(specs)

    def fresh():
        gs = [CBT(s.mesh, s.D, s.max_depth, device=dev) for s in specs]
        torch.cuda.synchronize()
        return gs

    packed = [B.pack_frames([s.frames[k] for s in specs], dev) for k in range(n_frames)]
    # counting pass: the work (live bisectors at each frame's start) and the reference states
    t0 = time.perf_counter()
    cnt = fresh()
    t_create = time.perf_counter() - t0
    h = B.handles_of(cnt)
    bis = 0
    for k in range(n_frames):
        B.update_many_packed(h, packed[k][0], n)
        bis += sum(g.stats()["live_before"] for g in cnt)
    ref = _final_states(cnt)
    del cnt, h
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(step):
        torch.cuda.synchronize()
        ev0.record()
        for k in range(n_frames):
            step(k)
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3

    plain = fresh()
    h = B.handles_of(plain)
    t_plain = timed(lambda k: B.update_many_packed(h, packed[k][0], n))
    same_plain = _same_states(ref, _final_states(plain))
    del plain, h
    tune = fresh()
    bt = Batch(tune)
    bt.autotune(tune_rounds)
    for k in range(min(n_frames, 10 * tune_rounds + 1)):
        bt.update_packed(packed[k][0])
    torch.cuda.synchronize()
    cfg = bt.config()
    del bt, tune
    gs = fresh()
    batch = Batch(gs)
    if cfg["fused"]:
        batch.set_fused(True)
    else:
        batch.set_config(cfg["tile_words"], cfg["blocks_per_sm"])
    batch.set_graph(True)
    t_batch = timed(lambda k: batch.update_packed(packed[k][0]))
    same_batch = _same_states(ref, _final_states(gs))
    del batch, gs
    out = {"instances": n, "frames": n_frames, "bisectors_per_frame": bis / n_frames,
           "plain": {"value": bis / t_plain, "ms_per_frame": t_plain / n_frames * 1e3,
                     "how": "one cbt_update per instance, one cbt_update_many call per frame"},
           "batched": {"value": bis / t_batch, "ms_per_frame": t_batch / n_frames * 1e3, "tuned": cfg},
           "speedup_batched_vs_plain": t_plain / t_batch, "create_s_per_set": t_create}
    same = same_plain and same_batch
    if serve:
        loop = ServeLoop(specs, hbm_budget_bytes=int(hbm_budget_gb * 2**30), inflight=2, max_batch=4096)
        torch.cuda.synchronize()
        r = loop.run(1.0, 0.0, seed=1, per_instance=n_frames)
        same_serve = len(loop.instances) == n and _same_states(ref, _final_states(loop.instances))
        same = same and same_serve
        out["served_saturated"] = {"value": bis / r["wall_s"], "wall_s": r["wall_s"], "ticks": r["ticks"],
                                   "mean_batch": r["mean_batch"],
                                   "how": "every instance's frames queued at the start; host wall clock"}
        out["speedup_served_vs_plain"] = t_plain / r["wall_s"]
        del loop
    out["identical_final_states"] = same
    out["identical_by_form"] = {"plain": same_plain, "batched": same_batch,
                                **({"served": same_serve} if serve else {})}
    del packed, ref
    torch.cuda.synchronize()
    return out


def bench_batch(args):
    """Batched form (BASELINE config 4: 256 uneven instances, 64 frames)
    against the plain per-instance launches and a saturated server, on the
    same frames, with the final states compared."""
    specs = W.configs.config4(n_inst=args.instances, n_frames=args.frames)
    r = forms_compare(specs, args.frames, args.hbm_budget_gb)
    return {"metric": METRIC + " [batched form]", "value": r["batched"]["value"], "unit": UNIT, **r,
            "config": {"workload": f"batch: {len(specs)} instances, H log-uniform 24..40k, pools 2^14..2^20, "
                                   f"{args.frames} frames"}}


def bench_serve(args):
    """Served form (BASELINE config 5: 1024 batch-like instances and 8
    planets): Poisson arrivals at several rates, p50/p99 latency beside
    throughput, both tick forms; and the plain, batched and saturated-served
    forms on the same population and frames (equal work, states compared)."""
    import torch

    from paper_2407_02215_gb300.serving import ServeLoop
    specs = W.configs.config5(n_inst=args.instances, n_planets=args.planets, n_frames=args.frames)
    rates = [float(r) for r in args.rates.split(",")]
    t0 = time.perf_counter()
    forms = {}
    for name, fused in (("per_step_overlapped_ticks", False), ("fused_serial_ticks", True)):
        loop = ServeLoop(specs, hbm_budget_bytes=int(args.hbm_budget_gb * 2**30), inflight=2, max_batch=4096,
                         fused=fused)
        torch.cuda.synchronize()
        out = []
        loop.run(rates[0], 0.5, seed=99)  # warm-up
        for r in rates:
            out.append(loop.run(r, args.duration, seed=int(r)))
        forms[name] = out
        admitted, rejected, used = len(loop.specs), len(loop.rejected), loop.hbm_used
        del loop
        torch.cuda.synchronize()
    t_rates = time.perf_counter() - t0
    cmp = forms_compare(specs, args.compare_frames, args.hbm_budget_gb)
    return {"metric": "served LOD-update requests: latency and throughput", "unit": "ms / bisectors/s",
            "admitted": admitted, "rejected": rejected,
            "hbm_used_gb": used / 2**30, "rates": forms["per_step_overlapped_ticks"], "forms": forms,
            "same_work_forms": cmp, "rates_wall_s": t_rates,
            "config": {"workload": f"served: {len(specs)} instances ({args.instances} batch-like + "
                                   f"{args.planets} planets), Poisson arrivals {args.duration} s per rate, "
                                   f"HBM budget {args.hbm_budget_gb} GB; same-work forms over "
                                   f"{args.compare_frames} frames"}}


def bench_reduce(args):
    """SumReduction (Sec. 3.1) alone, and with CachePointers (Alg. 7 for every
    index), at 2^27 slots, the size at which the paper times the prior
    method's reduction (0.4 ms on its GPU; context, not a ratio): a seeded
    random bitfield of 16 MB in, the 32 MB sum tree out, then the 256 MB live
    list; L2 flushed before every timed run."""
    import torch

    from paper_2407_02215_gb300 import compact, sum_reduce
    D = 27
    W = 1 << (D - 5)
    g = torch.Generator(device="cuda").manual_seed(27)
    bits = torch.randint(-2**31, 2**31 - 1, (W,), dtype=torch.int32, device="cuda", generator=g)
    sums = torch.zeros(2 * W, dtype=torch.int32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        sum_reduce(bits, D, sums)
    torch.cuda.synchronize()
    n = int(sums[1].item())
    live = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(max(args.warmup, 3)):
        compact(bits, sums, D, live)
    reps = 50

    def timed(fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for a, b in ev:
            flush.zero_()
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        return np.array([a.elapsed_time(b) for a, b in ev]) * 1e3

    us = timed(lambda: sum_reduce(bits, D, sums))
    us_c = timed(lambda: compact(bits, sums, D, live))
    us_rc = timed(lambda: (sum_reduce(bits, D, sums), compact(bits, sums, D, live)))
    # reduction: the bitfield is read once, every node of the tree (2W words)
    # written once; compaction: the bitfield read, 4 bytes per set bit written
    alg = 4.0 * W + 8.0 * W
    alg_c = 4.0 * W + 4.0 * n
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    gbs = alg / (us.mean() / 1e6) / 1e9
    gbs_c = alg_c / (us_c.mean() / 1e6) / 1e9
    root = int(sums[1].item())
    host = bits.cpu().numpy().view(np.uint32)
    want = int(np.unpackbits(host.view(np.uint8)).sum())
    lv = live.cpu().numpy().view(np.uint32).astype(np.int64)
    ok = bool(lv.size == want and np.all(np.diff(lv) > 0) and np.all((host[lv >> 5] >> (lv & 31).astype(np.uint32)) & 1))
    return {"metric": "CBT sum reduction over 2^27 slots (Sec. 3.1), us per reduction", "unit": "us",
            "value": float(us.mean()), "p50": float(np.median(us)), "p99": float(np.percentile(us, 99)),
            "higher_is_better": False,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "algorithmic_bytes": alg, "peak_source": "measured" if peaks else "fallback"},
            "root": root, "root_equals_popcount": root == want,
            "compaction": {"us_mean": float(us_c.mean()), "us_p50": float(np.median(us_c)),
                           "us_p99": float(np.percentile(us_c, 99)), "live": n,
                           "roofline": {"bound": "hbm", "achieved": gbs_c, "peak": peak, "unit": "GB/s",
                                        "frac": gbs_c / peak, "algorithmic_bytes": alg_c},
                           "live_list_valid": ok},
            "reduce_plus_compact": {"us_mean": float(us_rc.mean()), "us_p50": float(np.median(us_rc)),
                                    "us_p99": float(np.percentile(us_rc, 99))},
            "paper": {"value_us": 400.0, "what": "original implicit CBT sum reduction at 2^27 on an AMD 6800 XT",
                      "cite": "Sec. 4 (reduction cost of the prior method)"},
            "config": {"workload": "reduce: random bitfield (seeded), 2^27 slots, L2 flushed before every run",
                       "reps": reps}}


def _frames_timed(args, spec, vertices=True, busy_min=1000, point_cache=False):
    """One instance over its frames as a CUDA graph, L2 flushed before every
    frame, vertices exported every frame (with ``point_cache``, the sphere
    form's point cache attached): per-frame event times, live counts, and a
    device-timer phase breakdown (second run) of the frames with more than
    busy_min live bisectors."""
    import torch

    from paper_2407_02215_gb300 import CBT
    vbuf = torch.empty((1 << spec.D, 3, 3), dtype=torch.float32, device="cuda") if vertices else None
    g0 = CBT(spec.mesh, spec.D, spec.max_depth, point_cache=point_cache)
    for fp in spec.frames[:max(args.warmup, 3)]:
        g0.update(fp, vertices_out=vbuf)
    del g0
    g = CBT(spec.mesh, spec.D, spec.max_depth, point_cache=point_cache)
    g.set_graph(True)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in spec.frames]
    live = []
    for k, fp in enumerate(spec.frames):
        flush.zero_()
        ev[k][0].record()
        g.update(fp, vertices_out=vbuf)
        ev[k][1].record()
        live.append(g.stats()["live_before"])
    torch.cuda.synchronize()
    ms = np.array([a.elapsed_time(b) for a, b in ev])
    live = np.array(live)
    busy = live > busy_min
    gk = CBT(spec.mesh, spec.D, spec.max_depth, point_cache=point_cache)
    gk.set_timing(True)
    pt, nb = {}, 0
    for k, fp in enumerate(spec.frames):
        flush.zero_()
        gk.update(fp, vertices_out=vbuf)
        if busy[k]:
            nb += 1
            for name, v in gk.kernel_times().items():
                pt[name] = pt.get(name, 0.0) + v
    del gk
    return {"value": float(live.sum() / (ms.sum() / 1e3)), "unit": UNIT, "ms_per_frame_mean": float(ms.mean()),
            "ms_per_frame_p50": float(np.median(ms)), "ms_per_frame_p99": float(np.percentile(ms, 99)),
            "ms_per_frame_p50_in_view": float(np.median(ms[busy])) if busy.any() else None,
            "live_p50_in_view": float(np.median(live[busy])) if busy.any() else None, "live_max": int(live.max()),
            "phase_ms_per_frame_in_view": {k: round(v / max(nb, 1), 5) for k, v in pt.items()}}


def bench_dodeca(args):
    """The paper's planet scene shape (Sec. 4, Table 3: H = 60, D = 17, 0.1 ms
    per update on its GPU): dodecahedron base on an Earth-sized sphere,
    vertices projected onto the sphere in FP64, 14 px refinement edges, a
    300-frame descent from 2e7 m to 2 m; one instance, CUDA graph, vertices
    exported every frame, L2 flushed before every frame."""
    spec = W.configs.config_dodeca()
    out = {"metric": METRIC + " [paper's planet shape]", **_frames_timed(args, spec, point_cache=True)}
    out.update({"paper": {"ms_per_update": 0.1,
                          "what": "Table 3, water planet (H 60, D 17), AMD 6800 XT, FP64 vertex decode"},
                "config": {"workload": "dodeca planet: dodecahedron (60 halfedges), R 6.371e6 m, pool 2^17, "
                                       "max depth 50, 300-frame descent 2e7 m -> 2 m, sphere projection in FP64, "
                                       "14 px edges, point cache attached, L2 flushed before every frame",
                           "frames": len(spec.frames)}})
    return out


def bench_waves(args):
    """The paper's water planet (Sec. 4): the dodecahedron planet of the
    dodeca workload with the projected vertices displaced radially by a
    4-octave value noise (2 m, cells of 1 km to 125 m) standing in for its
    four FFT wave layers; the same descent, timing and export."""
    spec = W.configs.config_waves()
    out = {"metric": METRIC + " [water planet, displaced]", **_frames_timed(args, spec, point_cache=True)}
    out.update({"paper": {"ms_per_update": 0.1,
                          "what": "Table 3, water planet (H 60, D 17), AMD 6800 XT, FP64 vertex decode"},
                "config": {"workload": "wave planet: dodeca planet + radial displacement 2 m x fbm(4 octaves, "
                                       "1 km .. 125 m cells), pool 2^17, 300-frame descent, point cache attached, "
                                       "L2 flushed before every frame", "frames": len(spec.frames)}})
    return out


def bench_terrain(args):
    """Displaced terrain (the grid flythrough with z displaced by a 6-octave
    value noise, 0.02 amplitude, 4 to 128 cells per unit) beside the same
    flythrough undisplaced: what the noise evaluation adds to classify."""
    spec = W.configs.config_terrain()
    flat = W.configs.config2()
    out = {"metric": METRIC + " [displaced terrain]", **_frames_timed(args, spec)}
    ref = _frames_timed(args, flat)
    out.update({"undisplaced": {k: ref[k] for k in ("value", "ms_per_frame_p50", "live_p50_in_view",
                                                     "phase_ms_per_frame_in_view")},
                "config": {"workload": "terrain: 100 x 100 mixed grid (42k halfedges), pool 2^20, max depth 26, "
                                       "120-frame flythrough, tau 2 px, z displaced by 0.02 x fbm(6 octaves, 4 .. 128 "
                                       "cells per unit), vertices exported, L2 flushed before every frame",
                           "frames": len(spec.frames)}})
    return out


def bench_index(args):
    """Indexed export (cbt_index: deduplicated vertex buffer, index buffer and
    triangle heap IDs for a visibility buffer) after every frame of the grid
    flythrough; the export is timed alone (CUDA events around the call, which
    returns the counts)."""
    import torch

    from paper_2407_02215_gb300 import CBT
    spec = W.configs.config2()
    g = CBT(spec.mesh, spec.D, spec.max_depth)
    vbuf = torch.empty((1 << spec.D, 3, 3), dtype=torch.float32, device="cuda")
    cap = 1 << spec.D
    ws = g.index_workspace(cap)
    out = (torch.empty((3 * cap, 3), dtype=torch.float32, device="cuda"),
           torch.empty((cap, 3), dtype=torch.int32, device="cuda"), torch.empty(cap, dtype=torch.int64, device="cuda"))
    ms, tris, verts = [], [], []
    for k, fp in enumerate(spec.frames):
        g.update(fp, vertices_out=vbuf)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        v, idx, _ = g.index(vbuf, workspace=ws, out=out)
        b.record()
        torch.cuda.synchronize()
        n = idx.shape[0]
        if k >= max(args.warmup, 3):
            ms.append(a.elapsed_time(b))
            tris.append(n)
            verts.append(v.shape[0])
    ms, tris = np.array(ms), np.array(tris)
    return {"metric": "indexed export (vertex + index buffers), triangles/s", "unit": "triangles/s",
            "value": float(tris.sum() / (ms.sum() / 1e3)), "ms_p50": float(np.median(ms)),
            "ms_p99": float(np.percentile(ms, 99)), "triangles_p50": float(np.median(tris)),
            "vertices_per_triangle": float(np.sum(verts) / tris.sum()),
            "config": {"workload": "grid flythrough (100 x 100, pool 2^20, 120 frames): cbt_index after every "
                                   "update, inputs resident", "frames_timed": int(ms.size)}}


def _near_reference(heap, rows, ch, roots, radius_m, eye, project=None):
    """FP64 vertices, relative to the eye, of the given rows whose heap IDs
    have a vertex within radius_m of the eye: the oracle's exact integer
    weights over 2^d times its FP64 root table (absolute), optionally moved
    by `project` (absolute FP64 points [3, 3] -> points)."""
    from oracle.oracle import decode_weights
    out_rows, out_v = [], []
    for r in rows:
        j = int(heap[r])
        d = j.bit_length() - 1 - ch
        h = (j >> d) - (1 << ch)
        p = (decode_weights(j, ch).astype(np.float64) / float(2 ** d)) @ roots[h]
        if project is not None:
            p = project(p)
        v = p - eye[None, :]
        if np.sqrt((v * v).sum(axis=1)).min() <= radius_m:
            out_rows.append(r)
            out_v.append(v)
    return np.array(out_rows, np.int64), (np.stack(out_v) if out_v else np.zeros((0, 3, 3)))


def bench_precision(args):
    """Vertex error near the eye at the end of the planet descents, in mm,
    against FP64 evaluations of the oracle's exact weights (Sec. 4: FP64
    for planets; R10 fixed point; R13 sphere projection): the cube-sphere
    descent (pool 2^22, 600 frames) in its fixed-point, FP64 and FP32 forms,
    and the dodecahedron planet without and with its wave displacement (the
    sphere form), within 100 m of the final eye (2 m above the surface)."""
    import torch

    from oracle import Oracle
    from oracle import oracle as O
    from paper_2407_02215_gb300 import CBT
    out = {"metric": "vertex error near the eye at planet scale (max, mm)", "unit": "mm",
           "radius_m": 100.0, "reference": "FP64 of the oracle's exact integer weights and FP64 roots"}
    spec = W.configs.config3(n_frames=600)
    g = CBT(spec.mesh, spec.D, spec.max_depth)
    for fp in spec.frames:
        g.update(fp)
    eye = np.asarray(spec.frames[-1].eye, np.float64)
    o = Oracle(spec.mesh, 12, spec.max_depth)
    _, heap, _ = g.leaves()
    heap = heap.cpu().numpy().view(np.uint64)
    vf = g.vertices(eye, 1, 20).cpu().numpy().astype(np.float64)
    dist = np.sqrt((vf * vf).sum(axis=2)).min(axis=1)
    cand = np.flatnonzero(dist <= 101.0)
    order = cand[np.argsort(dist[cand], kind="stable")]
    cand = np.unique(np.concatenate([order[:10000], order[10000::max(1, (order.size - 10000) // 10000)]]))
    rows, ref = _near_reference(heap, cand, o.ch, o.root_table(), 100.0, eye)
    c3 = {"workload": "cube-sphere 1536 halfedges, R 6.371e6 m, pool 2^22, max depth 48, 600-frame descent to 2 m",
          "live": int(heap.size), "within_100m": int((dist <= 100.0).sum()), "sampled": int(rows.size),
          "sample": "the 10,000 nearest and 10,000 spread over the rest",
          "nearest_m": float(np.sqrt((ref * ref).sum(axis=2)).min()) if rows.size else None}
    for name, prec in (("fixed", 1), ("fp64", 2), ("fp32", 0)):
        v = g.vertices(eye, prec, 20).cpu().numpy().astype(np.float64)[rows]
        c3[name + "_max_mm"] = float(np.abs(v - ref).max() * 1e3) if rows.size else None
    out["planet_cube_sphere"] = c3
    del g
    for key, spec in (("dodeca", W.configs.config_dodeca()), ("waves", W.configs.config_waves())):
        g = CBT(spec.mesh, spec.D, spec.max_depth, point_cache=True)
        vbuf = torch.empty((1 << spec.D, 3, 3), dtype=torch.float32, device="cuda")
        for fp in spec.frames:
            g.update(fp, vertices_out=vbuf)
        torch.cuda.synchronize()
        last = spec.frames[-1]
        eye = np.asarray(last.eye, np.float64)
        R = float(last.sphere_radius)
        n = g.live_count()
        vg = vbuf[:n].cpu().numpy().astype(np.float64)
        _, heap, _ = g.leaves()
        heap = heap.cpu().numpy().view(np.uint64)
        o = Oracle(spec.mesh, 8, spec.max_depth)

        def project(p, fp=last):
            nrm = np.sqrt((p * p).sum(axis=1))
            rad = np.full(3, R)
            if fp.disp_amplitude:
                for k in range(3):
                    u = (p[k] / nrm[k]).astype(np.float32)
                    hgt = np.float32(fp.disp_amplitude) * np.float32(
                        O.fbm(u, fp.disp_frequency, fp.disp_octaves, fp.disp_seed))
                    rad[k] = R + float(hgt)
            return p * (rad / nrm)[:, None]

        # the pool saturates short of the eye: the 5,000 nearest bisectors
        dist = np.sqrt((vg * vg).sum(axis=2)).min(axis=1)
        cand = np.argsort(dist, kind="stable")[:5000]
        rows, ref = _near_reference(heap, cand, o.ch, o.root_table(), 1e30, eye, project)
        e = np.abs(vg[rows] - ref)
        dref = np.sqrt((ref * ref).sum(axis=2)).min(axis=1)
        out[key] = {"workload": f"{spec.name}: dodecahedron planet, pool 2^{spec.D}, "
                                f"{len(spec.frames)}-frame descent to 2 m, sphere form (FP64 projection)"
                                + (", 2 m wave displacement" if last.disp_amplitude else ""),
                    "live": int(n), "sampled": int(rows.size), "sample": "the 5,000 bisectors nearest the eye",
                    "sphere_max_mm": float(e.max() * 1e3),
                    "distance_m": [float(dref.min()), float(dref.max())]}
        del g, vbuf
    return out


def bench_planet(args):
    """Planet descent (pool 2^22, max depth 48, fixed point): frame times."""
    import torch

    from paper_2407_02215_gb300 import CBT
    spec = W.configs.config3(n_frames=600)
    g = CBT(spec.mesh, spec.D, spec.max_depth)
    vbuf = torch.empty((1 << spec.D, 3, 3), dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in spec.frames]
    bis = 0
    for k, fp in enumerate(spec.frames):
        ev[k][0].record()
        g.update(fp, vertices_out=vbuf)
        ev[k][1].record()
        bis += g.stats()["live_before"]
    torch.cuda.synchronize()
    ms = np.array([a.elapsed_time(b) for a, b in ev])
    return {"metric": METRIC + " [planet]", "value": bis / (ms.sum() / 1e3), "unit": UNIT,
            "ms_per_frame_p50": float(np.percentile(ms, 50)), "ms_per_frame_p99": float(np.percentile(ms, 99)),
            "final_live": g.live_count(),
            "config": {"workload": "planet: cube-sphere 1536 halfedges, R 6.371e6 m, pool 2^22, max depth 48, "
                                   "600-frame descent 2e7 m -> 2 m, fixed-point vertices, L2 not flushed"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=150.0)
    ap.add_argument("--workload", default="grid",
                    choices=["grid", "batch", "serve", "planet", "reduce", "dodeca", "waves", "terrain", "index",
                             "precision"],
                    help="grid = the headline workload; the others are extra measurements")
    ap.add_argument("--instances", type=int, default=None,
                    help="batch: 256 (config 4); serve: 1024 batch-like instances (config 5)")
    ap.add_argument("--planets", type=int, default=8)
    ap.add_argument("--frames", type=int, default=64)
    ap.add_argument("--compare-frames", type=int, default=16)
    ap.add_argument("--rates", default="2000,5000,10000,20000")
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--hbm-budget-gb", type=float, default=120.0)
    ap.add_argument("--no-forms", action="store_true",
                    help="grid line without the batched and served objects")
    ap.add_argument("--serve-rate", type=float, default=10000.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.instances is None:
        args.instances = 1024 if args.workload == "serve" else 256
    if args.workload != "grid":
        import paper_2407_02215_gb300 as P
        P.build_library()
        fn = {"batch": bench_batch, "serve": bench_serve, "planet": bench_planet,
              "reduce": bench_reduce, "dodeca": bench_dodeca, "waves": bench_waves,
              "terrain": bench_terrain, "index": bench_index, "precision": bench_precision}[args.workload]
        print(json.dumps(fn(args)))
        return
    if args.impl == "reference":
        line = bench_reference(args)
    else:
        import paper_2407_02215_gb300 as P
        P.build_library()
        line = bench_ours(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()

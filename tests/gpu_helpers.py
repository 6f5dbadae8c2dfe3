"""Helpers for the GPU parity tests: run the CUDA library and the CPU oracle
on the same inputs and compare their states element by element."""
from __future__ import annotations

import numpy as np


def gpu_state(g):
    slots, heap, links = g.leaves()
    bits, sums = g.cbt()
    return {
        "slots": slots.cpu().numpy().astype(np.uint32),
        "heap": heap.cpu().numpy().astype(np.uint64),
        "links": links.cpu().numpy().astype(np.uint32),
        "bits": bits.cpu().numpy().astype(np.uint32),
        "sums": sums.cpu().numpy().astype(np.uint32),
    }


def oracle_state(o):
    slots, heap, links = o.leaves()
    cbt = o.export()["cbt"]
    cap = o.cap
    W = max(1, cap // 32)
    leaf = cbt[cap:]
    padded = np.zeros(32 * W, np.uint64)
    padded[:cap] = leaf
    bits = (padded.reshape(W, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    sums = np.zeros(2 * W, np.uint32)
    sums[1:] = cbt[1:2 * W]
    return {"slots": slots, "heap": heap, "links": links, "bits": bits, "sums": sums}


def assert_same_state(g, o, where=""):
    a, b = gpu_state(g), oracle_state(o)
    assert a["slots"].shape == b["slots"].shape, f"{where}: live count {a['slots'].size} vs {b['slots'].size}"
    for k in ("slots", "heap", "links", "bits"):
        if not np.array_equal(a[k], b[k]):
            bad = np.nonzero(a[k].reshape(a[k].shape[0], -1) != b[k].reshape(b[k].shape[0], -1))[0]
            raise AssertionError(f"{where}: {k} differs at {bad[:10].tolist()} "
                                 f"(gpu {a[k][bad[:3]].tolist()} oracle {b[k][bad[:3]].tolist()})")
    assert np.array_equal(a["sums"][1:], b["sums"][1:]), f"{where}: CBT sums differ"


def run_pair(spec_mesh, D, max_depth, frames, CBT, Oracle, check_every=1, stats_keys=(
        "live_after", "split_granted", "merge_granted", "split_bisectors", "merged_bisectors",
        "merge_groups", "allocated")):
    g = CBT(spec_mesh, D, max_depth)
    o = Oracle(spec_mesh, D, max_depth)
    assert_same_state(g, o, "create")
    for k, fp in enumerate(frames):
        g.update(fp)
        so = o.update(fp)
        sg = g.stats()
        assert sg["error"] == 0, f"frame {k}: device error {sg['error']:#x}"
        assert so["ab_mismatch"] == 0
        for key in stats_keys:
            assert sg[key] == so[key], f"frame {k}: {key} gpu {sg[key]} oracle {so[key]}"
        if (k + 1) % check_every == 0 or k == len(frames) - 1:
            assert_same_state(g, o, f"frame {k}")
    return g, o

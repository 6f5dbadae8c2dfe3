"""Writes tests/golden/planet_oracle.json from the CPU oracle alone.

The planet workload (cube-sphere, 1536 halfedges, radius 6.371e6 m, pool
2^22, max depth 48, 600-frame descent from 2e7 m to 2 m, fixed-point vertex
evaluation) takes the oracle tens of minutes, so its results are stored: the
live count after every frame and, every 50 frames and at the end, a SHA-256
digest of the live slots, heap IDs, links and CBT bitfield, plus a digest of
the final vertices (fixed point, relative to the last eye).

Digest input, little-endian: slots u32[N], heap u64[N], links u32[N][3]
(Twin, Next, Prev), bitfield u32[max(1, 2^D / 32)] (bit s % 32 of word s / 32
is slot s); vertices f32[N][3][3].
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import Oracle  # noqa: E402


def state_digest(slots, heap, links, bits):
    h = hashlib.sha256()
    for a, dt in ((slots, "<u4"), (heap, "<u8"), (links, "<u4"), (bits, "<u4")):
        h.update(np.ascontiguousarray(a).astype(dt).tobytes())
    return h.hexdigest()


def oracle_bits(o):
    cbt = o.export()["cbt"]
    cap = o.cap
    W_ = max(1, cap // 32)
    padded = np.zeros(32 * W_, np.uint64)
    padded[:cap] = cbt[cap:]
    return (padded.reshape(W_, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)


def main(out=os.path.join(HERE, "planet_oracle.json"), n_frames=600, D=22):
    spec = W.configs.config3(n_frames=n_frames, D=D)
    o = Oracle(spec.mesh, spec.D, spec.max_depth)
    live, digests, t0 = [], {}, time.time()
    for k, fp in enumerate(spec.frames):
        st = o.update(fp)
        assert st["ab_mismatch"] == 0
        live.append(st["live_after"])
        if k % 50 == 49 or k == n_frames - 1:
            s, j, l = o.leaves()
            digests[str(k)] = state_digest(s, j, l, oracle_bits(o))
            print(k, st["live_after"], f"{time.time() - t0:.0f}s", flush=True)
    last = spec.frames[-1]
    v = o.vertices(last.eye, last.precision, last.fixed_shift)
    res = {"source": "CPU oracle (oracle/cbt_oracle.c) on the planet workload; written by "
                     "tests/golden/make_planet_golden.py",
           "D": spec.D, "max_depth": spec.max_depth, "frames": n_frames,
           "live_after": live, "state_digest": digests,
           "vertices_digest": hashlib.sha256(np.ascontiguousarray(v, "<f4").tobytes()).hexdigest()}
    with open(out, "w") as f:
        json.dump(res, f)


if __name__ == "__main__":
    main()

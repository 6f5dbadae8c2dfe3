"""Writes tests/golden/batch_oracle.json from the CPU oracle alone.

The batched workload (256 independent instances, H log-uniform over 24..40k
halfedges, pools 2^14..2^20, 64 frames of their own camera paths) is 1.5e9
bisector updates for the sequential oracle, so its results are stored: per
instance the live count after every frame, and SHA-256 digests of the state
after frames 31 and 63. The instances run in separate processes.

Digest input, little-endian: slots u32[N], heap u64[N], links u32[N][3]
(Twin, Next, Prev), bitfield u32[max(1, 2^D / 32)] (bit s % 32 of word s / 32
is slot s).
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

N_INST, N_FRAMES, CHECK = 256, 64, (31, 63)


def one(b):
    import workloads as W
    from oracle import Oracle
    from make_planet_golden import oracle_bits, state_digest
    spec = W.configs.config4(n_inst=N_INST, n_frames=N_FRAMES)[b]
    o = Oracle(spec.mesh, spec.D, spec.max_depth)
    live, dig = [], {}
    for k, fp in enumerate(spec.frames[:N_FRAMES]):
        st = o.update(fp)
        assert st["ab_mismatch"] == 0
        live.append(st["live_after"])
        if k in CHECK:
            s, j, l = o.leaves()
            dig[str(k)] = state_digest(s, j, l, oracle_bits(o))
    return b, {"name": spec.name, "H": spec.mesh.H, "D": spec.D, "live_after": live, "state_digest": dig}


def main(out=os.path.join(HERE, "batch_oracle.json"), workers=None):
    t0 = time.time()
    res = [None] * N_INST
    with mp.get_context("spawn").Pool(workers or os.cpu_count(), initializer=sys.path.insert,
                                      initargs=(0, HERE)) as pool:
        for b, r in pool.imap_unordered(one, range(N_INST)):
            res[b] = r
            print(b, r["name"], r["live_after"][-1], f"{time.time() - t0:.0f}s", flush=True)
    doc = {"source": "CPU oracle (oracle/cbt_oracle.c) on the batched workload; written by "
                     "tests/golden/make_batch_golden.py",
           "instances": N_INST, "frames": N_FRAMES, "checked_frames": list(CHECK), "per_instance": res}
    with open(out, "w") as f:
        json.dump(doc, f)


if __name__ == "__main__":
    main()

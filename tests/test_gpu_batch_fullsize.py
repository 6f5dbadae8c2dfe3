"""Full-size parity of the batched form on its own workload: 256 independent
instances (H log-uniform over 24..40k halfedges, pools 2^14..2^20), 64
frames, updated together by the batch in its one-launch form and in its
per-step form. Every instance's live count after every frame, and its whole
state (live slots, heap IDs, links, bitfield) after frames 31 and 63, equal
the CPU oracle's stored results (tests/golden/make_batch_golden.py)."""
import hashlib
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "batch_oracle.json")


def _digest(g):
    """Same byte layout as tests/golden/make_batch_golden.py."""
    slots, heap, links = g.leaves()
    bits, _ = g.cbt()
    h = hashlib.sha256()
    for t, dt in ((slots, "<u4"), (heap, "<u8"), (links, "<u4"), (bits, "<u4")):
        h.update(np.ascontiguousarray(t.cpu().numpy()).view(dt).tobytes())
    return h.hexdigest()


@pytest.mark.parametrize("fused", [True, False], ids=["one_launch", "per_step"])
def test_batch_population_against_stored_oracle(fused):
    if not os.path.exists(GOLD):
        pytest.skip("batch_oracle.json not generated")
    import paper_2407_02215_gb300 as P
    P.build_library()
    gold = json.load(open(GOLD))
    specs = W.configs.config4(n_inst=gold["instances"], n_frames=gold["frames"])
    gs = [P.CBT(s.mesh, s.D, s.max_depth) for s in specs]
    bt = P.Batch(gs)
    bt.set_fused(fused)
    for k in range(gold["frames"]):
        bt.update([s.frames[k] for s in specs])
        for b, g in enumerate(gs):
            ref = gold["per_instance"][b]
            assert g.live_count() == ref["live_after"][k], f"instance {b} ({ref['name']}) frame {k}"
        if str(k) in gold["per_instance"][0]["state_digest"]:
            for b, g in enumerate(gs):
                assert g.stats()["error"] == 0
                assert _digest(g) == gold["per_instance"][b]["state_digest"][str(k)], f"instance {b} frame {k}"

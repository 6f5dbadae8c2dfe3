"""Full-size parity on the benchmark workload: the 100 x 100 grid (42,034
halfedges, pool 2^20, max depth 26) over its whole 120-frame flythrough,
in the launch configuration bench.py times (fused vertex export included).
Every frame's counters and live count match the oracle; the full state
(slots, heap IDs, links, bitfield, sums) and the exported vertices are
compared bit-exactly every 10 frames."""
import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from tests.gpu_helpers import assert_same_state

pytestmark = pytest.mark.gpu


def test_grid_flythrough_full_size():
    import torch

    import paper_2407_02215_gb300 as P
    P.build_library()
    spec = W.configs.config2()
    g = P.CBT(spec.mesh, spec.D, spec.max_depth)
    o = Oracle(spec.mesh, spec.D, spec.max_depth)
    vbuf = torch.empty((1 << spec.D, 3, 3), dtype=torch.float32, device="cuda")
    keys = ("live_before", "live_after", "split_wishes", "merge_candidates", "split_granted",
            "merge_granted", "split_bisectors", "merged_bisectors", "merge_groups", "allocated")
    for k, fp in enumerate(spec.frames):
        g.update(fp, vertices_out=vbuf)
        so = o.update(fp)
        sg = g.stats()
        assert sg["error"] == 0
        assert so["ab_mismatch"] == 0
        for key in keys:
            assert sg[key] == so[key], f"frame {k}: {key} gpu {sg[key]} oracle {so[key]}"
        if k % 10 == 9:
            assert_same_state(g, o, f"frame {k}")
            n = so["live_after"]
            vo = o.vertices(fp.eye, fp.precision, fp.fixed_shift)
            vg = vbuf[:n].cpu().numpy()
            assert np.array_equal(vg.view(np.uint32), vo.view(np.uint32)), f"frame {k}: vertices"

"""The C ABI: the library loads and exports every entry point declared in
include/cbt.h; host-only entry points behave as documented (no GPU needed)."""
import ctypes
import os
import re

import numpy as np

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "cbt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cbt_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol():
    import paper_2407_02215_gb300 as P
    path = P.build_library()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(lib, s), s


def test_workspace_bytes_and_errors():
    import paper_2407_02215_gb300 as P
    P.build_library()
    assert P.workspace_bytes(24, 16) > 0
    assert P.workspace_bytes(2, 16) == 0       # H < 3
    assert P.workspace_bytes(24, 4) == 0       # 2^D < H
    assert P.workspace_bytes(24, 31) == 0      # D > 30
    # the indexed export's scratch needs a state (its pool and global points)
    assert P.load().cbt_index_workspace_bytes(None, 100) == 0


def test_host_ingest_matches_paper_table():
    """The library's own faces -> halfedges ingest reproduces Fig. 1."""
    import json
    import paper_2407_02215_gb300 as P
    P.build_library()
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "fig1_halfedges.json")))
    he = P.halfedges_from_faces(W.meshes.fig1_mesh())
    for k in ("twin", "next", "prev", "vert", "face"):
        assert he[k].tolist() == g[k]


def test_host_ingest_rejects_bad_faces():
    import paper_2407_02215_gb300 as P
    P.build_library()

    class M:
        face_sizes = np.array([3, 3], np.int32)
        face_verts = np.array([0, 1, 2, 0, 1, 2], np.int32)   # same edge twice, same direction
    try:
        P.halfedges_from_faces(M)
    except P.CBTError as e:
        assert e.code == 1
    else:
        raise AssertionError("expected CBT_EINVAL")


def _c_layout(struct: str, fields):
    """Offsets of `fields` and the size of `struct` as a C compiler lays out
    include/cbt.h (gcc on this host)."""
    import subprocess
    import tempfile
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cbt.h"', "int main(void) {",
             f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    return int(out[0]), [int(x) for x in out[1:]]


def test_binding_structs_match_the_header():
    """The ctypes mirrors of cbt_frame and cbt_frame_stats have the header's
    field offsets and sizes, so frames and counters cross the ABI intact."""
    from paper_2407_02215_gb300.cbt import Frame, Stats
    for cls, name in ((Frame, "cbt_frame"), (Stats, "cbt_frame_stats")):
        fields = [f for f, _ in cls._fields_]
        size, offs = _c_layout(name, fields)
        assert size == ctypes.sizeof(cls), name
        assert offs == [getattr(cls, f).offset for f in fields], name


def test_oracle_binding_structs_match_its_header():
    """The same for the oracle's or_frame (test infrastructure)."""
    import subprocess
    import tempfile
    from oracle.oracle import _Frame
    fields = [f for f, _ in _Frame._fields_]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cbt_oracle.h"', "int main(void) {",
             '  printf("%zu\\n", sizeof(or_frame));']
    lines += [f'  printf("%zu\\n", offsetof(or_frame, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines))
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "oracle"), src, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).decode().split()]
    assert out[0] == ctypes.sizeof(_Frame)
    assert out[1:] == [getattr(_Frame, f).offset for f in fields]

"""ctypes front end of the CPU oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.or_halfedges_from_faces.argtypes = [C.c_int32, P, P, C.c_int32, P, P, P, P, P]
        lib.or_create.argtypes = [C.c_int32, P, P, P, P, P, C.c_int32, P, C.c_int32, C.c_int32,
                                  C.POINTER(C.c_void_p)]
        lib.or_destroy.argtypes = [P]
        lib.or_update.argtypes = [P, P, P]
        lib.or_live_count.argtypes = [P]
        lib.or_live_count.restype = C.c_uint32
        lib.or_ceil_log2_H.argtypes = [P]
        lib.or_export.argtypes = [P, P, P, P, P, P]
        lib.or_leaves.argtypes = [P, P, P, P]
        lib.or_leaves.restype = C.c_uint32
        lib.or_vertices.argtypes = [P, P, C.c_uint32, C.c_int32, C.c_double, P, P]
        lib.or_vertices_f64.argtypes = [P, P]
        lib.or_export_indexed.argtypes = [P, P, P, P, P, C.POINTER(C.c_uint32)]
        lib.or_root_table.argtypes = [P, P]
        lib.or_set_order_seed.argtypes = [P, C.c_uint64]
        lib.or_chain_cost.argtypes = [P, C.c_uint32, C.POINTER(C.c_uint32)]
        lib.or_cbt_sum_reduction.argtypes = [C.c_int32, P]
        lib.or_cbt_one_to_bit.argtypes = [C.c_int32, P, C.c_uint32]
        lib.or_cbt_one_to_bit.restype = C.c_uint32
        lib.or_cbt_compact.argtypes = [C.c_int32, P, P]
        lib.or_cbt_zero_to_bit.argtypes = [C.c_int32, P, C.c_uint32]
        lib.or_cbt_zero_to_bit.restype = C.c_uint32
        lib.or_decode_weights.argtypes = [C.c_uint64, C.c_int32, P]
        lib.or_splitmix64.argtypes = [C.c_uint64]
        lib.or_splitmix64.restype = C.c_uint64
        lib.or_lod_test.argtypes = [P, P, C.c_uint32, C.c_float]
        lib.or_lod_test.restype = C.c_uint32
        lib.or_lowbias32.argtypes = [C.c_uint32]
        lib.or_lowbias32.restype = C.c_uint32
        lib.or_fbm.argtypes = [P, C.c_int32, C.c_float, C.c_uint32, C.c_uint32]
        lib.or_fbm.restype = C.c_float
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


class _Disp(C.Structure):
    _fields_ = [("amplitude", C.c_float), ("frequency", C.c_float), ("octaves", C.c_uint32), ("seed", C.c_uint32)]


def _disp(fp):
    d = _Disp()
    d.amplitude = float(getattr(fp, "disp_amplitude", 0.0))
    d.frequency = float(getattr(fp, "disp_frequency", 0.0))
    d.octaves = int(getattr(fp, "disp_octaves", 0))
    d.seed = int(getattr(fp, "disp_seed", 0))
    return d


class _Frame(C.Structure):
    _fields_ = [
        ("eye", C.c_double * 3),
        ("planes", C.c_float * 15),
        ("q", C.c_float),
        ("nplanes", C.c_uint32),
        ("mode", C.c_uint32),
        ("seed", C.c_uint32),
        ("precision", C.c_uint32),
        ("fixed_shift", C.c_int32),
        ("gate", C.c_uint32),
        ("split_list", C.c_void_p),
        ("n_split", C.c_uint32),
        ("merge_list", C.c_void_p),
        ("n_merge", C.c_uint32),
        ("sphere_radius", C.c_double),
        ("disp", _Disp),
    ]


STAT_FIELDS = ["live_before", "live_after", "free_before", "split_wishes", "merge_candidates",
               "split_granted", "merge_granted", "split_bisectors", "merged_bisectors",
               "merge_groups", "allocated", "max_depth", "ab_mismatch", "frame"]


class _Stats(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in STAT_FIELDS]


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def halfedges_from_faces(mesh):
    lib = _load()
    H = mesh.H
    arrs = {k: np.zeros(H, np.int32) for k in ("twin", "next", "prev", "vert", "face")}
    fs = np.ascontiguousarray(mesh.face_sizes, np.int32)
    fv = np.ascontiguousarray(mesh.face_verts, np.int32)
    rc = lib.or_halfedges_from_faces(mesh.F, _ptr(fs), _ptr(fv), H, _ptr(arrs["twin"]),
                                     _ptr(arrs["next"]), _ptr(arrs["prev"]), _ptr(arrs["vert"]),
                                     _ptr(arrs["face"]))
    if rc:
        raise OracleError(rc, "halfedges_from_faces")
    return arrs


class Oracle:
    """One instance: the halfedge mesh, a pool of 2^D bisectors, max depth."""

    def __init__(self, mesh=None, D=16, max_depth=14, halfedges=None, pos=None):
        lib = _load()
        if halfedges is None:
            halfedges = halfedges_from_faces(mesh)
        if pos is None:
            pos = mesh.pos
        self.halfedges = halfedges
        pos = np.ascontiguousarray(pos, np.float64)
        H = int(halfedges["twin"].shape[0])
        h = C.c_void_p()
        rc = lib.or_create(H, _ptr(halfedges["twin"]), _ptr(halfedges["next"]),
                           _ptr(halfedges["prev"]), _ptr(halfedges["vert"]),
                           _ptr(halfedges["face"]), pos.shape[0], _ptr(pos), D, max_depth,
                           C.byref(h))
        if rc:
            raise OracleError(rc, "create")
        self._h = h
        self.H, self.D, self.max_depth = H, D, max_depth
        self.cap = 1 << D
        self.ch = lib.or_ceil_log2_H(h)

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.or_destroy(self._h)
            self._h = None

    @staticmethod
    def frame_struct(fp):
        f = _Frame()
        for i in range(3):
            f.eye[i] = float(fp.eye[i])
        pl = np.asarray(fp.planes, np.float32).reshape(-1)
        for i in range(15):
            f.planes[i] = float(pl[i]) if i < pl.size else 0.0
        f.q = float(np.float32(fp.q))
        f.nplanes = int(fp.nplanes)
        f.mode = int(fp.mode)
        f.seed = int(fp.seed)
        f.precision = int(fp.precision)
        f.fixed_shift = int(fp.fixed_shift)
        f.gate = int(fp.gate)
        f.sphere_radius = float(getattr(fp, "sphere_radius", 0.0))
        f.disp = _disp(fp)
        keep = []
        for name, cnt, arr in (("split_list", "n_split", fp.split_list),
                               ("merge_list", "n_merge", fp.merge_list)):
            a = np.ascontiguousarray(np.sort(np.asarray(arr, np.uint64)))
            keep.append(a)
            setattr(f, name, a.ctypes.data if a.size else None)
            setattr(f, cnt, int(a.size))
        return f, keep

    def update(self, fp) -> dict:
        f, keep = self.frame_struct(fp)
        s = _Stats()
        rc = _lib.or_update(self._h, C.byref(f), C.byref(s))
        del keep
        if rc:
            raise OracleError(rc, "update")
        return {n: int(getattr(s, n)) for n in STAT_FIELDS}

    def set_order_seed(self, seed: int):
        _lib.or_set_order_seed(self._h, int(seed))

    def chain_cost(self, slot: int) -> int:
        c = C.c_uint32()
        rc = _lib.or_chain_cost(self._h, int(slot), C.byref(c))
        if rc:
            raise OracleError(rc, "chain_cost")
        return int(c.value)

    @property
    def live_count(self) -> int:
        return int(_lib.or_live_count(self._h))

    def export(self) -> dict:
        cap = self.cap
        out = {"cbt": np.zeros(2 * cap, np.uint32), "heap": np.zeros(cap, np.uint64),
               "twin": np.zeros(cap, np.uint32), "next": np.zeros(cap, np.uint32),
               "prev": np.zeros(cap, np.uint32)}
        _lib.or_export(self._h, _ptr(out["cbt"]), _ptr(out["heap"]), _ptr(out["twin"]),
                       _ptr(out["next"]), _ptr(out["prev"]))
        return out

    def leaves(self):
        n = self.live_count
        slots = np.zeros(n, np.uint32)
        heap = np.zeros(n, np.uint64)
        links = np.zeros((n, 3), np.uint32)
        _lib.or_leaves(self._h, _ptr(slots), _ptr(heap), _ptr(links))
        return slots, heap, links

    def vertices(self, origin, precision=0, fixed_shift=20, sphere_radius=0.0, frame=None):
        """Vertices of the live bisectors relative to ``origin``; with
        ``frame`` (a FrameParams) its displacement is applied."""
        n = self.live_count
        out = np.zeros((n, 3, 3), np.float32)
        o = np.ascontiguousarray(origin, np.float64)
        d = _disp(frame) if frame is not None else None
        _lib.or_vertices(self._h, _ptr(o), precision, fixed_shift, float(sphere_radius),
                         C.addressof(d) if d is not None else None, _ptr(out))
        return out

    def export_indexed(self, tri_vertices=None):
        """Indexed form of the live bisectors: (vertices [nv, 3] from
        tri_vertices [N, 3, 3] or None, indices [N, 3], heap IDs [N])."""
        n = self.live_count
        idx = np.zeros((n, 3), np.uint32)
        ids = np.zeros(n, np.uint64)
        tv = np.ascontiguousarray(tri_vertices, np.float32) if tri_vertices is not None else None
        vb = np.zeros((3 * n, 3), np.float32) if tv is not None else None
        nv = C.c_uint32()
        rc = _lib.or_export_indexed(self._h, _ptr(tv), _ptr(vb), _ptr(idx), _ptr(ids), C.byref(nv))
        if rc:
            raise OracleError(rc, "export_indexed")
        return (vb[:nv.value] if vb is not None else None), idx, ids

    def vertices_f64(self):
        out = np.zeros((self.live_count, 3, 3), np.float64)
        _lib.or_vertices_f64(self._h, _ptr(out))
        return out

    def root_table(self):
        out = np.zeros((self.H, 3, 3), np.float64)
        _lib.or_root_table(self._h, _ptr(out))
        return out


def lowbias32(x: int) -> int:
    """The displacement's lattice hash on one 32-bit word."""
    return int(_load().or_lowbias32(int(x) & 0xFFFFFFFF))


def fbm(x, frequency: float, octaves: int, seed: int) -> float:
    """Fractal value noise of 2 or 3 FP32 coordinates (the displacement's
    height before the amplitude)."""
    a = np.ascontiguousarray(x, np.float32)
    return float(_load().or_fbm(_ptr(a), int(a.size), float(np.float32(frequency)), int(octaves), int(seed)))


def cbt_sum_reduction(D: int, cbt: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(cbt, np.uint32).copy()
    _load().or_cbt_sum_reduction(D, _ptr(c))
    return c


def cbt_one_to_bit(D: int, cbt: np.ndarray, i: int) -> int:
    c = np.ascontiguousarray(cbt, np.uint32)
    return int(_load().or_cbt_one_to_bit(D, _ptr(c), i))


def cbt_compact(D: int, cbt: np.ndarray) -> np.ndarray:
    """OneToBitID(i) for every i below the root (CachePointers, Alg. 7)."""
    c = np.ascontiguousarray(cbt, np.uint32)
    out = np.zeros(max(int(c[1]), 1), np.uint32)
    _load().or_cbt_compact(D, _ptr(c), _ptr(out))
    return out[:int(c[1])]


def cbt_zero_to_bit(D: int, cbt: np.ndarray, i: int) -> int:
    c = np.ascontiguousarray(cbt, np.uint32)
    return int(_load().or_cbt_zero_to_bit(D, _ptr(c), i))


def decode_weights(j: int, ch: int) -> np.ndarray:
    W = np.zeros(9, np.uint64)
    _load().or_decode_weights(int(j), ch, _ptr(W))
    return W.reshape(3, 3)


def splitmix64(x: int) -> int:
    return int(_load().or_splitmix64(int(x) & 0xFFFFFFFFFFFFFFFF))


def lod_test(r9, planes15, nplanes, q) -> int:
    r = np.ascontiguousarray(r9, np.float32).reshape(-1)
    p = np.ascontiguousarray(planes15, np.float32).reshape(-1)
    if p.size < 15:
        p = np.concatenate([p, np.zeros(15 - p.size, np.float32)])
    return int(_load().or_lod_test(_ptr(r), _ptr(p), nplanes, float(np.float32(q))))

"""Python binding of libcbt.so (argument marshalling only).

Every step of the update runs in the library's CUDA kernels; torch supplies
device memory (the workspace and output buffers) and the stream. There is no
CPU path: the CUDA library must be loadable, else importing raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from .build import LIB as _LIB_PATH

_lib = None

CBT_NULL = 0xFFFFFFFF
ERRORS = {1: "EINVAL", 2: "ECAPACITY", 3: "EDEPTH", 4: "ENOMEM", 5: "ECUDA", 6: "EDEVICE",
          7: "ETIMEOUT"}


class CBTError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: CBT_{ERRORS.get(code, code)}")
        self.code = code


def load(path: str | None = None):
    """Loads the CUDA library (built in-tree by ``build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libcbt.so not built ({path}); run paper_2407_02215_gb300.build.build()")
    lib = C.CDLL(path)
    P, U32, I32 = C.c_void_p, C.c_uint32, C.c_int32
    lib.cbt_halfedges_from_faces.argtypes = [I32, P, P, I32, P, P, P, P, P]
    lib.cbt_workspace_bytes.argtypes = [I32, I32]
    lib.cbt_workspace_bytes.restype = C.c_size_t
    lib.cbt_point_cache_bytes.argtypes = [I32]
    lib.cbt_point_cache_bytes.restype = C.c_size_t
    lib.cbt_attach_point_cache.argtypes = [P, P, C.c_size_t, P]
    lib.cbt_create.argtypes = [I32, P, P, P, P, P, I32, P, I32, I32, P, C.c_size_t, P,
                               C.POINTER(C.c_void_p)]
    lib.cbt_update.argtypes = [P, P, P]
    lib.cbt_frame_from_camera.argtypes = [P, C.c_float, C.c_int, P]
    lib.cbt_update_many.argtypes = [P, P, I32, P]
    lib.cbt_live_count.argtypes = [P, C.POINTER(U32), P]
    lib.cbt_live_count_async.argtypes = [P, P, P]
    lib.cbt_vertices_to_host_async.argtypes = [P, P, U32, P]
    lib.cbt_leaves.argtypes = [P, P, P, P, U32, C.POINTER(U32), P]
    lib.cbt_vertices.argtypes = [P, P, P, U32, I32, U32, C.POINTER(U32), P]
    lib.cbt_host_device_pointer.argtypes = [P, C.POINTER(P)]
    lib.cbt_vertices_to_host.argtypes = [P, P, P, U32, P, P]
    lib.cbt_index_workspace_bytes.argtypes = [C.c_void_p, U32]
    lib.cbt_index_workspace_bytes.restype = C.c_size_t
    lib.cbt_index.argtypes = [P, P, P, C.c_size_t, P, U32, P, U32, P, C.POINTER(U32), C.POINTER(U32), P]
    lib.cbt_cbt.argtypes = [P, P, P, P]
    lib.cbt_stats.argtypes = [P, P, P]
    lib.cbt_destroy.argtypes = [P]
    lib.cbt_last_launch_count.argtypes = [P]
    lib.cbt_last_launch_count.restype = U32
    lib.cbt_set_graph.argtypes = [P, C.c_int]
    lib.cbt_batch_workspace_bytes.argtypes = [P, I32]
    lib.cbt_batch_workspace_bytes.restype = C.c_size_t
    lib.cbt_batch_create.argtypes = [P, I32, P, C.c_size_t, P, C.POINTER(C.c_void_p)]
    lib.cbt_batch_update.argtypes = [P, P, P]
    lib.cbt_batch_set_graph.argtypes = [P, C.c_int]
    lib.cbt_batch_autotune.argtypes = [P, U32]
    lib.cbt_batch_config.argtypes = [P, C.POINTER(U32), C.POINTER(U32), C.POINTER(C.c_int)]
    lib.cbt_batch_set_config.argtypes = [P, U32, U32, P]
    lib.cbt_batch_set_timing.argtypes = [P, C.c_int]
    lib.cbt_batch_kernel_times.argtypes = [P, P, U32]
    lib.cbt_batch_kernel_times.restype = U32
    lib.cbt_batch_last_launch_count.argtypes = [P]
    lib.cbt_batch_last_launch_count.restype = U32
    lib.cbt_batch_destroy.argtypes = [P]
    lib.cbt_server_workspace_bytes.argtypes = [P, I32, I32]
    lib.cbt_server_workspace_bytes.restype = C.c_size_t
    lib.cbt_server_create.argtypes = [P, I32, I32, P, C.c_size_t, C.POINTER(C.c_void_p)]
    lib.cbt_server_submit.argtypes = [P, P, P, I32, P, C.POINTER(I32)]
    lib.cbt_server_poll.argtypes = [P, I32, C.c_int, P]
    lib.cbt_server_next_slot_free.argtypes = [P]
    lib.cbt_server_next_slot_free.restype = I32
    lib.cbt_server_destroy.argtypes = [P]
    lib.cbt_set_timing.argtypes = [P, C.c_int]
    lib.cbt_kernel_times.argtypes = [P, P, U32]
    lib.cbt_kernel_times.restype = U32
    lib.cbt_kernel_name.argtypes = [U32]
    lib.cbt_kernel_name.restype = C.c_char_p
    lib.cbt_phase_name.argtypes = [U32]
    lib.cbt_phase_name.restype = C.c_char_p
    lib.cbt_state_phase_name.argtypes = [P, U32]
    lib.cbt_state_phase_name.restype = C.c_char_p
    lib.cbt_sum_reduce.argtypes = [P, I32, P, P]
    lib.cbt_compact.argtypes = [P, P, I32, P, C.c_uint32, P]
    lib.cbt_server_set_fused.argtypes = [P, C.c_int]
    lib.cbt_selftest_bounded_wait.argtypes = [P, I32, I32, P]
    lib.cbt_set_fused.argtypes = [P, C.c_int, P]
    lib.cbt_fused.argtypes = [P]
    lib.cbt_batch_set_fused.argtypes = [P, C.c_int, P]
    lib.cbt_batch_fused.argtypes = [P]
    _lib = lib
    return lib


class Frame(C.Structure):
    """Mirror of ``cbt_frame`` (include/cbt.h)."""

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
        ("vertices_out", C.c_void_p),
        ("vertices_cap", C.c_uint32),
        ("sphere_radius", C.c_double),
        ("disp_amplitude", C.c_float),
        ("disp_frequency", C.c_float),
        ("disp_octaves", C.c_uint32),
        ("disp_seed", C.c_uint32),
    ]


class Camera(C.Structure):
    """Mirror of ``cbt_camera`` (include/cbt.h)."""

    _fields_ = [
        ("eye", C.c_double * 3),
        ("target", C.c_double * 3),
        ("up", C.c_double * 3),
        ("fovy_rad", C.c_double),
        ("aspect", C.c_double),
        ("width_px", C.c_int32),
        ("height_px", C.c_int32),
    ]


def frame_from_camera(eye, target, up, fovy_rad: float, aspect: float, width_px: int, height_px: int,
                      tau_px: float, frustum: bool = True) -> dict:
    """cbt_frame_from_camera: the frame's eye, FP32 planes [5, 3], plane
    count and q from a camera (host only)."""
    lib = load()
    cam = Camera()
    for i in range(3):
        cam.eye[i], cam.target[i], cam.up[i] = float(eye[i]), float(target[i]), float(up[i])
    cam.fovy_rad, cam.aspect = float(fovy_rad), float(aspect)
    cam.width_px, cam.height_px = int(width_px), int(height_px)
    f = Frame()
    rc = lib.cbt_frame_from_camera(C.byref(cam), C.c_float(tau_px), 1 if frustum else 0, C.byref(f))
    if rc:
        raise CBTError(rc, "cbt_frame_from_camera")
    return {"eye": np.array(f.eye[:], np.float64), "planes": np.array(f.planes[:], np.float32).reshape(5, 3),
            "nplanes": int(f.nplanes), "q": np.float32(f.q)}


STAT_FIELDS = ["live_before", "live_after", "free_before", "split_wishes", "merge_candidates",
               "split_granted", "merge_granted", "split_bisectors", "merged_bisectors",
               "merge_groups", "allocated", "relinked", "frame", "error"]


class Stats(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in STAT_FIELDS]


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _t_ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def halfedges_from_faces(mesh) -> dict:
    """Faces -> halfedge arrays with the library's host ingest."""
    lib = load()
    H = int(np.asarray(mesh.face_sizes).sum())
    out = {k: np.zeros(H, np.int32) for k in ("twin", "next", "prev", "vert", "face")}
    fs = np.ascontiguousarray(mesh.face_sizes, np.int32)
    fv = np.ascontiguousarray(mesh.face_verts, np.int32)
    rc = lib.cbt_halfedges_from_faces(len(fs), _np_ptr(fs), _np_ptr(fv), H, _np_ptr(out["twin"]),
                                      _np_ptr(out["next"]), _np_ptr(out["prev"]),
                                      _np_ptr(out["vert"]), _np_ptr(out["face"]))
    if rc:
        raise CBTError(rc, "cbt_halfedges_from_faces")
    return out


def sum_reduce(bits, D: int, sums, stream=None):
    """SumReduction (Sec. 3.1) of a device bitfield (uint32 tensor of 2^D / 32
    words) into `sums` (uint32 tensor of 2W words, layout of CBT.cbt())."""
    rc = load().cbt_sum_reduce(_t_ptr(bits), int(D), _t_ptr(sums), _stream_ptr(stream))
    if rc:
        raise CBTError(rc, "cbt_sum_reduce")


def compact(bits, sums, D: int, live, stream=None):
    """CachePointers (Alg. 7) of a device bitfield with its sum tree (from
    sum_reduce): live[i] = position of the i-th set bit, for i < sums[1]
    (entries beyond live's length are dropped)."""
    rc = load().cbt_compact(_t_ptr(bits), _t_ptr(sums), int(D), _t_ptr(live), int(live.numel()),
                            _stream_ptr(stream))
    if rc:
        raise CBTError(rc, "cbt_compact")


def workspace_bytes(H: int, D: int) -> int:
    return int(load().cbt_workspace_bytes(H, D))


def device_address(t) -> int:
    """Address a kernel writes `t` at: its own for a device tensor, the
    mapped device alias for a pinned host tensor (cbt_host_device_pointer)."""
    if t.device.type == "cuda":
        return t.data_ptr()
    if not t.is_pinned():
        raise CBTError(1, "host outputs must be pinned (page-locked) tensors")
    d = C.c_void_p()
    rc = load().cbt_host_device_pointer(C.c_void_p(t.data_ptr()), C.byref(d))
    if rc:
        raise CBTError(rc, "cbt_host_device_pointer")
    return int(d.value)


def frame_struct(fp, device, vertices_out=None) -> tuple:
    """Packs a frame-parameter object (fields as in cbt_frame) into the C
    struct; LIST-mode heap IDs are uploaded to the device; vertices_out is an
    optional float32 [rows, 3, 3] tensor for the frame's vertex export, on
    the device or pinned in host memory (written there directly)."""
    f = Frame()
    if vertices_out is not None:
        f.vertices_out = device_address(vertices_out)
        f.vertices_cap = int(vertices_out.shape[0])
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
    f.disp_amplitude = float(getattr(fp, "disp_amplitude", 0.0))
    f.disp_frequency = float(getattr(fp, "disp_frequency", 0.0))
    f.disp_octaves = int(getattr(fp, "disp_octaves", 0))
    f.disp_seed = int(getattr(fp, "disp_seed", 0))
    keep = []
    for name, cnt, arr in (("split_list", "n_split", getattr(fp, "split_list", ())),
                           ("merge_list", "n_merge", getattr(fp, "merge_list", ()))):
        a = np.sort(np.asarray(arr, np.uint64))
        if a.size:
            t = torch.from_numpy(a.view(np.int64)).to(device)
            keep.append(t)
            setattr(f, name, t.data_ptr())
        setattr(f, cnt, int(a.size))
    return f, keep


class CBT:
    """One instance: a halfedge mesh and a pool of 2^D bisectors on a GPU."""

    def __init__(self, mesh=None, D: int = 16, max_depth: int = 14, halfedges=None, pos=None,
                 device="cuda", stream=None, workspace=None, point_cache=False):
        """``workspace``: optional caller memory (a contiguous uint8 CUDA tensor of
        at least cbt_workspace_bytes); ``point_cache``: True to attach a newly
        allocated sphere-form point cache (cbt_attach_point_cache), or a uint8
        CUDA tensor of at least cbt_point_cache_bytes to attach as it is."""
        lib = load()
        if halfedges is None:
            halfedges = halfedges_from_faces(mesh)
        if pos is None:
            pos = mesh.pos
        self.halfedges = halfedges
        pos = np.ascontiguousarray(pos, np.float64)
        H = int(halfedges["twin"].shape[0])
        self.H, self.D, self.max_depth = H, D, max_depth
        self.cap = 1 << D
        self.device = torch.device(device)
        nbytes = lib.cbt_workspace_bytes(H, D)
        if nbytes == 0:
            raise CBTError(1, "cbt_workspace_bytes")
        pbytes = lib.cbt_point_cache_bytes(D)
        if isinstance(point_cache, torch.Tensor):
            if (point_cache.dtype != torch.uint8 or not point_cache.is_cuda or not point_cache.is_contiguous()
                    or point_cache.numel() < pbytes):
                raise ValueError(f"point_cache: a contiguous uint8 CUDA tensor of at least {pbytes} bytes")
        elif not (point_cache is True or point_cache is False or point_cache is None):
            raise ValueError("point_cache: True, False or a uint8 CUDA tensor")
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        elif (workspace.dtype != torch.uint8 or not workspace.is_cuda or not workspace.is_contiguous()
              or workspace.numel() < nbytes):
            raise ValueError(f"workspace: a contiguous uint8 CUDA tensor of at least {nbytes} bytes")
        else:
            self.device = workspace.device
        self.workspace = workspace  # caller memory is reused as it is (cbt_create initialises what it reads)
        h = C.c_void_p()
        he = {k: np.ascontiguousarray(v, np.int32) for k, v in halfedges.items()}
        rc = lib.cbt_create(H, _np_ptr(he["twin"]), _np_ptr(he["next"]), _np_ptr(he["prev"]),
                            _np_ptr(he["vert"]), _np_ptr(he["face"]), pos.shape[0], _np_ptr(pos),
                            D, max_depth, _t_ptr(self.workspace), nbytes, _stream_ptr(stream),
                            C.byref(h))
        if rc:
            raise CBTError(rc, "cbt_create")
        self._h = h
        self._keep = []
        self.point_cache = None
        if point_cache is not False and point_cache is not None:
            if point_cache is True:
                point_cache = torch.empty(pbytes, dtype=torch.uint8, device=self.device)
            rc = lib.cbt_attach_point_cache(h, _t_ptr(point_cache), point_cache.numel(), _stream_ptr(stream))
            if rc:
                raise CBTError(rc, "cbt_attach_point_cache")
            self.point_cache = point_cache

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.cbt_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def update(self, fp, stream=None, vertices_out=None):
        f, keep = frame_struct(fp, self.device, vertices_out)
        self._keep = keep
        rc = _lib.cbt_update(self._h, C.byref(f), _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_update")

    @property
    def last_launch_count(self) -> int:
        return int(_lib.cbt_last_launch_count(self._h))

    def set_graph(self, on: bool = True):
        rc = _lib.cbt_set_graph(self._h, 1 if on else 0)
        if rc:
            raise CBTError(rc, "cbt_set_graph")

    def set_timing(self, on: bool = True):
        rc = _lib.cbt_set_timing(self._h, 1 if on else 0)
        if rc:
            raise CBTError(rc, "cbt_set_timing")

    def set_fused(self, on: bool = True, stream=None):
        """One cooperative launch per frame (default) or one launch per step."""
        rc = _lib.cbt_set_fused(self._h, 1 if on else 0, _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_set_fused")

    @property
    def fused(self) -> bool:
        return bool(_lib.cbt_fused(self._h))

    def kernel_times(self) -> dict:
        """Durations (ms) of the last frame: per kernel (per-step form) or
        per phase (fused form), by name."""
        buf = (C.c_float * 16)()
        n = _lib.cbt_kernel_times(self._h, buf, 16)
        if self.fused:
            return {_lib.cbt_state_phase_name(self._h, k).decode(): float(buf[k]) for k in range(n)}
        return {_lib.cbt_kernel_name(k).decode(): float(buf[k]) for k in range(n)}

    def live_count(self, stream=None) -> int:
        n = C.c_uint32()
        rc = _lib.cbt_live_count(self._h, C.byref(n), _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_live_count")
        return int(n.value)

    def live_count_async(self, out, stream=None):
        """Enqueues the live count into out[0] (a 4-byte CUDA tensor, or a
        pinned host tensor) on the stream, without synchronising."""
        if out.element_size() != 4 or not (out.is_cuda or out.is_pinned()):
            raise ValueError("out: a 4-byte CUDA or pinned host tensor")
        rc = _lib.cbt_live_count_async(self._h, C.c_void_p(out.data_ptr()), _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_live_count_async")

    def leaves(self, stream=None):
        n = self.live_count(stream)
        slots = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        heap = torch.empty(max(n, 1), dtype=torch.int64, device=self.device)
        links = torch.empty((max(n, 1), 3), dtype=torch.int32, device=self.device)
        cnt = C.c_uint32()
        rc = _lib.cbt_leaves(self._h, _t_ptr(slots), _t_ptr(heap), _t_ptr(links), max(n, 1),
                             C.byref(cnt), _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_leaves")
        n = int(cnt.value)
        return slots[:n], heap[:n], links[:n]

    def vertices(self, origin, precision=0, fixed_shift=20, out=None, stream=None):
        n = self.live_count(stream)
        if out is None:
            out = torch.empty((max(n, 1), 3, 3), dtype=torch.float32, device=self.device)
        o = (C.c_double * 3)(*[float(x) for x in origin])
        cnt = C.c_uint32()
        rc = _lib.cbt_vertices(self._h, _t_ptr(out), o, precision, fixed_shift, out.shape[0],
                               C.byref(cnt), _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_vertices")
        return out[:int(cnt.value)]

    def vertices_to_host(self, d_vertices, h_vertices, h_count, stream=None) -> int:
        """Copies the frame's exported vertices (device [N, 3, 3]) into the
        pinned host tensor h_vertices with one synchronisation; h_count is a
        pinned int32 tensor of one element. Returns N."""
        rc = _lib.cbt_vertices_to_host(self._h, _t_ptr(d_vertices), _t_ptr(h_vertices), int(h_vertices.shape[0]),
                                       _t_ptr(h_count), _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_vertices_to_host")
        return int(h_count[0])

    def index_workspace(self, max_live: int):
        """Device scratch for index() with up to max_live live bisectors."""
        return torch.empty(int(_lib.cbt_index_workspace_bytes(self._h, int(max_live))), dtype=torch.uint8,
                           device=self.device)

    def index(self, tri_vertices=None, workspace=None, out=None, stream=None):
        """Indexed export (cbt_index): (vertices [nv, 3] or None, indices
        [N, 3] int32, heap IDs [N] int64). tri_vertices: the per-bisector
        vertices [N, 3, 3] of the current live list. out: optional reusable
        buffers (vertices [rows, 3] or None, indices [cap, 3], heap IDs
        [cap]); the workspace must cover their capacity. One synchronisation."""
        if out is None:
            cap = self.cap
            verts = (torch.empty((3 * cap, 3), dtype=torch.float32, device=self.device)
                     if tri_vertices is not None else None)
            idx = torch.empty((cap, 3), dtype=torch.int32, device=self.device)
            heap = torch.empty(cap, dtype=torch.int64, device=self.device)
        else:
            verts, idx, heap = out
            cap = idx.shape[0]
        if workspace is None:
            workspace = self.index_workspace(cap)
        nv, nt = C.c_uint32(), C.c_uint32()
        rc = _lib.cbt_index(self._h, _t_ptr(tri_vertices) if tri_vertices is not None else None, _t_ptr(workspace),
                            workspace.numel(), _t_ptr(verts) if verts is not None else None,
                            verts.shape[0] if verts is not None else 0, _t_ptr(idx), cap, _t_ptr(heap),
                            C.byref(nv), C.byref(nt), _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_index")
        k = int(nt.value)
        return (verts[:int(nv.value)] if verts is not None else None), idx[:k], heap[:k]

    def cbt(self, stream=None):
        W = max(1, self.cap // 32)
        bits = torch.empty(W, dtype=torch.int32, device=self.device)
        sums = torch.empty(2 * W, dtype=torch.int32, device=self.device)
        rc = _lib.cbt_cbt(self._h, _t_ptr(bits), _t_ptr(sums), _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_cbt")
        return bits, sums

    def stats(self, stream=None, check=True) -> dict:
        s = Stats()
        rc = _lib.cbt_stats(self._h, C.byref(s), _stream_ptr(stream))
        if rc and (check or rc != 6):
            raise CBTError(rc, f"cbt_stats (device error bits {s.error:#x})")
        return {n: int(getattr(s, n)) for n in STAT_FIELDS}


def handles_of(instances):
    """The states' handles as a C array (for update_many_packed)."""
    return (C.c_void_p * len(instances))(*[g.handle.value for g in instances])


def pack_frames(fps, device, vertices_out=None):
    """The frames as a C array of cbt_frame, and the device buffers they
    point to (keep both alive while the frames are in use)."""
    arr = (Frame * len(fps))()
    keep = []
    for b, fp in enumerate(fps):
        vo = vertices_out[b] if vertices_out is not None else None
        f, k = frame_struct(fp, device, vo)
        arr[b] = f
        keep.extend(k)
    return arr, keep


def update_many_packed(handles, arr, n: int, stream=None):
    rc = load().cbt_update_many(handles, arr, n, _stream_ptr(stream))
    if rc:
        raise CBTError(rc, "cbt_update_many")


def vertices_to_host_async(d_vertices, h_vertices, rows: int, stream=None):
    """cbt_vertices_to_host_async: the first `rows` rows of a vertex export
    (CUDA tensor) into a pinned host tensor by the copy engine, on the
    stream, without synchronising."""
    if not d_vertices.is_cuda or not h_vertices.is_pinned():
        raise ValueError("d_vertices: a CUDA tensor; h_vertices: a pinned host tensor")
    if rows > min(d_vertices.shape[0], h_vertices.shape[0]):
        raise ValueError("rows beyond the buffers")
    rc = load().cbt_vertices_to_host_async(C.c_void_p(d_vertices.data_ptr()), C.c_void_p(h_vertices.data_ptr()),
                                           int(rows), _stream_ptr(stream))
    if rc:
        raise CBTError(rc, "cbt_vertices_to_host_async")


def update_many(instances, fps, stream=None, vertices_out=None):
    """cbt_update_many: one plain cbt_update per instance, issued from the
    library's host loop in one call (frames fps[b] for instances[b])."""
    arr, keep = pack_frames(fps, instances[0].device, vertices_out)
    update_many_packed(handles_of(instances), arr, len(instances), stream)
    del keep


class Batch:
    """Several CBT instances updated by one launch per kernel and frame."""

    def __init__(self, instances, stream=None):
        lib = load()
        self.instances = list(instances)
        n = len(self.instances)
        handles = (C.c_void_p * n)(*[g.handle.value for g in self.instances])
        self._handles = handles
        nbytes = lib.cbt_batch_workspace_bytes(handles, n)
        if nbytes == 0:
            raise CBTError(1, "cbt_batch_workspace_bytes")
        self.device = self.instances[0].device
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        rc = lib.cbt_batch_create(handles, n, _t_ptr(self.workspace), nbytes, _stream_ptr(stream), C.byref(h))
        if rc:
            raise CBTError(rc, "cbt_batch_create")
        self._h = h
        self._keep = []

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.cbt_batch_destroy(self._h)
            self._h = None

    def update(self, fps, stream=None, vertices_out=None):
        n = len(self.instances)
        arr = (Frame * n)()
        keep = []
        for b, fp in enumerate(fps):
            vo = vertices_out[b] if vertices_out is not None else None
            f, k = frame_struct(fp, self.device, vo)
            arr[b] = f
            keep.extend(k)
        self._keep = keep
        rc = _lib.cbt_batch_update(self._h, arr, _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_batch_update")

    def update_packed(self, arr, stream=None):
        """One frame from frames packed by pack_frames."""
        rc = _lib.cbt_batch_update(self._h, arr, _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_batch_update")

    def set_graph(self, on: bool = True):
        _lib.cbt_batch_set_graph(self._h, 1 if on else 0)

    def autotune(self, rounds: int = 2):
        rc = _lib.cbt_batch_autotune(self._h, rounds)
        if rc:
            raise CBTError(rc, "cbt_batch_autotune")

    def config(self):
        tw, bm, tun = C.c_uint32(), C.c_uint32(), C.c_int()
        _lib.cbt_batch_config(self._h, C.byref(tw), C.byref(bm), C.byref(tun))
        return {"tile_words": tw.value, "blocks_per_sm": bm.value, "tuning": bool(tun.value),
                "fused": self.fused}

    def set_config(self, tile_words: int, blocks_per_sm: int, stream=None):
        rc = _lib.cbt_batch_set_config(self._h, tile_words, blocks_per_sm, _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_batch_set_config")

    def set_timing(self, on: bool = True):
        _lib.cbt_batch_set_timing(self._h, 1 if on else 0)

    def set_fused(self, on: bool = True, stream=None):
        rc = _lib.cbt_batch_set_fused(self._h, 1 if on else 0, _stream_ptr(stream))
        if rc:
            raise CBTError(rc, "cbt_batch_set_fused")

    @property
    def fused(self) -> bool:
        return bool(_lib.cbt_batch_fused(self._h))

    def kernel_times(self) -> dict:
        buf = (C.c_float * 16)()
        n = _lib.cbt_batch_kernel_times(self._h, buf, 16)
        name = _lib.cbt_phase_name if self.fused else _lib.cbt_kernel_name
        return {name(k).decode(): float(buf[k]) for k in range(n)}

    @property
    def last_launch_count(self) -> int:
        return int(_lib.cbt_batch_last_launch_count(self._h))


class Server:
    """Resident instances served by ticks (see cbt_server in include/cbt.h)."""

    def __init__(self, instances, inflight: int = 2):
        lib = load()
        self.instances = list(instances)
        n = len(self.instances)
        self._handles = (C.c_void_p * n)(*[g.handle.value for g in self.instances])
        nbytes = lib.cbt_server_workspace_bytes(self._handles, n, inflight)
        if nbytes == 0:
            raise CBTError(1, "cbt_server_workspace_bytes")
        self.device = self.instances[0].device
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        rc = lib.cbt_server_create(self._handles, n, inflight, _t_ptr(self.workspace), nbytes, C.byref(h))
        if rc:
            raise CBTError(rc, "cbt_server_create")
        self._h = h
        self.inflight = inflight
        self._pending = {}

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.cbt_server_destroy(self._h)
            self._h = None

    def set_fused(self, on: bool = True):
        """Ticks as one cooperative launch each, one at a time on the device."""
        rc = _lib.cbt_server_set_fused(self._h, 1 if on else 0)
        if rc:
            raise CBTError(rc, "cbt_server_set_fused")

    def next_slot_free(self) -> bool:
        return bool(_lib.cbt_server_next_slot_free(self._h))

    def submit(self, idx, fps, stream=None, vertices_out=None) -> int:
        k = len(idx)
        arr = (Frame * k)()
        keep = []
        for i, fp in enumerate(fps):
            vo = vertices_out[i] if vertices_out is not None else None
            f, kp = frame_struct(fp, self.device, vo)
            arr[i] = f
            keep.extend(kp)
        ids = (C.c_int32 * k)(*idx)
        t = C.c_int32()
        rc = _lib.cbt_server_submit(self._h, ids, arr, k, _stream_ptr(stream), C.byref(t))
        if rc:
            raise CBTError(rc, "cbt_server_submit")
        self._pending[t.value] = (list(idx), keep)
        return t.value

    def poll(self, ticket: int, wait: bool = False):
        """None while pending, else the live counts at frame start."""
        idx, _ = self._pending[ticket]
        out = (C.c_uint32 * len(idx))()
        r = _lib.cbt_server_poll(self._h, ticket, 1 if wait else 0, out)
        if r < 0:
            raise CBTError(-r, "cbt_server_poll")
        if r == 0:
            return None
        del self._pending[ticket]
        return list(out)

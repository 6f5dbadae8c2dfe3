"""cbt_frame_from_camera gives, bit for bit, the frame inputs the harness
derives from the same camera: the eye, the five FP32 plane normals through
the eye and q = (K / tau)^2 (the paper leaves the LOD criterion to the
application, Sec. 3.3 kernel 4). Host only: no GPU needed."""
import ctypes as C
import math

import numpy as np
import pytest

import workloads as W
from workloads import cameras as Cm
from paper_2407_02215_gb300 import cbt as B


def _c_frame(cam, tau, frustum=True):
    return B.frame_from_camera(cam.eye, cam.target, cam.up, cam.fovy_rad, cam.aspect, cam.width_px,
                               cam.height_px, tau, frustum)


def _same(fp, got):
    assert np.array_equal(np.asarray(fp.planes, np.float32).view(np.uint32), got["planes"].view(np.uint32))
    assert np.float32(fp.q).view(np.uint32) == got["q"].view(np.uint32)
    assert np.array_equal(np.asarray(fp.eye, np.float64).view(np.uint64), got["eye"].view(np.uint64))
    assert got["nplanes"] == fp.nplanes


def test_workload_cameras_bit_identical():
    """The cameras of the cube orbit, the grid flythrough, the planet
    descents and the dodecahedron descent."""
    paths = [(Cm.orbit_path(16, 1), 4.0), (Cm.flythrough_path(120, 2), 2.0),
             (Cm.descent_path(W.meshes.cube_sphere_mesh(8), 600, 3), 4.0),
             (Cm.sphere_descent_path(W.meshes.dodecahedron_mesh(), 6.371e6, 300, 6), 14.0)]
    n = 0
    for cams, tau in paths:
        for cam in cams:
            _same(Cm.frame_params(cam, tau), _c_frame(cam, tau))
            n += 1
    assert n == 16 + 120 + 600 + 300


def test_random_cameras_bit_identical():
    """Seeded cameras over many scales, fields of view, aspects and
    viewports, with up directions along the view (the fallback taken)."""
    rng = np.random.default_rng(7)
    for k in range(3000):
        scale = 10.0 ** rng.uniform(-3, 7)
        eye = rng.normal(size=3) * scale
        target = eye + rng.normal(size=3) * scale * 10.0 ** rng.uniform(-4, 1)
        up = rng.normal(size=3)
        if k % 7 == 0:
            up = (target - eye) * rng.uniform(0.1, 10.0)  # parallel to the view
        if k % 11 == 0:
            up = np.array([0.0, 0.0, 1.0]); target = eye + np.array([0.0, 1e-4, 5.0])  # nearly along up
        cam = Cm.Camera(eye=eye, target=target, up=up, fovy_rad=rng.uniform(0.05, 3.0), aspect=rng.uniform(0.3, 3.0),
                        width_px=int(rng.integers(64, 8192)), height_px=int(rng.integers(64, 8192)))
        tau = float(np.float32(rng.uniform(0.25, 32.0)))
        fr = k % 5 != 0
        _same(Cm.frame_params(cam, tau, frustum=fr), _c_frame(cam, tau, frustum=fr))


def test_frame_fields_left_alone_and_errors():
    lib = B.load()
    cam = B.Camera()
    for i in range(3):
        cam.eye[i], cam.target[i], cam.up[i] = 0.0, (1.0 if i == 0 else 0.0), (1.0 if i == 2 else 0.0)
    cam.fovy_rad, cam.aspect, cam.width_px, cam.height_px = math.pi / 2, 16 / 9, 1920, 1080
    f = B.Frame()
    f.mode, f.precision, f.seed, f.vertices_cap = 3, 1, 99, 1234
    assert lib.cbt_frame_from_camera(C.byref(cam), C.c_float(2.0), 1, C.byref(f)) == 0
    assert (f.mode, f.precision, f.seed, f.vertices_cap) == (3, 1, 99, 1234)
    # K = 540 / tan(pi/4) at 1080 px, q = (K / 2)^2
    assert abs(f.q - (540.0 / math.tan(math.pi / 4) / 2.0) ** 2) <= 1e-3 * f.q
    assert f.nplanes == 5
    bad = [("fovy_rad", 0.0), ("fovy_rad", 4.0), ("aspect", 0.0), ("height_px", 0), ("width_px", -1)]
    for name, v in bad:
        c2 = B.Camera.from_buffer_copy(cam)
        setattr(c2, name, v)
        assert lib.cbt_frame_from_camera(C.byref(c2), C.c_float(2.0), 1, C.byref(f)) == 1, name
    c2 = B.Camera.from_buffer_copy(cam)
    c2.target[0] = 0.0  # eye = target
    assert lib.cbt_frame_from_camera(C.byref(c2), C.c_float(2.0), 1, C.byref(f)) == 1
    c2 = B.Camera.from_buffer_copy(cam)
    c2.up[2] = 0.0  # zero up
    assert lib.cbt_frame_from_camera(C.byref(c2), C.c_float(2.0), 1, C.byref(f)) == 1
    for tau in (0.0, -1.0, float("inf"), float("nan")):
        assert lib.cbt_frame_from_camera(C.byref(cam), C.c_float(tau), 1, C.byref(f)) == 1
    assert lib.cbt_frame_from_camera(None, C.c_float(2.0), 1, C.byref(f)) == 1
    assert lib.cbt_frame_from_camera(C.byref(cam), C.c_float(2.0), 1, None) == 1

"""Seeded camera paths and the per-frame LOD inputs derived from a camera.

The paper leaves the level-of-detail criterion to the application (Sec. 3.3,
kernel 4, GenerateCommands). The inputs both implementations receive per frame
are derived here on the host in FP64 and rounded once to FP32:

* ``eye`` (FP64) - the camera position;
* ``planes`` - 5 inward plane normals through the eye (4 sides + near), FP32;
* ``q`` - ``((height_px / (2 tan(fovy / 2))) / tau_px)^2`` in FP32.

Nothing here is the method's arithmetic: it is the camera model feeding it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Wish modes shared by both implementations (frame parameter ``mode``).
MODE_LOD, MODE_FORCE_SPLIT, MODE_FORCE_MERGE, MODE_RANDOM, MODE_LIST = 0, 1, 2, 3, 4
# Vertex-evaluation precision (frame parameter ``precision``).
PREC_FP32, PREC_FIXED, PREC_FP64 = 0, 1, 2
# Vertices projected onto a sphere about the origin, evaluated in FP64.
PREC_SPHERE = 3
# Gate (frame parameter ``gate``).
GATE_CHAIN, GATE_PAPER = 0, 1


@dataclass
class Camera:
    eye: np.ndarray
    target: np.ndarray
    up: np.ndarray
    fovy_rad: float = np.pi / 2
    aspect: float = 1920 / 1080
    width_px: int = 1920
    height_px: int = 1080


@dataclass
class FrameParams:
    """One frame's inputs, identical for the oracle and the CUDA library."""

    eye: np.ndarray = field(default_factory=lambda: np.zeros(3))
    planes: np.ndarray = field(default_factory=lambda: np.zeros((5, 3), np.float32))
    nplanes: int = 5
    q: float = 1.0
    mode: int = MODE_LOD
    seed: int = 0
    precision: int = PREC_FP32
    fixed_shift: int = 20
    gate: int = GATE_CHAIN
    split_list: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint64))
    merge_list: np.ndarray = field(default_factory=lambda: np.zeros(0, np.uint64))
    sphere_radius: float = 0.0  # PREC_SPHERE: radius of the sphere about the origin
    # displacement (FP32 and sphere forms): amplitude * fractal value noise
    # of `disp_octaves` octaves at `disp_frequency` lattice cells per unit
    disp_amplitude: float = 0.0
    disp_frequency: float = 0.0
    disp_octaves: int = 0
    disp_seed: int = 0


# The camera model is written as scalar FP64 operations in a fixed order
# (every norm sqrt((x x + y y) + z z), every operation rounded on its own),
# so that cbt_frame_from_camera, which takes the same steps in C, gives the
# same bits.
def _norm3(v):
    return math.sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2])


def _cross3(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def camera_basis(cam: Camera):
    """Forward, right and up unit vectors (FP64 lists); the up direction
    falls back to +y (+x when the view runs along y) when nearly parallel
    to the view."""
    e = [float(x) for x in cam.eye]
    t = [float(x) for x in cam.target]
    up = [float(x) for x in cam.up]
    f = [t[c] - e[c] for c in range(3)]
    fn = _norm3(f)
    f = [x / fn for x in f]
    un = _norm3(up)
    if abs((f[0] * (up[0] / un) + f[1] * (up[1] / un)) + f[2] * (up[2] / un)) > 0.999:
        up = [0.0, 1.0, 0.0] if abs(f[1]) < 0.9 else [1.0, 0.0, 0.0]
    r = _cross3(f, up)
    rn = _norm3(r)
    r = [x / rn for x in r]
    return f, r, _cross3(r, f)


def frame_params(cam: Camera, tau_px: float, frustum: bool = True, **kw) -> FrameParams:
    f, r, u = camera_basis(cam)
    ty = math.tan(float(cam.fovy_rad) / 2.0)
    tx = float(cam.aspect) * ty
    planes = np.array([[tx * f[c] + r[c] for c in range(3)], [tx * f[c] - r[c] for c in range(3)],
                       [ty * f[c] + u[c] for c in range(3)], [ty * f[c] - u[c] for c in range(3)], f], np.float32)
    kq = float(cam.height_px) / (2.0 * ty) / float(tau_px)
    q = np.float32(kq * kq)
    return FrameParams(eye=np.asarray(cam.eye, np.float64).copy(), planes=planes,
                       nplanes=5 if frustum else 0, q=float(q), **kw)


def forced_params(mode: int, seed: int = 0, **kw) -> FrameParams:
    """Geometry-free frame (FORCE_SPLIT, FORCE_MERGE, RANDOM or LIST)."""
    return FrameParams(mode=mode, seed=seed, nplanes=0, q=1.0, **kw)


# ----------------------------------------------------------------- paths

def orbit_path(n_frames: int, seed: int, r_min=1.5, r_max=3.0):
    """Eyes at radius U[r_min, r_max] along uniform directions, looking at
    the origin, up = +z (the basis falls back when nearly parallel)."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n_frames):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        rad = rng.uniform(r_min, r_max)
        cams.append(Camera(eye=d * rad, target=np.zeros(3), up=np.array([0.0, 0.0, 1.0])))
    return cams


def _catmull_rom(P, t):
    """Uniform Catmull-Rom through control points P (clamped ends), t in [0,1]."""
    n = len(P)
    s = t * (n - 1)
    i = min(int(np.floor(s)), n - 2)
    u = s - i
    p0 = P[max(i - 1, 0)]
    p1, p2 = P[i], P[i + 1]
    p3 = P[min(i + 2, n - 1)]
    return 0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u * u
                  + (-p0 + 3 * p1 - 3 * p2 + p3) * u * u * u)


def flythrough_path(n_frames: int, seed: int, alt_hi=0.5, alt_lo=0.01, pitch_deg=30.0):
    """Eye on a seeded Catmull-Rom path through 8 points in [0.1, 0.9]^2;
    altitude log-interpolated alt_hi -> alt_lo -> alt_hi; looking along the
    path tangent pitched down by ``pitch_deg``; up = +z."""
    rng = np.random.default_rng(seed)
    P = rng.uniform(0.1, 0.9, size=(8, 2))
    cams = []
    for k in range(n_frames):
        t = k / max(1, n_frames - 1)
        xy = _catmull_rom(P, t)
        xy2 = _catmull_rom(P, min(1.0, t + 1e-3)) if t < 1 else xy + (xy - _catmull_rom(P, t - 1e-3))
        tang = xy2 - xy
        nrm = np.linalg.norm(tang)
        tang = tang / nrm if nrm > 0 else np.array([1.0, 0.0])
        s = 2 * t if t <= 0.5 else 2 * (1 - t)
        alt = np.exp(np.log(alt_hi) + (np.log(alt_lo) - np.log(alt_hi)) * s)
        eye = np.array([xy[0], xy[1], alt])
        pitch = np.deg2rad(pitch_deg)
        fwd = np.array([tang[0] * np.cos(pitch), tang[1] * np.cos(pitch), -np.sin(pitch)])
        cams.append(Camera(eye=eye, target=eye + fwd, up=np.array([0.0, 0.0, 1.0])))
    return cams


def descent_path(mesh, n_frames: int, seed: int, alt_hi=2e7, alt_lo=2.0):
    """Planet descent onto the surface the method refines: a seeded interior
    point of one root triangle (Vert h, Vert Next h, face centroid) of a
    seeded coarse face is the target; the altitude above that triangle's
    plane is log-spaced alt_hi -> alt_lo; looking at target + tangent * 10 *
    altitude; up = the triangle's outward normal (a coarse face of a
    cube-sphere is not planar, so its root triangles lie in different
    planes)."""
    rng = np.random.default_rng(seed)
    f = int(rng.integers(mesh.F))
    off = int(mesh.face_sizes[:f].sum())
    idx = mesh.face_verts[off:off + int(mesh.face_sizes[f])]
    P = mesh.pos[idx]
    n = len(idx)
    k = int(rng.integers(n))
    a, b, c = P[k], P[(k + 1) % n], P.sum(0) / n
    w = rng.dirichlet(np.ones(3))
    target = w[0] * a + w[1] * b + w[2] * c
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm)
    if np.dot(nrm, target) < 0:
        nrm = -nrm
    tang = b - a
    tang -= nrm * np.dot(tang, nrm)
    tang /= np.linalg.norm(tang)
    cams = []
    for k in range(n_frames):
        t = k / max(1, n_frames - 1)
        alt = np.exp(np.log(alt_hi) + (np.log(alt_lo) - np.log(alt_hi)) * t)
        eye = target + nrm * alt
        cams.append(Camera(eye=eye, target=target + tang * 10.0 * alt, up=nrm))
    return cams


def sphere_descent_path(mesh, radius: float, n_frames: int, seed: int, alt_hi=2e7, alt_lo=2.0):
    """Descent onto a sphere of the given radius about the origin: a seeded
    interior point of one coarse face, projected onto the sphere, is the
    target; the altitude above the sphere is log-spaced alt_hi -> alt_lo;
    the camera looks at target + tangent * 10 * altitude; up = the radial
    direction."""
    rng = np.random.default_rng(seed)
    f = int(rng.integers(mesh.F))
    off = int(mesh.face_sizes[:f].sum())
    idx = mesh.face_verts[off:off + int(mesh.face_sizes[f])]
    P = mesh.pos[idx]
    w = rng.dirichlet(np.ones(len(idx)))
    nrm = (w[:, None] * P).sum(0)
    nrm /= np.linalg.norm(nrm)
    target = nrm * radius
    tang = P[1] - P[0]
    tang -= nrm * np.dot(tang, nrm)
    tang /= np.linalg.norm(tang)
    cams = []
    for k in range(n_frames):
        t = k / max(1, n_frames - 1)
        alt = np.exp(np.log(alt_hi) + (np.log(alt_lo) - np.log(alt_hi)) * t)
        cams.append(Camera(eye=nrm * (radius + alt), target=target + tang * 10.0 * alt, up=nrm))
    return cams

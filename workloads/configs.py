"""The five synthetic workloads (seed = workload number) as instance specs.

1. cube: unit cube (H=24), pool 2^16, max depth 14, 16-frame orbit, tau 4 px.
2. grid: 100x100 mixed quads/triangles (~42k halfedges), pool 2^20, max
   depth 26, 120-frame flythrough at altitude 0.5 -> 0.01 -> 0.5, tau 2 px.
3. planet: cube-sphere 6 x 8 x 8 quads (H=1536) of radius 6.371e6 m, pool
   2^22, max depth 48, 600-frame descent 2e7 m -> 2 m, fixed-point vertices.
4. batch: 256 instances, H log-uniform over [24, 40k] (cube below 100,
   otherwise a grid sized to H), pools 2^14..2^20, 64 frames each.
5. served: the batch population (1024 instances) plus 8 planets.

These stand in for the paper's scenes (a dodecahedron planet with FFT waves,
a NASA Moon heightfield and an unnamed 21k-halfedge asset), whose data is not
available; only their sizes and structure are imitated.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import cameras as C
from . import meshes as M


@dataclass
class InstanceSpec:
    name: str
    mesh: M.PolyMesh
    D: int
    max_depth: int
    frames: list = field(default_factory=list)


def ceil_log2(x: int) -> int:
    c = 0
    while (1 << c) < x:
        c += 1
    return c


def config1(n_frames: int = 16, tau_px: float = 4.0) -> InstanceSpec:
    cams = C.orbit_path(n_frames, seed=1)
    frames = [C.frame_params(c, tau_px) for c in cams]
    return InstanceSpec("cube", M.cube_mesh(), 16, 14, frames)


def config1_uniform(depth: int = 10) -> InstanceSpec:
    """Forced uniform refinement to ``depth`` then forced merging back to 0."""
    frames = [C.forced_params(C.MODE_FORCE_SPLIT) for _ in range(depth)]
    frames += [C.forced_params(C.MODE_FORCE_MERGE) for _ in range(depth)]
    return InstanceSpec("cube-uniform", M.cube_mesh(), 16, 14, frames)


def config2(n_frames: int = 120, tau_px: float = 2.0, nx: int = 100) -> InstanceSpec:
    mesh = M.grid_mesh(nx, nx, tri_frac=0.1, seed=2, height_sigma=0.05)
    cams = C.flythrough_path(n_frames, seed=2)
    frames = [C.frame_params(c, tau_px) for c in cams]
    return InstanceSpec("grid", mesh, 20, 26, frames)


def config3(n_frames: int = 600, tau_px: float = 4.0, precision: int = C.PREC_FIXED,
            D: int = 22) -> InstanceSpec:
    mesh = M.cube_sphere_mesh(8, 6.371e6)
    cams = C.descent_path(mesh, n_frames, seed=3)
    frames = [C.frame_params(c, tau_px, precision=precision, fixed_shift=20) for c in cams]
    return InstanceSpec("planet", mesh, D, 48, frames)


def config_dodeca(n_frames: int = 300, tau_px: float = 14.0, D: int = 17, max_depth: int = 50,
                  radius: float = 6.371e6) -> InstanceSpec:
    """The paper's planet scene shape (Sec. 4 and Table 3): a regular
    dodecahedron base (60 halfedges) on an Earth-sized sphere, pool 2^17,
    vertices projected onto the sphere during refinement, triangles of about
    49 px (a refinement edge of 14 px), a seeded descent from 2e7 m to 2 m
    above the sphere."""
    mesh = M.dodecahedron_mesh(radius)
    cams = C.sphere_descent_path(mesh, radius, n_frames, seed=17)
    frames = [C.frame_params(c, tau_px, precision=C.PREC_SPHERE, sphere_radius=radius) for c in cams]
    return InstanceSpec("dodeca-planet", mesh, D, max_depth, frames)


def config4(n_inst: int = 256, n_frames: int = 64, seed: int = 4, tau_px: float = 4.0,
            h_max: int = 40000) -> list[InstanceSpec]:
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(n_inst):
        H = int(np.exp(rng.uniform(np.log(24), np.log(h_max))))
        dsel = int(rng.integers(14, 21))
        sub = int(rng.integers(1 << 30))
        if H < 100:
            mesh = M.cube_mesh()
            maxd = 14
            cams = C.orbit_path(n_frames, seed=sub)
        else:
            mesh = M.grid_for_halfedges(H, seed=sub)
            maxd = 26
            cams = C.flythrough_path(n_frames, seed=sub)
        D = max(dsel, ceil_log2(mesh.H) + 2)
        frames = [C.frame_params(c, tau_px) for c in cams]
        specs.append(InstanceSpec(f"b{k}-{mesh.name}", mesh, D, maxd, frames))
    return specs


def config5(n_inst: int = 1024, n_planets: int = 8, n_frames: int = 64, seed: int = 5):
    specs = config4(n_inst=n_inst, n_frames=n_frames, seed=seed)
    for k in range(n_planets):
        p = config3(n_frames=n_frames)
        p.name = f"planet{k}"
        specs.append(p)
    return specs


def _displaced(spec: InstanceSpec, amp: float, freq: float, octaves: int, seed: int) -> InstanceSpec:
    for fp in spec.frames:
        fp.disp_amplitude, fp.disp_frequency, fp.disp_octaves, fp.disp_seed = amp, freq, octaves, seed
    return spec


def config_terrain(n_frames: int = 120, tau_px: float = 2.0, nx: int = 100, D: int = 20, amp: float = 0.02,
                   freq: float = 4.0, octaves: int = 6, seed: int = 23) -> InstanceSpec:
    """Config 2's grid flythrough with the surface displaced: z grows by
    amp * fbm(world x, y), a 6-octave value noise from 4 to 128 cells per
    unit, standing in for the paper's elevation data plus noise octaves
    (Sec. 4). The LOD test sees the displaced vertices."""
    mesh = M.grid_mesh(nx, nx, tri_frac=0.1, seed=2, height_sigma=0.05)
    cams = C.flythrough_path(n_frames, seed=2)
    frames = [C.frame_params(c, tau_px) for c in cams]
    return _displaced(InstanceSpec("terrain", mesh, D, 26, frames), amp, freq, octaves, seed)


def config_waves(n_frames: int = 300, tau_px: float = 14.0, D: int = 17, max_depth: int = 50,
                 radius: float = 6.371e6, amp: float = 2.0, freq: float = 6371.0, octaves: int = 4,
                 seed: int = 29) -> InstanceSpec:
    """The paper's water planet (Sec. 4): the dodecahedron planet with the
    projected vertices displaced radially by amp * fbm(unit direction), a
    4-octave value noise with cells of 1 km down to 125 m, standing in for
    its four FFT wave layers."""
    spec = config_dodeca(n_frames, tau_px, D, max_depth, radius)
    spec.name = "wave-planet"
    return _displaced(spec, amp, freq, octaves, seed)

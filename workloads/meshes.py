"""Seeded synthetic polygon meshes given as face lists.

This module only produces inputs: vertex positions and faces (lists of vertex
indices in counter-clockwise order seen from outside). It holds none of the
method's arithmetic; the conversion of faces into a halfedge mesh, the root
bisectors and everything after belong to the two implementations (the oracle
and the CUDA library), each with its own code.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class PolyMesh:
    """A polygon mesh: ``face_sizes[f]`` vertices per face, concatenated in
    ``face_verts``; ``pos`` is float64 ``[V, 3]``. ``fp32`` says the mesh is
    meant to be handed over as FP32 positions (``pos`` then holds values
    exactly representable in FP32)."""

    name: str
    face_sizes: np.ndarray
    face_verts: np.ndarray
    pos: np.ndarray
    fp32: bool = True

    @property
    def H(self) -> int:
        return int(self.face_sizes.sum())

    @property
    def V(self) -> int:
        return int(self.pos.shape[0])

    @property
    def F(self) -> int:
        return int(self.face_sizes.shape[0])


def _mesh(name, faces, pos, fp32=True) -> PolyMesh:
    sizes = np.asarray([len(f) for f in faces], dtype=np.int32)
    verts = np.asarray([v for f in faces for v in f], dtype=np.int32)
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    if fp32:
        pos = pos.astype(np.float32).astype(np.float64)
    return PolyMesh(name, sizes, verts, pos, fp32)


def fig1_mesh() -> PolyMesh:
    """The 12-halfedge example of the paper's halfedge figure (Fig. 1): a quad
    (3,2,1,0), a triangle (3,4,2) and a pentagon (1,2,4,5,6). The figure's
    vertex coordinates are not part of the text, so a convex planar layout
    with the same connectivity is used."""
    faces = [[3, 2, 1, 0], [3, 4, 2], [1, 2, 4, 5, 6]]
    pos = [(0, 1, 0), (1, 1, 0), (1, 0, 0), (0, 0, 0), (1.5, -1, 0), (3, -1, 0), (3, 1, 0)]
    return _mesh("fig1", faces, pos)


def cube_mesh(half: float = 0.5) -> PolyMesh:
    """Axis-aligned cube ``[-half, half]^3``: 6 quads, 24 halfedges."""
    p = []
    for i in range(8):
        p.append(((i & 1) * 2 - 1, ((i >> 1) & 1) * 2 - 1, ((i >> 2) & 1) * 2 - 1))
    p = np.asarray(p, dtype=np.float64) * half
    faces = [
        [0, 2, 3, 1],  # z = -half (normal -z)
        [4, 5, 7, 6],  # z = +half
        [0, 1, 5, 4],  # y = -half
        [2, 6, 7, 3],  # y = +half
        [0, 4, 6, 2],  # x = -half
        [1, 3, 7, 5],  # x = +half
    ]
    return _mesh("cube", faces, p)


def tetra_mesh() -> PolyMesh:
    """Regular tetrahedron: 4 triangles, 12 halfedges, closed."""
    p = [(1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)]
    faces = [[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]]
    return _mesh("tetra", faces, p)


def grid_mesh(nx: int, ny: int, tri_frac: float = 0.1, seed: int = 2,
              height_sigma: float = 0.05, name: str | None = None) -> PolyMesh:
    """``nx`` x ``ny`` cells on the unit square with an open border. Each cell
    is a quad, except a seeded fraction ``tri_frac`` split into two triangles
    along a seeded diagonal. Heights ~ N(0, height_sigma), FP32."""
    rng = np.random.default_rng(seed)
    xs = np.arange(nx + 1) / nx
    ys = np.arange(ny + 1) / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    Z = rng.normal(0.0, height_sigma, size=X.shape) if height_sigma > 0 else np.zeros_like(X)
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(i, j):
        return j * (nx + 1) + i

    split = rng.random((ny, nx)) < tri_frac
    diag = rng.random((ny, nx)) < 0.5
    faces = []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            if not split[j, i]:
                faces.append([a, b, c, d])
            elif diag[j, i]:
                faces.append([a, b, c])
                faces.append([a, c, d])
            else:
                faces.append([a, b, d])
                faces.append([b, c, d])
    return _mesh(name or f"grid{nx}x{ny}", faces, pos)


def grid_for_halfedges(H_target: int, seed: int, tri_frac: float = 0.1) -> PolyMesh:
    """A grid whose halfedge count is close to ``H_target`` (about 4.2 per cell)."""
    cells = max(1.0, H_target / (4.0 * (1.0 + 0.5 * tri_frac)))
    n = max(1, int(round(np.sqrt(cells))))
    return grid_mesh(n, n, tri_frac=tri_frac, seed=seed, name=f"grid{n}x{n}")


def cube_sphere_mesh(n: int = 8, radius: float = 6.371e6) -> PolyMesh:
    """Cube-sphere: 6 faces x n x n quads whose vertices lie on a sphere of the
    given radius, FP64 positions (6 * n * n * 4 halfedges; 1536 for n = 8)."""
    index = {}
    pos = []

    def vid(p):
        key = tuple(int(v) for v in p)
        if key not in index:
            index[key] = len(pos)
            q = np.asarray(key, dtype=np.float64) - n / 2.0
            pos.append(q / np.linalg.norm(q) * radius)
        return index[key]

    faces = []
    # Each cube face: a fixed axis at 0 or n, two running axes (u, v) with
    # u x v pointing outward.
    for axis in range(3):
        for side in (0, n):
            u_ax, v_ax = (axis + 1) % 3, (axis + 2) % 3
            outward = 1 if side == n else -1
            for a in range(n):
                for b in range(n):
                    def P(du, dv):
                        p = [0, 0, 0]
                        p[axis] = side
                        p[u_ax] = a + du
                        p[v_ax] = b + dv
                        return p
                    quad = [vid(P(0, 0)), vid(P(1, 0)), vid(P(1, 1)), vid(P(0, 1))]
                    if outward < 0:
                        quad = quad[::-1]
                    faces.append(quad)
    return _mesh(f"cubesphere{n}", faces, np.asarray(pos), fp32=False)


def dodecahedron_mesh(radius: float = 6.371e6) -> PolyMesh:
    """Regular dodecahedron inscribed in a sphere of the given radius: 20
    vertices, 12 planar pentagons (60 halfedges), outward counter-clockwise
    faces, FP64 positions. Each face is the five vertices farthest along one
    of the 12 directions (0, +-phi, +-1) and their cyclic permutations."""
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(x, y, z) for x in (-1.0, 1.0) for y in (-1.0, 1.0) for z in (-1.0, 1.0)]
    for a in (-1.0 / phi, 1.0 / phi):
        for b in (-phi, phi):
            v += [(0.0, a, b), (a, b, 0.0), (b, 0.0, a)]
    pos = np.asarray(v, np.float64) * (radius / 3.0 ** 0.5)
    normals = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            normals += [(0.0, b, a), (b, a, 0.0), (a, 0.0, b)]
    faces = []
    for n in np.asarray(normals, np.float64):
        n = n / np.linalg.norm(n)
        d = pos @ n
        idx = np.argsort(-d)[:5]
        c = pos[idx].mean(0)
        e1 = pos[idx[0]] - c
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(n, e1)
        ang = np.arctan2((pos[idx] - c) @ e2, (pos[idx] - c) @ e1)
        faces.append([int(k) for k in idx[np.argsort(ang)]])
    return _mesh("dodecahedron", faces, pos, fp32=False)

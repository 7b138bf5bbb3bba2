"""Synthetic triangle meshes shaped like the paper's workloads.

The paper's scanned models are not available, so three families stand in:

* ``icosphere(level)``: regular icosahedron (vertices at the cyclic
  permutations of (0, +-1, +-phi)) refined ``level`` times by midpoint
  subdivision, every new vertex projected to the unit sphere;
  10 * 4**level + 2 vertices.
* ``planar_grid(n, jitter, seed)``: n x n unit-spacing grid in the z = 0 plane,
  each cell split along its main diagonal when (i + j) is even and along the
  anti-diagonal otherwise, every vertex moved in x and y by U(-jitter, +jitter).
* ``noisy_torus(n, ...)``: periodic (u, v) grid on the torus of radii R, r with
  the same alternating split, displaced along the tube normal by
  ``amp * noise(u, v)`` with ``noise`` a 4-octave periodic value noise.

All triangles are counter-clockwise seen from outside (from +z for the grid).
Vertex (i, j) of a grid-like mesh has index ``j * n + i``.
"""
from dataclasses import dataclass, field
from itertools import combinations

import numpy as np

from .rng import uniform, uniform01


@dataclass
class Mesh:
    V: np.ndarray          # (n_v, 3) float64
    F: np.ndarray          # (n_f, 3) int32, 0-based, CCW
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_v(self):
        return int(self.V.shape[0])

    @property
    def n_f(self):
        return int(self.F.shape[0])


def _icosahedron():
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    pts = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            pts.append((0.0, a, b))
            pts.append((a, b, 0.0))
            pts.append((b, 0.0, a))
    V = np.array(pts, dtype=np.float64)
    # faces = vertex triples whose three sides all have the edge length 2
    faces = []
    for a, b, c in combinations(range(12), 3):
        d = [np.linalg.norm(V[a] - V[b]), np.linalg.norm(V[b] - V[c]), np.linalg.norm(V[c] - V[a])]
        if all(abs(x - 2.0) < 1e-9 for x in d):
            n = np.cross(V[b] - V[a], V[c] - V[a])
            if np.dot(n, V[a] + V[b] + V[c]) < 0:
                b, c = c, b
            faces.append((a, b, c))
    F = np.array(faces, dtype=np.int64)
    assert F.shape == (20, 3)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    return V, F


def _subdivide(V, F):
    n = V.shape[0]
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    uniq, inv = np.unique(e, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    m = F.shape[0]
    ab = n + inv[0:m]
    bc = n + inv[m:2 * m]
    ca = n + inv[2 * m:3 * m]
    mid = 0.5 * (V[uniq[:, 0]] + V[uniq[:, 1]])
    mid /= np.linalg.norm(mid, axis=1, keepdims=True)
    V2 = np.concatenate([V, mid], axis=0)
    a, b, c = F[:, 0], F[:, 1], F[:, 2]
    F2 = np.concatenate([
        np.stack([a, ab, ca], 1),
        np.stack([ab, b, bc], 1),
        np.stack([ca, bc, c], 1),
        np.stack([ab, bc, ca], 1),
    ], axis=0)
    return V2, F2


def icosphere(level, radius=1.0):
    V, F = _icosahedron()
    for _ in range(level):
        V, F = _subdivide(V, F)
    return Mesh(V * radius, F.astype(np.int32), name=f"icosphere{level}",
                meta={"kind": "icosphere", "level": level, "radius": radius})


def _grid_faces(nx, ny, periodic):
    """Two triangles per cell; main diagonal when (i + j) is even."""
    ci = np.arange(nx if periodic else nx - 1)
    cj = np.arange(ny if periodic else ny - 1)
    I, J = np.meshgrid(ci, cj, indexing="xy")
    I = I.reshape(-1)
    J = J.reshape(-1)
    I1 = (I + 1) % nx
    J1 = (J + 1) % ny
    v00 = J * nx + I
    v10 = J * nx + I1
    v01 = J1 * nx + I
    v11 = J1 * nx + I1
    even = ((I + J) % 2) == 0
    t1 = np.where(even[:, None], np.stack([v00, v10, v11], 1), np.stack([v00, v10, v01], 1))
    t2 = np.where(even[:, None], np.stack([v00, v11, v01], 1), np.stack([v10, v11, v01], 1))
    F = np.empty((2 * I.size, 3), dtype=np.int64)
    F[0::2] = t1
    F[1::2] = t2
    return F.astype(np.int32)


def planar_grid(n, jitter=0.2, seed=2, spacing=1.0):
    i = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(i, i, indexing="xy")
    V = np.zeros((n * n, 3), dtype=np.float64)
    V[:, 0] = X.reshape(-1)
    V[:, 1] = Y.reshape(-1)
    if jitter:
        d = uniform(seed, 2 * n * n, -jitter, jitter).reshape(n * n, 2)
        V[:, :2] += d
    V *= spacing
    return Mesh(V, _grid_faces(n, n, periodic=False), name=f"grid{n}",
                meta={"kind": "grid", "n": n, "jitter": jitter, "seed": seed})


def _smoothstep(f):
    return f * f * (3.0 - 2.0 * f)


def value_noise(s, t, seed=4, octaves=4, base=8):
    """Periodic value noise on the unit square, values in [-1, 1].

    Octave o has a (base * 2**o)-cell lattice and weight 2**-o; lattice values
    are 2u - 1 with u drawn from stream ``seed`` at counter
    (o * 1024 + ix) * 1024 + iy; cells are blended with the smoothstep
    f^2 (3 - 2f) and the weighted sum is divided by the sum of weights.
    """
    s = np.asarray(s, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros(np.broadcast(s, t).shape)
    wsum = 0.0
    for o in range(octaves):
        P = base * (2 ** o)
        amp = 2.0 ** (-o)
        x = s * P
        y = t * P
        ix = np.floor(x).astype(np.int64)
        iy = np.floor(y).astype(np.int64)
        fx = _smoothstep(x - ix)
        fy = _smoothstep(y - iy)

        def h(a, b):
            a = a % P
            b = b % P
            ctr = ((o * 1024 + a) * 1024 + b).astype(np.uint64)
            return 2.0 * uniform01(seed, ctr) - 1.0

        v00 = h(ix, iy)
        v10 = h(ix + 1, iy)
        v01 = h(ix, iy + 1)
        v11 = h(ix + 1, iy + 1)
        out += amp * ((v00 * (1 - fx) + v10 * fx) * (1 - fy) + (v01 * (1 - fx) + v11 * fx) * fy)
        wsum += amp
    return out / wsum


def noisy_torus(n, R=1.0, r=0.35, amp=0.02, seed=4, octaves=4):
    i = np.arange(n, dtype=np.float64)
    S, T = np.meshgrid(i / n, i / n, indexing="xy")
    S = S.reshape(-1)
    T = T.reshape(-1)
    u = 2.0 * np.pi * S
    v = 2.0 * np.pi * T
    nrm = np.stack([np.cos(v) * np.cos(u), np.cos(v) * np.sin(u), np.sin(v)], 1)
    ctr = np.stack([R * np.cos(u), R * np.sin(u), np.zeros_like(u)], 1)
    disp = r + (amp * value_noise(S, T, seed=seed, octaves=octaves) if amp else 0.0)
    V = ctr + nrm * np.reshape(disp, (-1, 1))
    return Mesh(V, _grid_faces(n, n, periodic=True), name=f"torus{n}",
                meta={"kind": "torus", "n": n, "R": R, "r": r, "amp": amp, "seed": seed})


def shuffled(mesh, seed=21):
    """The same mesh with its vertices renumbered by a seeded random
    permutation (faces keep their orientation): a numbering without locality,
    as a scan or an edited mesh may have."""
    u = uniform01(seed, np.arange(mesh.n_v, dtype=np.uint64))
    old_of_new = np.argsort(u, kind="stable")
    new_of_old = np.empty_like(old_of_new)
    new_of_old[old_of_new] = np.arange(mesh.n_v)
    return Mesh(np.ascontiguousarray(mesh.V[old_of_new]), new_of_old[mesh.F].astype(np.int32),
                name=mesh.name, meta={"new_of_old": new_of_old})

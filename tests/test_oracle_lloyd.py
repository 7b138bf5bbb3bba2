"""Pins of the Lloyd-like reseeding oracle (Sec. 5) against geometry fixed
independently of it: the shoelace centroid of a planar region, exact line-
triangle intersections, a ring-shaped cell whose centre of mass misses it,
conflict cases worked by hand, and the paper's claim that the iterations
balance the cells."""
import numpy as np
import pytest

import synth
from oracle import tessellation as tz


class Field:
    def __init__(self, rowptr, ids, vals):
        self.rowptr, self.ids, self.vals = (np.asarray(rowptr, np.int64), np.asarray(ids, np.int32),
                                            np.asarray(vals, np.float64))


def field_from_labels(lab, k):
    """One entry per vertex: the cell of the label, or the base layer k for -1."""
    n = len(lab)
    ids = np.where(lab < 0, k, lab)
    return Field(np.arange(n + 1), ids, np.ones(n))


def shoelace_centroid(P):
    x, y = P[:, 0], P[:, 1]
    x1, y1 = np.roll(x, -1), np.roll(y, -1)
    cr = x * y1 - x1 * y
    A = cr.sum() / 2.0
    return np.array([((x + x1) * cr).sum() / (6 * A), ((y + y1) * cr).sum() / (6 * A)])


def boundary_loop(n, V):
    """Boundary vertices of the n x n grid in counter-clockwise order."""
    b = [0 * n + i for i in range(n)]                       # bottom, j = 0
    b += [j * n + (n - 1) for j in range(1, n)]             # right
    b += [(n - 1) * n + i for i in range(n - 2, -1, -1)]    # top
    b += [j * n + 0 for j in range(n - 2, 0, -1)]           # left
    return V[b, :2]


def test_line_hit_closed_forms():
    a, b, c = np.array([0.0, 0, 0]), np.array([2.0, 0, 0]), np.array([0.0, 2, 0])
    s, u, v = tz.line_hit(np.array([0.5, 0.5, 3.0]), np.array([0, 0, 1.0]), a, b, c)
    assert s == pytest.approx(-3.0) and u == pytest.approx(0.25) and v == pytest.approx(0.25)
    s, u, v = tz.line_hit(np.array([0.5, 0.5, -1.0]), np.array([0, 0, -1.0]), a, b, c)
    assert s == pytest.approx(-1.0)                          # behind the origin counts: a line
    assert tz.line_hit(np.array([0, 0, 1.0]), np.array([1.0, 0, 0]), a, b, c) is None   # parallel
    assert tz.line_hit(np.array([1.5, 1.5, 1.0]), np.array([0, 0, 1.0]), a, b, c) is None
    h = tz.line_hit(np.array([0.0, 0, 1.0]), np.array([0, 0, 1.0]), a, b, c)          # at a vertex
    assert h is not None and h[1] == 0.0 and h[2] == 0.0


def test_geometry_of_a_right_triangle():
    V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    area, bary, normal = tz.triangle_geometry(V, np.array([[0, 1, 2]]))
    assert area[0] == 0.5 and np.allclose(bary[0], [1 / 3, 1 / 3, 0]) and np.allclose(normal[0], [0, 0, 1])


@pytest.mark.parametrize("jitter", [0.0, 0.2])
def test_whole_mesh_cell_has_the_shoelace_centroid(jitter):
    n = 15
    m = synth.planar_grid(n, jitter=jitter, seed=2)
    F = field_from_labels(np.zeros(m.n_v, np.int64), 1)
    (P, d, ts), = tz.cell_frames(m.V, m.F, F, 1)
    assert len(ts) == m.n_f
    assert np.allclose(P[:2], shoelace_centroid(boundary_loop(n, m.V)), atol=1e-12)
    assert P[2] == 0.0 and np.allclose(d, [0, 0, 1])
    # the line meets the plane at the centroid: the new seed is the nearest
    # corner of the triangle containing it (found here by brute force)
    new = tz.lloyd_seeds(m.V, m.F, F, [0])
    X = P[:2]
    for t in range(m.n_f):
        A, B, C = (m.V[m.F[t, j], :2] for j in range(3))
        M = np.array([B - A, C - A]).T
        u, v = np.linalg.solve(M, X - A)
        if u >= 0 and v >= 0 and u + v <= 1:
            break
    corners = sorted((np.linalg.norm(m.V[m.F[t, j], :2] - X), int(m.F[t, j])) for j in range(3))
    assert new[0] == corners[0][1]
    if jitter == 0.0:
        assert new[0] == (n // 2) * n + n // 2               # the central vertex


def test_ring_cell_misses_and_keeps_its_seed():
    n = 21
    m = synth.planar_grid(n, jitter=0.0)
    i, j = np.meshgrid(np.arange(n), np.arange(n))
    r = np.hypot(i - 10, j - 10).ravel()
    lab = np.where((r >= 6) & (r <= 8), 0, -1)              # an annulus: its centroid is in the hole
    F = field_from_labels(lab, 1)
    seed = int(np.flatnonzero(lab == 0)[0])
    (P, d, ts), = tz.cell_frames(m.V, m.F, F, 1)
    assert np.allclose(P[:2], [10, 10], atol=1e-9)
    assert tz.lloyd_seeds(m.V, m.F, F, [seed])[0] == seed


def test_conflicts_worked_by_hand():
    assert list(tz.resolve_conflicts([1, 2, 3], [5, 5, 7])) == [5, 2, 7]
    assert list(tz.resolve_conflicts([1, 2, 3], [2, 2, 9])) == [1, 2, 9]      # cell 1 holds its own seed
    assert list(tz.resolve_conflicts([1, 2, 3], [3, 1, 3])) == [1, 2, 3]      # a chain of returns
    assert list(tz.resolve_conflicts([4, 5, 6], [7, 8, 9])) == [7, 8, 9]


def test_sphere_cap_projects_back_onto_the_cap():
    m = synth.icosphere(3)
    lab = np.where(m.V[:, 2] > 0.6, 0, -1)
    F = field_from_labels(lab, 1)
    (P, d, ts), = tz.cell_frames(m.V, m.F, F, 1)
    assert abs(P[0]) < 0.02 and abs(P[1]) < 0.02 and 0.6 < P[2] < 1.0     # inside the sphere
    assert d[2] > 0.999
    new = tz.lloyd_seeds(m.V, m.F, F, [int(np.argmin(m.V[:, 2]))])
    top = m.V[new[0]]
    assert top[2] > 0.97 and lab[new[0]] == 0


def test_lloyd_rounds_balance_the_cells(oracle_mod):
    # seeds crowded into one corner of a planar grid: a few Lloyd-like rounds
    # spread them, so the cell sizes grow more even (Sec. 5, Fig. on the
    # area distributions)
    n, k = 40, 12
    m = synth.planar_grid(n, jitter=0.2, seed=2)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    corner = [j * n + i for j in range(8) for i in range(8)]
    seeds = np.array(corner[::5][:k])

    def sizes(seeds):
        F = oracle_mod.seed(m.n_v, seeds)
        for _ in range(120):
            F, _ = oracle_mod.step(L, F)
        lab = oracle_mod.labels(F)
        return F, np.bincount(lab[lab >= 0], minlength=k)

    F, s0 = sizes(seeds)
    for _ in range(4):
        seeds = tz.lloyd_seeds(m.V, m.F, F, seeds)
        assert len(set(seeds.tolist())) == k
        F, s1 = sizes(seeds)
    assert s1.std() / s1.mean() < 0.6 * (s0.std() / s0.mean())


def test_symmetric_seeds_are_stationary(oracle_mod):
    # the 12 icosahedron vertices as seeds on the subdivided icosahedron: each
    # cell is symmetric about its seed's axis, so its centre of mass and normal
    # lie on that axis and the back-projection returns the seed itself
    m = synth.icosphere(3)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    seeds = np.arange(12)
    F = oracle_mod.seed(m.n_v, seeds)
    for _ in range(60):
        F, _ = oracle_mod.step(L, F)
    frames = tz.cell_frames(m.V, m.F, F, 12)
    for c, (P, d, ts) in enumerate(frames):
        axis = m.V[c] / np.linalg.norm(m.V[c])
        assert abs(abs(d @ axis) - 1.0) < 1e-3          # normal along the seed axis
    assert np.array_equal(tz.lloyd_seeds(m.V, m.F, F, seeds), seeds)

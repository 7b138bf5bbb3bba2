"""Pins of the dual-mesh oracle (Sec. 5.2): isolines and crossings worked by
hand, the two-cell / three-cell face cases fixed by linear algebra, spurious
triangles and orientation on hand-built adjacencies, and -- on converged
fields -- closed manifolds with the Euler characteristic of the surface and,
on the sphere, agreement with the convex hull of the seeds (the Delaunay
triangulation on the sphere the paper compares against in Sec. 3)."""
from collections import Counter

import numpy as np
import pytest

import synth
from oracle import dual


def test_isoline_closed_forms():
    a, b = dual.isoline([1.0, 0.0, 0.0], 0.25)
    assert np.allclose(sorted([tuple(a), tuple(b)]), [(0.0, 0.75), (0.75, 0.0)])
    assert dual.isoline([0.1, 0.2, 0.0], 0.25) is None          # all outside
    assert dual.isoline([0.3, 0.9, 0.25], 0.25) is None         # all inside (iso itself is inside)
    a, b = dual.isoline([0.25, 0.0, 0.0], 0.25)                 # a vertex exactly at iso
    assert np.allclose(sorted([tuple(a), tuple(b)]), [(0.0, 0.0), (0.0, 0.0)])


def test_segment_crossings():
    P = lambda x, y: np.array([x, y], float)
    assert dual.segments_cross((P(0, 0), P(1, 1)), (P(0, 1), P(1, 0)))[0]
    assert not dual.segments_cross((P(0, 0), P(1, 0)), (P(0, 1), P(1, 1)))[0]      # parallel
    assert dual.segments_cross((P(0, 0), P(1, 0)), (P(1, 0), P(2, 5)))[0]          # touching end
    assert dual.segments_cross((P(0, 0), P(2, 0)), (P(1, 0), P(3, 0)))[0]          # collinear overlap
    assert not dual.segments_cross((P(0, 0), P(1, 0)), (P(2, 0), P(3, 0)))[0]      # collinear apart


@pytest.mark.parametrize("phi_c", [[1.0, 0.0, 0.0], [1.0, 0.0, 1.0], [0.7, 0.1, 0.4]])
def test_two_cells_summing_to_one_never_cross(phi_c):
    # phi_d = 1 - phi_c: the isolines are the levels 0.25 and 0.75 of one
    # linear function, hence parallel
    phi_d = [1.0 - x for x in phi_c]
    sc, sd = dual.isoline(phi_c, 0.25), dual.isoline(phi_d, 0.25)
    assert sc is None or sd is None or not dual.segments_cross(sc, sd)[0]


def test_three_cells_on_a_face_all_cross():
    phis = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]
    for i in range(3):
        for j in range(i + 1, 3):
            assert dual.segments_cross(dual.isoline(phis[i], 0.25), dual.isoline(phis[j], 0.25))[0]


def test_spurious_triangle_is_removed():
    # a triangular bipyramid: cells 3 and 4 each have the three mutually
    # adjacent neighbours 0, 1, 2, so the clique (0, 1, 2) is spurious
    N = [{1, 2, 3, 4}, {0, 2, 3, 4}, {0, 1, 3, 4}, {0, 1, 2}, {0, 1, 2}]
    assert dual.triangles(N) == [(0, 1, 3), (0, 1, 4), (0, 2, 3), (0, 2, 4), (1, 2, 3), (1, 2, 4)]
    x, edges, dirs, n_vert = topology(dual.triangles(N))
    assert x == 2 and set(edges.values()) == {2}


def test_manifold_check_drops_a_diagonal_of_a_vertex_shared_quad():
    # cells 0..3 around a point, sides from A_v, both diagonals crossing:
    # each diagonal's ends already share two confirmed neighbours
    Av = {(0, 1), (1, 2), (2, 3), (0, 3)}
    N = dual.manifold_filter(Av, {(0, 2), (1, 3)}, 4)
    assert N == [{1, 3}, {0, 2}, {1, 3}, {0, 2}]
    N = dual.manifold_filter(set(), {(0, 2), (1, 3), (0, 1)}, 4)
    assert N[0] == {1, 2} and N[1] == {0, 3}


def test_orientation_of_a_strip():
    tris = [(0, 1, 2), (1, 2, 3), (2, 3, 4)]
    pos = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 2, 0]], float)
    nrm = np.tile([0.0, 0.0, 1.0], (5, 1))
    out, margin = dual.orient_triangles(tris, pos, nrm)
    for a, b, c in out:
        assert np.cross(pos[b] - pos[a], pos[c] - pos[a])[2] > 0
    dirs = Counter()
    for a, b, c in out:
        dirs.update([(a, b), (b, c), (c, a)])
    assert max(dirs.values()) == 1 and margin == pytest.approx(1.0)


def converged(oracle_mod, m, k, sid, steps, lloyd=0):
    """Seeds and field after `steps` steps, then `lloyd` Lloyd-like rounds of
    the same length (Sec. 5), as the paper extracts its dual meshes."""
    from oracle import tessellation as tz
    seeds = synth.sample_seeds(m.n_v, k, sid)
    L = oracle_mod.cotan_laplacian(m.V, m.F)

    def field(s):
        F = oracle_mod.seed(m.n_v, s)
        for _ in range(steps):
            F, _ = oracle_mod.step(L, F)
        return F

    F = field(seeds)
    for _ in range(lloyd):
        seeds = tz.lloyd_seeds(m.V, m.F, F, seeds)
        F = field(seeds)
    return seeds, F


def topology(tri):
    edges = Counter()
    dirs = Counter()
    for a, b, c in tri:
        for u, v in ((a, b), (b, c), (c, a)):
            edges[(min(u, v), max(u, v))] += 1
            dirs[(u, v)] += 1
    n_vert = len(set(np.asarray(tri).ravel().tolist()))
    return n_vert - len(edges) + len(tri), edges, dirs, n_vert


@pytest.mark.parametrize("mesh,k,sid,steps,lloyd,chi", [
    (lambda: synth.icosphere(3), 16, 1, 150, 0, 2),
    (lambda: synth.icosphere(4), 64, 2, 200, 2, 2),
    (lambda: synth.noisy_torus(60), 48, 5, 250, 0, 0),
])
def test_converged_fields_give_closed_oriented_manifolds(oracle_mod, mesh, k, sid, steps, lloyd, chi):
    m = mesh()
    seeds, F = converged(oracle_mod, m, k, sid, steps, lloyd)
    tri = dual.dual_mesh(m.V, m.F, F, seeds)
    x, edges, dirs, n_vert = topology(tri)
    assert n_vert == k and x == chi
    assert set(edges.values()) == {2} and max(dirs.values()) == 1      # manifold, consistently oriented
    if chi == 2:                                                       # sphere: outward normals
        P = m.V[tri]
        n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        assert (np.einsum("ij,ij->i", n, P.mean(1)) > 0).all()


def test_sphere_dual_matches_the_convex_hull(oracle_mod):
    spatial = pytest.importorskip("scipy.spatial")
    m = synth.icosphere(4)
    seeds, F = converged(oracle_mod, m, 64, 2, 200)
    tri = dual.dual_mesh(m.V, m.F, F, seeds)
    hull = spatial.ConvexHull(m.V[seeds])
    hull_sets = {frozenset(int(seeds[i]) for i in s) for s in hull.simplices}
    ours = {frozenset(int(v) for v in t) for t in tri}
    assert len(ours & hull_sets) >= 0.9 * len(hull_sets)

"""Oracle for the Lloyd-like reseeding (Sec. 5) -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy and Python loops, written for small meshes; it shares no code
with the CUDA library.  Only ``tests/`` and the benchmark's CPU leg use it.

One Lloyd-like update of the seeds, in the paper's order (Sec. 5):

1. the vertices of cell c are those with a nonzero entry in the cell's layer
   of the field (the base layer is not a cell);
2. the triangles of the cell are those with at least one cell vertex;
3. its centre of mass is the mean of the triangle barycentres weighted by the
   triangle areas;
4. the back-projection direction is the mean of the triangle normals
   weighted by the areas;
5. the line through the centre of mass along that direction (both ways) is
   intersected with the cell's triangles; of several hits the one closest to
   the centre of mass wins;
6. the new seed is the vertex of the hit triangle nearest to the hit point;
7. a miss keeps the old seed.

Readings where the paper is silent: ties of step 5 go to the lowest triangle
id and of step 6 to the lowest vertex id; a zero direction is a miss; a hit is
the closed triangle (barycentric coordinates >= 0); two cells that pick the
same vertex are separated by the rule in ``resolve_conflicts``.
"""
import numpy as np


def cell_members(F, k):
    """members[v] = sorted list of the cells (layers < k) with F(v, c) > 0."""
    n_v = len(F.rowptr) - 1
    out = []
    for v in range(n_v):
        a, b = F.rowptr[v], F.rowptr[v + 1]
        out.append([int(l) for l, x in zip(F.ids[a:b], F.vals[a:b]) if l < k and x > 0.0])
    return out


def triangle_geometry(V, T):
    """Areas, barycentres and unit normals of the faces (FP64)."""
    V = np.asarray(V, np.float64)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cr = np.cross(b - a, c - a)
    twice = np.sqrt((cr * cr).sum(1))
    area = 0.5 * twice
    bary = (a + b + c) / 3.0
    normal = cr / twice[:, None]
    return area, bary, normal


def line_hit(o, d, a, b, c):
    """Moller-Trumbore for the whole line o + s d against triangle (a, b, c):
    (s, u, v) or None when the line is parallel to the plane or misses the
    closed triangle."""
    e1, e2 = b - a, c - a
    p = np.cross(d, e2)
    det = float(e1 @ p)
    if det == 0.0:
        return None
    tv = o - a
    u = float(tv @ p) / det
    q = np.cross(tv, e1)
    v = float(d @ q) / det
    s = float(e2 @ q) / det
    if u < 0.0 or v < 0.0 or u + v > 1.0:
        return None
    return s, u, v


def cell_triangles(T, F, k):
    """tris_of[c] = ascending ids of the faces with at least one vertex of cell c."""
    mem = cell_members(F, k)
    tris_of = [[] for _ in range(k)]
    for t in range(len(T)):
        cells = set()
        for v in T[t]:
            cells.update(mem[int(v)])
        for c in sorted(cells):
            tris_of[c].append(t)
    return tris_of


def cell_frames(V, T, F, k):
    """Per cell: (centre of mass, unit back-projection direction or None, faces)."""
    V = np.asarray(V, np.float64)
    T = np.asarray(T, np.int64)
    area, bary, normal = triangle_geometry(V, T)
    out = []
    for ts in cell_triangles(T, F, k):
        if not ts:
            out.append((None, None, ts))
            continue
        A = sum(area[t] for t in ts)
        P = sum(area[t] * bary[t] for t in ts) / A
        N = sum(area[t] * normal[t] for t in ts)
        nn = float(np.sqrt(N @ N))
        out.append((P, N / nn if nn > 0.0 else None, ts))
    return out


def candidate_seeds(V, T, F, seeds, margins=False):
    """Steps 1-7 for every cell: the proposed new seed of each cell (before
    conflicts are resolved).  With margins, also per cell the smallest relative
    gap of a decision: of the barycentric tests of the winning hit, between the
    two nearest hits and between the two nearest vertices."""
    V = np.asarray(V, np.float64)
    T = np.asarray(T, np.int64)
    k = len(seeds)
    new = np.array(seeds, np.int64)
    marg = np.full(k, np.inf)
    for c, (P, d, ts) in enumerate(cell_frames(V, T, F, k)):
        if d is None:
            continue
        hits = []
        for t in ts:
            h = line_hit(P, d, V[T[t, 0]], V[T[t, 1]], V[T[t, 2]])
            if h is not None:
                hits.append((abs(h[0]), t, h))
        if not hits:
            continue
        hits.sort(key=lambda x: (x[0], x[1]))
        s_abs, t, (s, u, v) = hits[0]
        X = P + s * d
        dist = [(float(np.sqrt(((V[T[t, j]] - X) ** 2).sum())), int(T[t, j])) for j in range(3)]
        dist.sort()
        new[c] = dist[0][1]
        if margins:
            scale = max(float(np.sqrt(((V[T[t, 1]] - V[T[t, 0]]) ** 2).sum())), 1e-300)
            m = min(u, v, 1.0 - u - v)
            if len(hits) > 1 and hits[1][1] != t:
                m = min(m, (hits[1][0] - s_abs) / scale)
            m = min(m, (dist[1][0] - dist[0][0]) / scale)
            marg[c] = m
    return (new, marg) if margins else new


def resolve_conflicts(old, cand):
    """Distinct seeds from the candidates: while two cells hold the same
    vertex, a cell holding its old seed keeps it and the others return to their
    old seeds; among candidates only, the lowest cell id keeps the vertex.
    Old seeds are distinct, so this ends with distinct seeds."""
    old = np.asarray(old, np.int64)
    cur = np.asarray(cand, np.int64).copy()
    while True:
        owners = {}
        for c, v in enumerate(cur):
            owners.setdefault(int(v), []).append(c)
        changed = False
        for v, cs in owners.items():
            if len(cs) < 2:
                continue
            keep = [c for c in cs if cur[c] == old[c]]
            winner = keep[0] if keep else min(cs)
            for c in cs:
                if c != winner:
                    cur[c] = old[c]
                    changed = True
        if not changed:
            return cur


def lloyd_seeds(V, T, F, seeds):
    """One Lloyd-like seed update (Sec. 5) from the current field."""
    return resolve_conflicts(seeds, candidate_seeds(V, T, F, seeds))

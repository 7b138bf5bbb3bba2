"""Oracle for the dual-mesh extraction (Sec. 5.2) -- TEST INFRASTRUCTURE ONLY.

Plain Python sets and loops over the field, for small meshes; it shares no
code with the CUDA library.  The steps, in the paper's order:

1. threshold the field: a cell covers vertex v when F(v, c) >= iso (cells are
   the layers below k; iso = 0.25 by default);
2. A_v: cells c, d are adjacent when they cover a common vertex;
3. A_t: cells are adjacent when they cover vertices of a common face;
4. pairs of A_t missing from A_v are kept only where the two cells' isolines
   (level iso of the field, linear on each face) cross on one of those faces;
5. manifold check: a kept pair is dropped when c and d already share two or
   more confirmed neighbours; the others join the adjacency;
6. triangles: every three mutually adjacent cells;
7. a cell with exactly three neighbours that are mutually adjacent marks the
   triangle of those three as spurious: it is removed;
8. orientation: breadth-first over triangles sharing an edge, from the first
   triangle of each connected part in sorted order, each neighbour taking the
   opposite direction on the shared edge.

Readings where the paper is silent: the threshold includes iso itself; the
isolines are compared in each face's barycentric plane (crossing is affine
invariant) as closed segments; "confirmed" neighbours in step 5 are those of
A_v (an order of the checks is not given, and if accepted pairs counted, every
edge of a closed triangulation -- which has two common neighbours -- would be
dropped once its two wing edges were in); the first triangle of a part is oriented so
that its normal, from the seed positions, points along the sum of the mesh
normals at its three seed vertices; triangles are returned as seed vertex ids,
sorted by their vertex sets.
"""
from collections import deque

import numpy as np


def covers(F, k, iso):
    """cov[v] = sorted cells c < k with F(v, c) >= iso."""
    n_v = len(F.rowptr) - 1
    return [[int(l) for l, x in zip(F.ids[F.rowptr[v]:F.rowptr[v + 1]], F.vals[F.rowptr[v]:F.rowptr[v + 1]])
             if l < k and x >= iso] for v in range(n_v)]


def value(F, v, c):
    a, b = F.rowptr[v], F.rowptr[v + 1]
    for l, x in zip(F.ids[a:b], F.vals[a:b]):
        if l == c:
            return float(x)
    return 0.0


BARY = [np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([0.0, 1.0])]


def isoline(phi, iso):
    """The segment {phi = iso} of a linear function on the reference triangle,
    or None.  A vertex with phi >= iso counts as inside; exactly two edges then
    change side, or none."""
    pts = []
    for i, j in ((0, 1), (1, 2), (2, 0)):
        si, sj = phi[i] - iso, phi[j] - iso
        if (si >= 0.0) != (sj >= 0.0):
            t = si / (si - sj)
            pts.append((1.0 - t) * BARY[i] + t * BARY[j])
    return (pts[0], pts[1]) if len(pts) == 2 else None


def orient(a, b, c):
    return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])


def segments_cross(p, q):
    """Closed segments p, q in the plane; also the smallest |orientation| met,
    the margin of the decision."""
    (a, b), (c, d) = p, q
    o1, o2, o3, o4 = orient(a, b, c), orient(a, b, d), orient(c, d, a), orient(c, d, b)
    margin = min(abs(o1), abs(o2), abs(o3), abs(o4))
    if o1 == 0.0 and o2 == 0.0:                    # collinear: overlap of the projections
        ax = 0 if abs(b[0] - a[0]) >= abs(b[1] - a[1]) else 1
        lo1, hi1 = sorted((a[ax], b[ax]))
        lo2, hi2 = sorted((c[ax], d[ax]))
        return max(lo1, lo2) <= min(hi1, hi2), margin
    return (o1 * o2 <= 0.0) and (o3 * o4 <= 0.0), margin


def adjacency(T, F, k, iso, margins=False):
    """Steps 1-4: (A_v pairs, confirmed candidate pairs), each a set of (c, d), c < d."""
    cov = covers(F, k, iso)
    Av = set()
    for cs in cov:
        for x in range(len(cs)):
            for y in range(x + 1, len(cs)):
                Av.add((cs[x], cs[y]))
    At_only = {}
    min_margin = np.inf
    for t in range(len(T)):
        vs = [int(v) for v in T[t]]
        cs = sorted(set(cov[vs[0]]) | set(cov[vs[1]]) | set(cov[vs[2]]))
        for x in range(len(cs)):
            for y in range(x + 1, len(cs)):
                pr = (cs[x], cs[y])
                if pr in Av:
                    continue
                segc = isoline([value(F, v, pr[0]) for v in vs], iso)
                segd = isoline([value(F, v, pr[1]) for v in vs], iso)
                hit = False
                if segc is not None and segd is not None:
                    hit, mg = segments_cross(segc, segd)
                    min_margin = min(min_margin, mg)
                At_only[pr] = At_only.get(pr, False) or hit
    cand = {pr for pr, h in At_only.items() if h}
    return (Av, cand, min_margin) if margins else (Av, cand)


def manifold_filter(Av, cand, k):
    """Step 5: the adjacency as neighbour sets."""
    Nv = [set() for _ in range(k)]
    for c, d in Av:
        Nv[c].add(d)
        Nv[d].add(c)
    N = [set(x) for x in Nv]
    for c, d in cand:
        if len(Nv[c] & Nv[d]) >= 2:
            continue
        N[c].add(d)
        N[d].add(c)
    return N


def triangles(N):
    """Steps 6-7: sorted cell triples."""
    k = len(N)
    tri = set()
    for i in range(k):
        for j in N[i]:
            if j <= i:
                continue
            for l in N[i] & N[j]:
                if l > j:
                    tri.add((i, j, l))
    spurious = set()
    for i in range(k):
        if len(N[i]) == 3:
            a, b, c = sorted(N[i])
            if (a, b, c) in tri:
                spurious.add((a, b, c))
    return sorted(tri - spurious)


def vertex_normals(V, T):
    V = np.asarray(V, np.float64)
    n = np.zeros_like(V)
    for t in range(len(T)):
        a, b, c = (V[int(T[t, j])] for j in range(3))
        cr = 0.5 * np.cross(b - a, c - a)
        for j in range(3):
            n[int(T[t, j])] += cr
    return n


def orient_triangles(tris, pos, nrm):
    """Step 8 on sorted cell triples; pos and nrm are per cell.  Returns the
    oriented triples in the same order and the smallest |n . N| of the parts'
    first triangles (the margin of their orientation)."""
    edge_tris = {}
    for ti, (a, b, c) in enumerate(tris):
        for e in ((a, b), (b, c), (a, c)):
            edge_tris.setdefault(e, []).append(ti)
    out = [None] * len(tris)
    margin = np.inf
    for start in range(len(tris)):
        if out[start] is not None:
            continue
        a, b, c = tris[start]
        n = np.cross(pos[b] - pos[a], pos[c] - pos[a])
        s = float(n @ (nrm[a] + nrm[b] + nrm[c]))
        margin = min(margin, abs(s) / max(np.linalg.norm(n) * np.linalg.norm(nrm[a] + nrm[b] + nrm[c]), 1e-300))
        out[start] = (a, b, c) if s >= 0.0 else (a, c, b)
        q = deque([start])
        while q:
            ti = q.popleft()
            x, y, z = out[ti]
            for u, v in ((x, y), (y, z), (z, x)):
                for tj in sorted(edge_tris[(min(u, v), max(u, v))]):
                    if out[tj] is not None:
                        continue
                    p, r, s3 = tris[tj]
                    # the neighbour must run v -> u; (p, r, s3) or its reverse
                    cyc = [(p, r), (r, s3), (s3, p)]
                    out[tj] = (p, r, s3) if (v, u) in cyc else (p, s3, r)
                    q.append(tj)
    return out, margin


def dual_mesh(V, T, F, seeds, iso=0.25, margins=False):
    """Steps 1-8: oriented triangles over seed vertex ids, (n, 3) int64."""
    T = np.asarray(T, np.int64)
    k = len(seeds)
    Av, cand, m_iso = adjacency(T, F, k, iso, margins=True)
    N = manifold_filter(Av, cand, k)
    tris = triangles(N)
    V = np.asarray(V, np.float64)
    seeds = np.asarray(seeds, np.int64)
    vn = vertex_normals(V, T)
    oriented, m_or = orient_triangles(tris, V[seeds], vn[seeds])
    out = np.array([[seeds[a], seeds[b], seeds[c]] for a, b, c in oriented], np.int64).reshape(-1, 3)
    return (out, min(m_iso, m_or)) if margins else out

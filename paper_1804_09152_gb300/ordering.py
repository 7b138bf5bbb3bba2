"""Vertex order for locality of the step kernel's gather (host preprocessing).

The step kernel gives one thread to each vertex, in vertex order, and reads
the rows of its neighbours; those reads hit L1 when neighbouring vertices sit
close together in the numbering.  Generated meshes come in scan order; a
mesh whose numbering is scattered (a scan, a mesh after editing) loses that.
``locality_order`` renumbers a mesh so that the two ends of every edge lie
close together (reverse Cuthill-McKee on the mesh graph, or a Morton curve of
the positions) and sorts its faces by their first vertex in the new order;
the layered-field result is the same partition up to the renumbering (only
the order of additions inside a row of L changes, so values agree to
rounding).  Map seeds with ``new_of_old[seeds]`` and results back with
``values[new_of_old]``.
"""
import numpy as np


def _spread_bits(x):
    """The low 21 bits of x spread to every third bit of a 63-bit code."""
    x = x.astype(np.uint64) & np.uint64(0x1FFFFF)
    x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
    return x


def morton_codes(V):
    """Z-order code of each vertex position (21 bits per axis over the bounding cube)."""
    V = np.asarray(V, dtype=np.float64)
    lo = V.min(axis=0)
    ext = float((V.max(axis=0) - lo).max()) or 1.0
    q = np.floor((V - lo) / ext * (2 ** 21 - 1)).astype(np.int64)
    return _spread_bits(q[:, 0]) | (_spread_bits(q[:, 1]) << np.uint64(1)) | (_spread_bits(q[:, 2]) << np.uint64(2))


def rcm_order(n_v, F):
    """Reverse Cuthill-McKee order of the mesh graph (scipy's implementation):
    breadth-first level sets from a peripheral vertex, reversed, which keeps
    every edge's two ends close in the numbering (small bandwidth)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]).astype(np.int64)
    A = sp.coo_matrix((np.ones(len(e), np.int8), (e[:, 0], e[:, 1])), shape=(n_v, n_v)).tocsr()
    A = ((A + A.T) > 0).astype(np.int8).tocsr()
    return np.asarray(reverse_cuthill_mckee(A, symmetric_mode=True), dtype=np.int64)


def locality_order(V, F, method="rcm"):
    """Returns (V_new, F_new, new_of_old): the mesh renumbered (method "rcm":
    reverse Cuthill-McKee on the mesh graph; "morton": along a Morton curve of
    the positions, ties by old id) with its faces sorted by their smallest new
    vertex id, and the map from old to new vertex ids."""
    V = np.asarray(V, dtype=np.float64)
    F = np.asarray(F, dtype=np.int32)
    if method == "rcm":
        old_of_new = rcm_order(V.shape[0], F)
    elif method == "morton":
        old_of_new = np.argsort(morton_codes(V), kind="stable")
    else:
        raise ValueError(f"unknown method {method!r}")
    new_of_old = np.empty_like(old_of_new)
    new_of_old[old_of_new] = np.arange(V.shape[0])
    F_new = new_of_old[F].astype(np.int32)
    F_new = F_new[np.argsort(F_new.min(axis=1), kind="stable")]
    return np.ascontiguousarray(V[old_of_new]), np.ascontiguousarray(F_new), new_of_old.astype(np.int32)

"""Pins of the region-seed initialisation (Sec. 3.2): a seed's immediate
neighbours, read from the faces (not from the operator), take its layer; the
own seed wins at a seed vertex, the lowest seed id elsewhere."""
import numpy as np

import synth


def neighbours_from_faces(F, n_v):
    nb = [set() for _ in range(n_v)]
    for a, b, c in F:
        for x, y in ((a, b), (b, c), (c, a)):
            nb[x].add(int(y))
            nb[y].add(int(x))
    return nb


def test_ring_zero_is_the_point_seed(oracle_mod):
    m = synth.icosphere(2)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    seeds = synth.sample_seeds(m.n_v, 8, 1)
    a, b = oracle_mod.seed_regions(L, seeds, 0), oracle_mod.seed(m.n_v, seeds)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.ids, b.ids) and np.array_equal(a.vals, b.vals)


def test_rings_follow_the_faces_and_the_tie_rules(oracle_mod):
    m = synth.icosphere(2)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    nb = neighbours_from_faces(m.F, m.n_v)
    a = 0
    b = sorted(nb[a])[0]                      # two adjacent seeds: their rings overlap
    far = max(range(m.n_v), key=lambda v: np.linalg.norm(m.V[v] - m.V[a]))
    seeds = [far, b, a]                       # ids: far = 0, b = 1, a = 2
    F = oracle_mod.seed_regions(L, seeds, 1)
    k = len(seeds)
    assert F.n_layers == k + 1 and np.all(np.diff(F.rowptr) == 1) and np.all(F.vals == 1.0)
    want = np.full(m.n_v, k)
    for v in range(m.n_v):
        claims = [c for c, s in enumerate(seeds) if v in nb[s]]
        if claims:
            want[v] = min(claims)
    for c, s in enumerate(seeds):
        want[s] = c                           # a seed vertex keeps its own layer
    assert np.array_equal(F.ids, want)
    assert F.ids[a] == 2 and F.ids[b] == 1    # adjacent seeds keep their own layers
    shared = (nb[a] & nb[b]) - {a, b}
    assert shared and all(F.ids[v] == 1 for v in shared)   # the lower id of the two

"""CPU checks of the locality renumbering (paper_1804_09152_gb300.ordering)."""
import numpy as np
import pytest

import synth
from paper_1804_09152_gb300 import ordering


def spread_by_loop(x):
    out = 0
    for b in range(21):
        out |= ((x >> b) & 1) << (3 * b)
    return out


def test_morton_bit_spreading_matches_a_loop():
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 2 ** 21, size=200)
    got = ordering._spread_bits(xs)
    for x, g in zip(xs.tolist(), got.tolist()):
        assert g == spread_by_loop(x)


def test_morton_order_of_a_cube_lattice():
    # on a 4 x 4 x 4 lattice the Z-order code is the interleaved integer coordinate
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij"), -1).reshape(-1, 3)
    codes = ordering.morton_codes(g.astype(np.float64) / 3.0)
    q = np.floor(g / 3.0 * (2 ** 21 - 1)).astype(np.int64)
    want = [spread_by_loop(a) | spread_by_loop(b) << 1 | spread_by_loop(c) << 2 for a, b, c in q.tolist()]
    assert codes.tolist() == want


def edge_spread(F):
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    return float(np.mean(np.abs(e[:, 0] - e[:, 1])))


@pytest.mark.parametrize("method", ["rcm", "morton"])
def test_locality_order_renumbers_without_changing_the_mesh(method):
    m = synth.shuffled(synth.planar_grid(40, seed=2), seed=5)
    V2, F2, new_of_old = ordering.locality_order(m.V, m.F, method)
    assert sorted(new_of_old.tolist()) == list(range(m.n_v))
    assert np.array_equal(V2[new_of_old], m.V)
    # the same faces with the same orientation (cyclic order), renumbered
    def canon(F):
        k = np.argmin(F, axis=1)
        rolled = np.stack([np.roll(f, -i) for f, i in zip(F, k)])
        return sorted(map(tuple, rolled.tolist()))
    assert canon(F2) == canon(new_of_old[m.F])
    # faces sorted by their smallest vertex, and edges short in the new numbering
    assert np.all(np.diff(F2.min(axis=1)) >= 0)
    assert edge_spread(F2) < 0.15 * edge_spread(m.F)


def test_shuffled_keeps_geometry_and_orientation():
    m = synth.icosphere(2)
    s = synth.shuffled(m, seed=9)
    P, Q = m.V[m.F], s.V[s.F]
    n1 = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    n2 = np.cross(Q[:, 1] - Q[:, 0], Q[:, 2] - Q[:, 0])
    assert np.allclose(np.sort(np.linalg.norm(n1, axis=1)), np.sort(np.linalg.norm(n2, axis=1)))
    assert (np.einsum("ij,ij->i", n2, Q.mean(1)) > 0).all()        # still outward

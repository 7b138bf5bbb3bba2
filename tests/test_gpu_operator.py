"""The cotangent operator built on the device (lf_create_mesh) against the oracle's.

lf_get_operator returns the stored off-diagonal entries in FP32.  The pattern
must equal the oracle's off-diagonal pattern exactly (every edge, including
edges of weight 0), and each value must be the oracle's FP64 value rounded to
FP32, within one FP32 rounding (the two FP64 sums may differ in their last
bits).  Cases: closed and open surfaces, obtuse angles (negative weights), a
vertex of high valence, and a vertex that no face uses.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


class Mesh:
    def __init__(self, V, F):
        self.V, self.F, self.n_v = V, F, V.shape[0]


def fan(n):
    """A disk of n triangles around vertex 0 (valence n), rim slightly wavy."""
    t = 2 * np.pi * np.arange(n) / n
    rim = np.stack([np.cos(t), np.sin(t), 0.05 * np.sin(3 * t)], 1)
    V = np.vstack([np.zeros((1, 3)), rim])
    F = np.array([[0, 1 + i, 1 + (i + 1) % n] for i in range(n)], np.int32)
    return Mesh(V, F)


def with_unused_vertex(m):
    V = np.vstack([m.V, [[10.0, 10.0, 10.0]]])
    return Mesh(V, m.F.copy())


CASES = {
    "ico3": lambda: synth.icosphere(3),
    "torus30": lambda: synth.noisy_torus(30),
    "grid41": lambda: synth.planar_grid(41, seed=2),
    "grid_unjittered": lambda: synth.planar_grid(17, jitter=0.0),      # weights exactly 0 on diagonals
    "fan300": lambda: fan(300),
    "unused_vertex": lambda: with_unused_vertex(synth.planar_grid(12, seed=4)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_device_operator_matches_the_oracle(lf, oracle_mod, name):
    m = CASES[name]()
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    rows = np.repeat(np.arange(m.n_v), np.diff(L.rowptr))
    off = L.col != rows
    want_rp = np.zeros(m.n_v + 1, np.int64)
    np.add.at(want_rp, rows[off] + 1, 1)
    want_rp = np.cumsum(want_rp)
    with lf.Mesh(m.V, m.F) as mesh:
        rp, col, val = mesh.get_operator()
        assert mesh.stats()["operator_nnz"] == col.size
    assert np.array_equal(rp, want_rp)
    assert np.array_equal(col, L.col[off])
    w = L.val[off]
    assert np.all(np.abs(val.astype(np.float64) - w) <= np.abs(w) * 2.0 ** -23 + 1e-300)
    # nearly all entries are exactly the FP32 rounding of the oracle's value
    assert np.mean(val == w.astype(np.float32)) > 0.999


def test_device_operator_is_deterministic(lf):
    m = synth.noisy_torus(64)
    outs = []
    for _ in range(3):
        with lf.Mesh(m.V, m.F) as mesh:
            outs.append(mesh.get_operator())
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x, y)

"""GPU parity of the Lloyd-like seed update (Sec. 5) through lf_lloyd.

The oracle and the GPU start from the same field (an oracle trajectory rounded
to FP32) and the same seeds; one update (rounds = 1, no steps after it) must
give the same new seeds.  A cell whose oracle decision is within rounding of
going the other way (hit on a face edge, two hits or two vertices at nearly
the same distance) is a tie; the GPU's per-cell sums are FP64 atomics in
varying order, so such a cell may differ, and so may cells it meets in a
conflict over its candidate vertex (and so on along the chain of conflicts);
every other cell must match.  Longer runs are checked for what holds at any
size.
"""
import numpy as np
import pytest

import synth
from oracle import tessellation as tz
from parity_util import lloyd_differences_explained, to_f32

pytestmark = pytest.mark.gpu

TIE = 1e-9          # relative margin below which a decision is a tie (FP64 sums in varying order)


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


CASES = {
    "ico3": (lambda: synth.icosphere(3), 16, 1, 40),
    "grid61": (lambda: synth.planar_grid(61, seed=2), 64, 3, 60),
    "torus50": (lambda: synth.noisy_torus(50), 48, 5, 60),
    "ico4_early": (lambda: synth.icosphere(4), 200, 7, 3),      # small cells, few steps: exact ties
    "grid30_crowded": (lambda: synth.planar_grid(30, seed=2), 300, 5, 1),   # 16 cells lose a conflict
}


@pytest.mark.parametrize("name", list(CASES))
def test_one_update_matches_the_oracle(lf, oracle_mod, name):
    fac, k, sid, steps = CASES[name]
    m = fac()
    seeds = synth.sample_seeds(m.n_v, k, sid)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = oracle_mod.seed(m.n_v, seeds)
    for _ in range(steps):
        F, _ = oracle_mod.step(L, F)
    F32 = to_f32(F, oracle_mod)
    cand, marg = tz.candidate_seeds(m.V, m.F, F32, seeds, margins=True)
    want = tz.resolve_conflicts(seeds, cand)
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(seeds)
        mesh.set_field(F32.rowptr, F32.ids, F32.vals, F32.n_layers)
        got = mesh.lloyd(1, 0)
        assert np.array_equal(mesh.lloyd(0, 0), got)          # rounds = 0 reports the seeds
    assert len(set(got.tolist())) == k
    ties = np.flatnonzero(marg < TIE)
    bad = np.flatnonzero(got != want)
    if ties.size == 0:
        assert bad.size == 0, (bad, got[bad], want[bad])
    else:
        # a differing cell is a tie, or met a tie cell (or a cell explained
        # so) in a conflict over its candidate
        left = lloyd_differences_explained(got, want, seeds, cand, ties)
        assert not left, (left, got[left], want[left], cand[left])
    assert (got != seeds).any()                                # the update moves seeds


def test_rounds_balance_cells_on_the_gpu(lf):
    # seeds crowded in one corner of a 128 x 128 grid; Lloyd-like rounds
    # spread them (Sec. 5): the coefficient of variation of the cell sizes
    # drops, and every round leaves k distinct seeds
    n, k = 128, 64
    m = synth.planar_grid(n, jitter=0.2, seed=2)
    corner = np.array([j * n + i for j in range(24) for i in range(24)])
    seeds = corner[synth.sample_seeds(corner.size, k, 5)]
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(seeds)
        mesh.step(400)
        lab0 = mesh.labels()
        cv0 = np.bincount(lab0[lab0 >= 0], minlength=k).std() / (m.n_v / k)
        s = seeds
        for _ in range(5):
            s = mesh.lloyd(1, 400)
            assert len(set(s.tolist())) == k and s.min() >= 0 and s.max() < m.n_v
        lab = mesh.labels()
        cv = np.bincount(lab[lab >= 0], minlength=k).std() / (m.n_v / k)
        assert cv < 0.6 * cv0, (cv0, cv)
        assert mesh.stats()["steps"] == 400


def test_lloyd_needs_geometry_and_seeds(lf, oracle_mod):
    m = synth.icosphere(2)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    with lf.Mesh(csr=(L.rowptr, L.col, L.val)) as mesh:
        mesh.seed(synth.sample_seeds(m.n_v, 8, 1))
        with pytest.raises(lf.LFError) as ei:
            mesh.lloyd(1, 0)
        assert ei.value.status == lf.LF_ERR_STATE
    with lf.Mesh(m.V, m.F) as mesh:
        with pytest.raises(lf.LFError) as ei:
            lf.lf_lloyd(mesh.h, 1, 0, 8)
        assert ei.value.status == lf.LF_ERR_STATE                 # no field yet
        mesh.seed(synth.sample_seeds(m.n_v, 8, 1))
        F = oracle_mod.seed(m.n_v, synth.sample_seeds(m.n_v, 5, 2))
        mesh.set_field(F.rowptr, F.ids, F.vals.astype(np.float32), F.n_layers)
        with pytest.raises(lf.LFError) as ei:
            lf.lf_lloyd(mesh.h, 1, 0, 5)
        assert ei.value.status == lf.LF_ERR_STATE                 # seeds of that field unknown
        with pytest.raises(lf.LFError) as ei:
            lf.lf_lloyd(mesh.h, -1, 0, 5)
        assert ei.value.status == lf.LF_ERR_INVALID


def test_symmetric_seeds_are_stationary_on_the_gpu(lf):
    m = synth.icosphere(4)
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(np.arange(12, dtype=np.int32))
        mesh.step(150)
        assert np.array_equal(mesh.lloyd(1, 0), np.arange(12))

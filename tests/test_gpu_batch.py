"""lf_step_batch: several meshes advanced in shared launches.

The batch runs the same per-vertex arithmetic as lf_step in the same order,
so each mesh of a batch must end bit for bit where lf_step alone takes it:
same pattern, same FP32 values, same skeleton and traffic counters.  One
member is also checked against the FP64 oracle directly.  Cases: meshes of
different sizes (ragged last tiles) starting on different buffer parities, a
run long enough for the graph path plus a remainder, the 64-mesh maximum, a
member whose segments overflow and are grown mid-batch, and invalid batches.
"""
import numpy as np
import pytest

import synth
from parity_util import ambiguous_rows, check_compare, compare, field_from_lib, to_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


CASES = [
    # (mesh factory, seeds, seed stream, steps taken before the batch, storage type)
    (lambda: synth.planar_grid(61, seed=2), 64, 3, 0, "f32"),
    (lambda: synth.icosphere(3), 16, 1, 3, "bf16"),
    (lambda: synth.noisy_torus(40), 32, 5, 1, "f32"),
    (lambda: synth.planar_grid(33, seed=7), 24, 9, 2, "f16"),
]


def make(lf, m, k, sid, pre, dtype="f32", **params):
    mesh = lf.Mesh(m.V, m.F, field_dtype=dtype, **params)
    mesh.seed(synth.sample_seeds(m.n_v, k, sid))
    if pre:
        mesh.step(pre)
    return mesh


def assert_same(a, b):
    fa, fb = a.get_field(), b.get_field()
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1]), "pattern differs"
    assert np.array_equal(fa[2], fb[2]), "values differ"
    sa, sb = a.stats(), b.stats()
    for key in ("steps", "nnz", "skeleton_total", "nnz_io_total"):
        assert sa[key] == sb[key], (key, sa[key], sb[key])


def test_batch_matches_lf_step(lf):
    # mixed storage types (one launch chain each) and different step counts:
    # the chunks are 129 (graph + 1), 131 (graph + 3) and 40 steps
    meshes = [fac() for fac, *_ in CASES]
    batch = [make(lf, m, *c[1:]) for m, c in zip(meshes, CASES)]
    alone = [make(lf, m, *c[1:]) for m, c in zip(meshes, CASES)]
    counts = [300, 260, 300, 129]
    lf.lf_step_batch(batch, counts)
    for b, a, n in zip(batch, alone, counts):
        a.step(n)
        assert_same(b, a)
    lf.lf_step_batch(batch, 5)                     # short call: single launches only
    for b, a in zip(batch, alone):
        a.step(5)
        assert_same(b, a)
    for x in batch + alone:
        x.close()


def test_batch_member_against_oracle(lf, oracle_mod):
    # one step of a batch member from an oracle state, the other members busy
    m = synth.planar_grid(61, seed=2)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = oracle_mod.seed(m.n_v, synth.sample_seeds(m.n_v, 64, 3))
    for _ in range(25):
        F, _ = oracle_mod.step(L, F, {})
    F32 = to_f32(F, oracle_mod)
    Fo, sko, mg = oracle_mod.step(L, F32, {}, margins=True)
    target = lf.Mesh(m.V, m.F)
    target.set_field(F32.rowptr, F32.ids, F32.vals, F32.n_layers)
    others = [make(lf, c[0](), *c[1:]) for c in CASES[1:]]
    sk0 = target.stats()["skeleton_total"]
    lf.lf_step_batch([others[0], target] + others[1:], 1)
    skg = target.stats()["skeleton_total"] - sk0
    Fg = field_from_lib(*target.get_field(), F.n_layers, oracle_mod)
    r = compare(Fo, Fg, ambiguous_rows(mg), oracle_mod)
    check_compare(r)
    assert abs(int(skg) - int(sko)) <= 16 * r["disagreeing_rows"], (skg, sko)
    for x in others + [target]:
        x.close()


def test_batch_of_64_meshes(lf):
    m = synth.icosphere(1)                          # 42 vertices: one partial tile each
    dt = lambda i: "bf16" if i % 4 == 1 else "f32"
    batch = [make(lf, m, 4 + i % 5, 100 + i, i % 2, dt(i)) for i in range(64)]
    pick = (0, 1, 31, 62, 63)
    alone = [make(lf, m, 4 + i % 5, 100 + i, i % 2, dt(i)) for i in pick]
    lf.lf_step_batch(batch, 130)
    for i, a in zip(pick, alone):
        a.step(130)
        assert_same(batch[i], a)
    for x in batch + alone:
        x.close()


def test_batch_grows_a_member(lf):
    # the first member (no steps before the batch) starts with one entry per
    # vertex of segment room, so it overflows as soon as a second layer
    # reaches a vertex and is grown and re-run while the other members continue
    meshes = [c[0]() for c in CASES[:3]]
    batch = [make(lf, m, *c[1:], **({"initial_capacity": 1} if i == 0 else {}))
             for i, (m, c) in enumerate(zip(meshes, CASES[:3]))]
    alone = [make(lf, m, *c[1:]) for m, c in zip(meshes, CASES[:3])]
    assert batch[0].stats()["retries"] == 0
    lf.lf_step_batch(batch, 200)
    assert batch[0].stats()["retries"] > 0
    for b, a in zip(batch, alone):
        a.step(200)
        assert_same(b, a)
    for x in batch + alone:
        x.close()


def test_batch_rejects_invalid(lf):
    import ctypes
    m = synth.icosphere(1)
    a = make(lf, m, 4, 1, 0)
    b = make(lf, m, 4, 2, 0)
    unseeded = lf.Mesh(m.V, m.F)
    for bad, counts, status in (([], 3, lf.LF_ERR_INVALID), ([a] * 65, 3, lf.LF_ERR_INVALID),
                                ([a, b, a], 3, lf.LF_ERR_INVALID), ([a, b], [3, -1], lf.LF_ERR_INVALID),
                                ([a, unseeded], 3, lf.LF_ERR_STATE)):
        with pytest.raises(lf.LFError) as ei:
            lf.lf_step_batch(bad, counts)
        assert ei.value.status == status, (len(bad), ei.value)
    arr = (ctypes.c_void_p * 2)(a.h, b.h)
    assert lf._lib.lf_step_batch(arr, 2, None) == lf.LF_ERR_INVALID
    assert a.stats()["steps"] == 0 and b.stats()["steps"] == 0
    lf.lf_step_batch([a, b], 0)
    lf.lf_step_batch([a, b], [0, 2])
    assert a.stats()["steps"] == 0 and b.stats()["steps"] == 2
    for x in (a, b, unseeded):
        x.close()

"""GPU parity of the dual-mesh extraction (Sec. 5.2) through lf_extract_dual.

Both sides start from the same field (an oracle run rounded to FP32) and the
same seeds.  The threshold and isoline decisions use the same FP32 values and
explicitly rounded FP64 arithmetic on both sides, so the triangle lists must
match exactly, orientation included, unless the oracle reports a decision
within rounding of a flip.  At larger sizes the GPU result is checked for the
topology of the surface.
"""
from collections import Counter

import numpy as np
import pytest

import synth
from oracle import dual, tessellation as tz
from parity_util import to_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


def oracle_state(oracle_mod, m, k, sid, steps, lloyd=0):
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
    return np.asarray(seeds), to_f32(F, oracle_mod)


def topology(tri):
    edges, dirs = Counter(), Counter()
    for a, b, c in tri:
        for u, v in ((a, b), (b, c), (c, a)):
            edges[(min(u, v), max(u, v))] += 1
            dirs[(u, v)] += 1
    n_vert = len(set(np.asarray(tri).ravel().tolist()))
    return n_vert - len(edges) + len(tri), edges, dirs


CASES = {
    "ico3": (lambda: synth.icosphere(3), 16, 1, 150, 0),
    "ico4_lloyd": (lambda: synth.icosphere(4), 64, 2, 200, 2),
    "torus60": (lambda: synth.noisy_torus(60), 48, 5, 250, 0),
    "grid61": (lambda: synth.planar_grid(61, seed=2), 64, 3, 120, 0),      # open surface, boundary
    "ico4_random": (lambda: synth.icosphere(4), 64, 2, 200, 0),            # a four-cell junction
}


@pytest.mark.parametrize("name", list(CASES))
def test_dual_matches_the_oracle(lf, oracle_mod, name):
    fac, k, sid, steps, lloyd = CASES[name]
    m = fac()
    seeds, F32 = oracle_state(oracle_mod, m, k, sid, steps, lloyd)
    want, margin = dual.dual_mesh(m.V, m.F, F32, seeds, margins=True)
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(seeds)
        mesh.set_field(F32.rowptr, F32.ids, F32.vals, F32.n_layers)
        got = mesh.extract_dual()
        again = mesh.extract_dual()                       # cached: same answer
    assert np.array_equal(got, again)
    assert margin > 1e-12, margin
    assert got.shape == want.shape and np.array_equal(got, want)


def test_dual_of_a_lloyd_relaxed_sphere_is_a_closed_oriented_surface(lf):
    m = synth.icosphere(6)                                  # 40,962 vertices
    k = 512
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(synth.sample_seeds(m.n_v, k, 9))
        mesh.step(400)
        seeds = mesh.lloyd(2, 400)
        tri = mesh.extract_dual()
    chi, edges, dirs = topology(tri)
    assert set(tri.ravel().tolist()) <= set(seeds.tolist())
    assert chi == 2 and set(edges.values()) == {2} and max(dirs.values()) == 1
    P = m.V[tri]
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    assert (np.einsum("ij,ij->i", n, P.mean(1)) > 0).all()   # outward


def test_dual_errors(lf, oracle_mod):
    m = synth.icosphere(3)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    with lf.Mesh(csr=(L.rowptr, L.col, L.val)) as mesh:
        mesh.seed(synth.sample_seeds(m.n_v, 8, 1))
        with pytest.raises(lf.LFError) as ei:
            mesh.extract_dual()
        assert ei.value.status == lf.LF_ERR_STATE
    with lf.Mesh(m.V, m.F, iso=0.01) as mesh:
        mesh.seed(synth.sample_seeds(m.n_v, 8, 1))
        with pytest.raises(lf.LFError) as ei:
            mesh.extract_dual()
        assert ei.value.status == lf.LF_ERR_INVALID
    import ctypes
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(synth.sample_seeds(m.n_v, 16, 1))
        mesh.step(150)
        n = ctypes.c_int64()
        assert lf._lib.lf_extract_dual(mesh.h, None, 0, ctypes.byref(n)) == lf.LF_OK and n.value > 0
        small = np.zeros((1, 3), np.int32)
        st = lf._lib.lf_extract_dual(mesh.h, small.ctypes.data_as(ctypes.c_void_p), 1, ctypes.byref(n))
        assert st == lf.LF_ERR_CAPACITY and n.value > 1
        bf = lf.Mesh(m.V, m.F, field_dtype="bf16")
        bf.seed(synth.sample_seeds(m.n_v, 16, 1))
        bf.step(150)
        assert bf.extract_dual().shape[0] > 0
        bf.close()

"""General coefficient matrices (Algorithm 1 with any w_jl, a_jl, e_jk) on the GPU.

lf_set_coefficients hands the step kernel dense FP32 matrices; the oracle
takes the same matrices in FP64.  Single-step parity as in test_gpu_parity
(same input state on both sides, element-wise comparison with tie rows
excused by the oracle's margins), on every tier of the kernel: register map,
shared-memory map and the storage-free enumeration of large layer unions.
Also: a batch that mixes a mesh with matrices and one without gives each
mesh its own result bit for bit, and the matrices' lifetime rules.
"""
import numpy as np
import pytest

import synth
from parity_util import ambiguous_rows, check_compare, compare, field_from_lib, to_f32
from test_gpu_parity import check_results, random_field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


CLASS = dict(w_cc=0.2, w_cb=0.0, a_cc=0.04, a_cb=0.04, e_cc=0.0, e_cb=0.5, e_bc=-0.5)


def class_matrices(n, p=CLASS):
    """The class rule written out as dense matrices (base layer n - 1)."""
    cell = np.arange(n) < n - 1
    both = np.outer(cell, cell)
    W = np.where(both, p["w_cc"], p["w_cb"])
    A = np.where(both, p["a_cc"], p["a_cb"])
    E = np.where(both, p["e_cc"], 0.0)
    E[cell, n - 1] = p["e_cb"]
    E[n - 1, cell] = p["e_bc"]
    for M in (W, A, E):
        np.fill_diagonal(M, 0.0)
    return W, A, E


def perturbed(n, seed, scale=0.05):
    """Class matrices plus a seeded asymmetric perturbation, in FP32 values."""
    rng = np.random.default_rng(seed)
    out = []
    for M in class_matrices(n):
        M = M + scale * (rng.random((n, n)) - 0.5)
        out.append(M.astype(np.float32).astype(np.float64))
    return out


def parity_run(lf, oracle, m, seeds, checks, mats):
    W, A, E = mats
    L = oracle.cotan_laplacian(m.V, m.F)
    F = oracle.seed(m.n_v, seeds)
    out = []
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(seeds)
        mesh.set_coefficients(W, A, E)
        for t in range(max(checks) + 1):
            if t in checks:
                F32 = to_f32(F, oracle)
                Fo, sko, mg = oracle.step(L, F32, W=W, A=A, E=E, margins=True)
                mesh.set_field(F32.rowptr, F32.ids, F32.vals, F32.n_layers)
                sk0 = mesh.stats()["skeleton_total"]
                mesh.step(1)
                skg = mesh.stats()["skeleton_total"] - sk0
                Fg = field_from_lib(*mesh.get_field(), F.n_layers, oracle)
                r = compare(Fo, Fg, ambiguous_rows(mg), oracle)
                r.update(t=t, sk_diff=abs(int(skg) - int(sko)))
                out.append(r)
            F, _ = oracle.step(L, F, W=W, A=A, E=E)
    return out


@pytest.mark.parametrize("name,fac,k,sid", [
    ("grid40", lambda: synth.planar_grid(40, seed=8), 30, 4),
    ("ico3", lambda: synth.icosphere(3), 16, 1),
])
def test_general_matrices_single_step_parity(lf, oracle_mod, name, fac, k, sid):
    m = fac()
    mats = perturbed(k + 1, sid)
    res = parity_run(lf, oracle_mod, m, synth.sample_seeds(m.n_v, k, sid), set(range(0, 60, 3)), mats)
    check_results(res)


def test_class_rule_as_matrices_matches_the_oracle_class_step(lf, oracle_mod):
    # the class rule written out as matrices: the general kernel form against
    # the oracle's class step (the same update, another arithmetic form)
    m = synth.noisy_torus(40)
    k = 32
    mats = [M.astype(np.float32).astype(np.float64) for M in class_matrices(k + 1)]
    res = parity_run(lf, oracle_mod, m, synth.sample_seeds(m.n_v, k, 5), set(range(0, 90, 5)), mats)
    check_results(res)


@pytest.mark.parametrize("per_row,n_layers", [(2, 50), (5, 200), (14, 400)])
def test_general_matrices_on_large_layer_unions(lf, oracle_mod, per_row, n_layers):
    # beyond the register map: the shared-memory map and the storage-free
    # enumeration of the union, both with the matrices
    m = synth.planar_grid(20, seed=6)
    rng = np.random.default_rng(100 + per_row)
    rp, ids, vals = random_field(m.n_v, n_layers, per_row, rng)
    W, A, E = perturbed(n_layers, per_row, scale=0.1)
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.set_field(rp, ids, vals, n_layers)
        mesh.set_coefficients(W, A, E)
        mesh.step(1)
        Fg = field_from_lib(*mesh.get_field(), n_layers, oracle_mod)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    Fin = oracle_mod.Field(rp, ids, vals.astype(np.float64), n_layers)
    Fo, _, mg = oracle_mod.step(L, Fin, W=W, A=A, E=E, margins=True)
    r = compare(Fo, Fg, ambiguous_rows(mg), oracle_mod)
    check_compare(r)


def test_one_matrix_keeps_the_class_rule_for_the_others(lf, oracle_mod):
    m = synth.planar_grid(33, seed=7)
    k = 24
    seeds = synth.sample_seeds(m.n_v, k, 9)
    W, _, _ = perturbed(k + 1, 3, scale=0.2)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = oracle_mod.seed(m.n_v, seeds)
    for _ in range(20):
        F, _ = oracle_mod.step(L, F, W=W)
    F32 = to_f32(F, oracle_mod)
    Fo, _, mg = oracle_mod.step(L, F32, W=W, margins=True)
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(seeds)
        mesh.set_coefficients(W=W)
        mesh.set_field(F32.rowptr, F32.ids, F32.vals, F32.n_layers)   # same layer count: kept
        mesh.step(1)
        Fg = field_from_lib(*mesh.get_field(), k + 1, oracle_mod)
    r = compare(Fo, Fg, ambiguous_rows(mg), oracle_mod)
    check_compare(r)


def run_alone(lf, m, seeds, steps, mats=None):
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(seeds)
        if mats is not None:
            mesh.set_coefficients(*mats)
        mesh.step(steps)
        return mesh.get_field()


def test_batch_mixing_general_and_class_meshes_is_bit_exact(lf):
    g = synth.planar_grid(61, seed=2)
    t = synth.noisy_torus(40)
    sg, st = synth.sample_seeds(g.n_v, 64, 3), synth.sample_seeds(t.n_v, 32, 5)
    mats = perturbed(65, 11)
    want_g = run_alone(lf, g, sg, 300, mats)
    want_t = run_alone(lf, t, st, 300)
    a, b = lf.Mesh(g.V, g.F), lf.Mesh(t.V, t.F)
    try:
        a.seed(sg)
        a.set_coefficients(*mats)
        b.seed(st)
        lf.lf_step_batch([a, b], 300)
        for want, mesh in ((want_g, a), (want_t, b)):
            for x, y in zip(want, mesh.get_field()):
                assert np.array_equal(x, y)
    finally:
        a.close()
        b.close()


def test_coefficient_lifetime_and_errors(lf):
    m = synth.icosphere(3)
    seeds = synth.sample_seeds(m.n_v, 16, 1)
    plain = run_alone(lf, m, seeds, 120)
    mats = perturbed(17, 2, scale=0.2)
    general = run_alone(lf, m, seeds, 120, mats)
    assert not all(np.array_equal(x, y) for x, y in zip(plain, general))
    with lf.Mesh(m.V, m.F) as mesh:
        with pytest.raises(lf.LFError) as ei:
            lf.lf_set_coefficients(mesh.h, 17, *mats)             # no field yet
        assert ei.value.status == lf.LF_ERR_STATE
        mesh.seed(seeds)
        with pytest.raises(lf.LFError) as ei:
            lf.lf_set_coefficients(mesh.h, 18, *perturbed(18, 2))  # wrong layer count
        assert ei.value.status == lf.LF_ERR_INVALID
        bad = mats[0].copy()
        bad[3, 4] = np.nan
        with pytest.raises(lf.LFError) as ei:
            mesh.set_coefficients(W=bad)
        assert ei.value.status == lf.LF_ERR_INVALID
        # reseeding with the same k keeps the matrices
        mesh.set_coefficients(*mats)
        mesh.seed(seeds)
        mesh.step(120)
        assert all(np.array_equal(x, y) for x, y in zip(general, mesh.get_field()))
        # all three None: back to the class coefficients, bit for bit
        mesh.set_coefficients()
        mesh.seed(seeds)
        mesh.step(120)
        assert all(np.array_equal(x, y) for x, y in zip(plain, mesh.get_field()))
        # another layer count drops them
        mesh.set_coefficients(*mats)
        mesh.seed(seeds[:15])
        mesh.seed(seeds)
        mesh.step(120)
        assert all(np.array_equal(x, y) for x, y in zip(plain, mesh.get_field()))


def test_reduced_storage_with_matrices_is_bit_exact_in_a_batch(lf):
    # the general form of the BF16 and FP16 kernels: each mesh in a batch
    # (with a class-coefficient FP32 mesh beside them) equals its run alone
    g = synth.planar_grid(61, seed=2)
    t = synth.noisy_torus(40)
    mats = perturbed(33, 12)
    runs = [(g, synth.sample_seeds(g.n_v, 32, 3), "bf16", mats), (t, synth.sample_seeds(t.n_v, 32, 5), "f16", mats),
            (synth.icosphere(3), synth.sample_seeds(642, 16, 1), "f32", None)]
    want = []
    for m, sd, dt, M in runs:
        with lf.Mesh(m.V, m.F, field_dtype=dt) as mesh:
            mesh.seed(sd)
            if M is not None:
                mesh.set_coefficients(*M)
            mesh.step(150)
            want.append(mesh.get_field())
    meshes = [lf.Mesh(m.V, m.F, field_dtype=dt) for m, _, dt, _ in runs]
    try:
        for mesh, (m, sd, dt, M) in zip(meshes, runs):
            mesh.seed(sd)
            if M is not None:
                mesh.set_coefficients(*M)
        lf.lf_step_batch(meshes, 150)
        for mesh, w in zip(meshes, want):
            for x, y in zip(w, mesh.get_field()):
                assert np.array_equal(x, y)
    finally:
        for mesh in meshes:
            mesh.close()

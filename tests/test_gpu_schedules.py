"""The step-kernel schedules and the autotuner.

The five schedules (the step kernel's registers allocated for 4, 5 and 3
resident CTAs per SM; the lean register-tier path with the full step for
the tiles outside its shape; the lean gather with the other tiers per
vertex) must give the same bits on every job, alone and in batches that mix
them; the autotuner (lf_tune) advances the job like lf_step while it times
them.  The cases run through the first steps from the seeds, where most
tiles are outside the lean path's shape, and a crowded mesh where many
vertices stay outside it.
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


CASES = [
    (lambda: synth.planar_grid(61, seed=2), 64, 3, "f32"),
    (lambda: synth.noisy_torus(50), 48, 5, "bf16"),
    (lambda: synth.icosphere(5), 3000, 9, "f32"),       # crowded: many rows of several cells
    (lambda: synth.icosphere(3), 16, 1, "f16"),
]


def run(lf, m, k, sid, dt, schedule, steps=(3, 40, 300)):
    out = []
    with lf.Mesh(m.V, m.F, field_dtype=dt) as mesh:
        mesh.set_schedule(schedule)
        assert mesh.schedule == lf.SCHEDULES[schedule]
        mesh.seed(synth.sample_seeds(m.n_v, k, sid))
        for t in steps:
            mesh.step(t)
            out.append(mesh.get_field())
        out.append((mesh.stats()["skeleton_total"], mesh.stats()["nnz_io_total"]))
    return out


@pytest.mark.parametrize("case", range(len(CASES)))
def test_schedules_give_the_same_bits(lf, case):
    fac, k, sid, dt = CASES[case]
    m = fac()
    a = run(lf, m, k, sid, dt, "ctas4")
    for other in ("ctas5", "ctas3", "hot", "lean"):
        b = run(lf, m, k, sid, dt, other)
        for fa, fb in zip(a[:-1], b[:-1]):
            for x, y in zip(fa, fb):
                assert np.array_equal(x, y)
        assert a[-1] == b[-1]


def full_rows_field(m, cells, specials):
    """Every vertex holds cell 0 (0.9) and the base layer (0.1); each vertex of
    specials holds `cells` cells (0, 1, ...) in equal parts and no base entry.
    Its neighbours bring no cell it lacks, so a register map that has room
    for `cells` cells keeps it on its fastest tier to the end of the gather."""
    base = cells + 2
    rp, ids, vals = [0], [], []
    for v in range(m.n_v):
        if v in specials:
            ids += list(range(cells))
            vals += [1.0 / cells] * cells
        else:
            ids += [0, base]
            vals += [0.9, 0.1]
        rp.append(len(ids))
    return (np.array(rp, np.int64), np.array(ids, np.int32), np.array(vals, np.float32)), base + 1


@pytest.mark.parametrize("cells", [4, 5, 6])
def test_full_own_rows_on_every_schedule(lf, oracle_mod, cells):
    """Own rows of as many cells as a register map has slots (five slots at
    4 CTAs per SM, six in the lean forms) and no base entry: the base layer
    must not take a cell's slot.  One step on every schedule, bit for bit,
    and against the oracle."""
    from parity_util import ambiguous_rows, check_compare, compare, field_from_lib
    m = synth.planar_grid(16, seed=4)
    specials = {5 * 16 + 5, 8 * 16 + 9, 10 * 16 + 4}
    state, n_layers = full_rows_field(m, cells, specials)
    got = {}
    for sched in lf.SCHEDULES:
        with lf.Mesh(m.V, m.F) as mesh:
            mesh.set_schedule(sched)
            mesh.set_field(*state, n_layers)
            mesh.step(1)
            got[sched] = mesh.get_field()
    for sched, f in got.items():
        for x, y in zip(f, got["ctas4"]):
            assert np.array_equal(x, y), sched
    rp, ids, vals = got["ctas4"]
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    Fin = oracle_mod.Field(state[0], state[1], state[2].astype(np.float64), n_layers)
    Fo, _, mg = oracle_mod.step(L, Fin, margins=True)
    check_compare(compare(Fo, field_from_lib(rp, ids, vals, n_layers, oracle_mod), ambiguous_rows(mg), oracle_mod))


def test_batch_mixing_schedules_matches_alone(lf):
    ms = [c[0]() for c in CASES]
    alone = []
    for (fac, k, sid, dt), m in zip(CASES, ms):
        alone.append(run(lf, m, k, sid, dt, "ctas4", steps=(150,))[0])
    meshes = []
    for j, ((fac, k, sid, dt), m) in enumerate(zip(CASES, ms)):
        x = lf.Mesh(m.V, m.F, field_dtype=dt)
        x.set_schedule(["ctas5", "hot", "lean", "ctas3"][j])
        x.seed(synth.sample_seeds(m.n_v, k, sid))
        meshes.append(x)
    lf.lf_step_batch(meshes, 150)
    for x, want in zip(meshes, alone):
        for p, q in zip(x.get_field(), want):
            assert np.array_equal(p, q)
        x.close()


def test_tune_advances_the_job_and_keeps_a_schedule(lf):
    m = synth.planar_grid(96, seed=9)
    seeds = synth.sample_seeds(m.n_v, 80, 9)
    with lf.Mesh(m.V, m.F) as a, lf.Mesh(m.V, m.F) as b:
        a.seed(seeds)
        b.seed(seeds)
        s = a.tune(64)                     # two rounds over five schedules: 640 steps
        assert s in (0, 1, 2, 3, 4) and a.schedule == s
        assert a.stats()["steps"] == 640
        b.step(640)
        for x, y in zip(a.get_field(), b.get_field()):
            assert np.array_equal(x, y)
        with pytest.raises(lf.LFError):
            a.set_schedule(5)
        with pytest.raises(lf.LFError):
            a.tune(0)
    with lf.Mesh(m.V, m.F) as c:
        with pytest.raises(lf.LFError):
            c.tune(16)                      # no field yet

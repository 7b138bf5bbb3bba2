"""Serving form: jobs through lf_server against the same jobs run alone.

A job's result does not depend on what runs beside it: the labels a server
returns must equal, bit for bit, those of lf_seed + lf_step + lf_labels on the
job alone, whatever the admission order, chunking and batch mates.  Also:
admission under the memory budget, a job larger than the budget, a failing job
(a vertex that sums to zero, raised on the device and read by the host) that
leaves the others untouched, timeouts and invalid calls.
"""
import time

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


JOBS = [
    # (mesh factory, seeds, seed stream, steps, storage type)
    (lambda: synth.icosphere(3), 16, 1, 300, "f32"),
    (lambda: synth.planar_grid(61, seed=2), 64, 3, 170, "f32"),
    (lambda: synth.noisy_torus(40), 32, 5, 230, "bf16"),
    (lambda: synth.planar_grid(33, seed=7), 24, 9, 90, "f32"),
    (lambda: synth.icosphere(2), 8, 11, 400, "f16"),
    (lambda: synth.noisy_torus(24), 12, 13, 129, "f32"),
]


def alone(lf, m, k, sid, steps, dtype, **params):
    with lf.Mesh(m.V, m.F, field_dtype=dtype, **params) as mesh:
        mesh.seed(synth.sample_seeds(m.n_v, k, sid))
        mesh.step(steps)
        return mesh.labels(), mesh.stats()


def test_server_matches_jobs_alone(lf):
    meshes = [fac() for fac, *_ in JOBS]
    with lf.Server(max_active=3, chunk_steps=64) as srv:
        ids = []
        for m, (_, k, sid, steps, dt) in zip(meshes, JOBS):
            ids.append(srv.submit(m.V, m.F, synth.sample_seeds(m.n_v, k, sid), steps, field_dtype=dt))
        assert srv.drain(120.0) == lf.LF_OK
        st = srv.stats()
        assert st["done"] == len(JOBS) and st["failed"] == 0 and st["peak_running"] <= 3
        assert st["running"] == 0 and st["queued"] == 0 and st["bytes_in_use"] == 0
        total = 0
        for jid, m, (_, k, sid, steps, dt) in zip(ids, meshes, JOBS):
            status, info, labels = srv.wait(jid, 0.0, n_v=m.n_v, release=True)
            assert status == lf.LF_OK and info["state"] == lf.LF_JOB_DONE
            assert info["steps_done"] == steps and info["n_v"] == m.n_v
            assert info["arrival_ns"] <= info["admit_ns"] <= info["finish_ns"]
            want, wst = alone(lf, m, k, sid, steps, dt)
            assert np.array_equal(labels, want)
            assert info["skeleton_total"] == wst["skeleton_total"]
            total += info["skeleton_total"]
            with pytest.raises(lf.LFError):
                srv.wait(jid, 0.0)                 # released: the id is gone
        assert st["skeleton_total"] == total


def test_server_admits_under_the_memory_budget(lf, oracle_mod):
    m = synth.planar_grid(61, seed=2)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    with lf.Mesh(csr=(L.rowptr, L.col, L.val)) as probe:      # a server job holds no geometry
        one = probe.stats()["device_bytes"]
    big = synth.planar_grid(200, seed=2)
    # room for one grid61 job at a time (its estimate is its device bytes
    # plus the label buffer), never for the 200x200 grid
    with lf.Server(hbm_budget_bytes=int(1.6 * one), chunk_steps=50) as srv:
        ids = [srv.submit(m.V, m.F, synth.sample_seeds(m.n_v, 16, 20 + i), 120) for i in range(3)]
        jbig = srv.submit(big.V, big.F, synth.sample_seeds(big.n_v, 16, 1), 10)
        assert srv.drain(120.0) == lf.LF_OK
        st = srv.stats()
        assert st["peak_running"] == 1 and st["done"] == 3 and st["failed"] == 1
        status, info, _ = srv.wait(jbig, 0.0)
        assert status == lf.LF_ERR_OOM and info["state"] == lf.LF_JOB_FAILED and info["admit_ns"] == 0
        finish = []
        for i, jid in enumerate(ids):
            status, info, labels = srv.wait(jid, 0.0, n_v=m.n_v)
            assert status == lf.LF_OK
            want, _ = alone(lf, m, 16, 20 + i, 120, "f32")
            assert np.array_equal(labels, want)
            finish.append((info["admit_ns"], info["finish_ns"]))
        # one at a time, in arrival order
        for (a0, f0), (a1, f1) in zip(finish, finish[1:]):
            assert f0 <= a1


def test_server_isolates_a_failing_job(lf):
    # strongly negative band coefficients drive every entry of a two-layer
    # vertex to zero: the step kernel flags the zero sum and the host retires
    # that job alone
    bad = dict(e_cb=-1e6, e_bc=-1e6)
    m = synth.icosphere(3)
    g = synth.planar_grid(33, seed=7)
    with lf.Server(chunk_steps=32) as srv:
        j_ok1 = srv.submit(g.V, g.F, synth.sample_seeds(g.n_v, 24, 9), 100)
        j_bad = srv.submit(m.V, m.F, synth.sample_seeds(m.n_v, 16, 1), 100, **bad)
        j_ok2 = srv.submit(m.V, m.F, synth.sample_seeds(m.n_v, 16, 1), 100)
        assert srv.drain(120.0) == lf.LF_OK
        status, info, labels = srv.wait(j_bad, 0.0, n_v=m.n_v)
        assert status == lf.LF_ERR_STATE and info["state"] == lf.LF_JOB_FAILED and labels is None
        assert info["steps_done"] < 100
        for jid, mesh, k, sid in ((j_ok1, g, 24, 9), (j_ok2, m, 16, 1)):
            status, info, labels = srv.wait(jid, 0.0, n_v=mesh.n_v)
            assert status == lf.LF_OK
            want, _ = alone(lf, mesh, k, sid, 100, "f32")
            assert np.array_equal(labels, want)
        assert srv.stats()["failed"] == 1


def test_server_timeouts_and_invalid_calls(lf):
    m = synth.planar_grid(120, seed=2)
    with lf.Server(chunk_steps=16) as srv:
        jid = srv.submit(m.V, m.F, synth.sample_seeds(m.n_v, 32, 1), 3000)
        status, info, _ = srv.wait(jid, 0.0)
        assert status == lf.LF_ERR_TIMEOUT and info["state"] in (lf.LF_JOB_QUEUED, lf.LF_JOB_RUNNING)
        with pytest.raises(lf.LFError) as ei:
            srv.submit(m.V, m.F, np.array([0, 0], np.int32), 10)          # repeated seed
        assert ei.value.status == lf.LF_ERR_INVALID
        with pytest.raises(lf.LFError) as ei:
            srv.submit(m.V, m.F, np.array([1], np.int32), -1)
        assert ei.value.status == lf.LF_ERR_INVALID
        with pytest.raises(lf.LFError):
            srv.wait(12345, 0.0)
        t0 = time.monotonic()
        status, info, _ = srv.wait(jid, 60.0, n_v=m.n_v)
        assert status == lf.LF_OK and info["steps_done"] == 3000
        assert time.monotonic() - t0 < 60.0
    # destroying a server with work queued returns without waiting for it
    srv = lf.Server(chunk_steps=16)
    for i in range(4):
        srv.submit(m.V, m.F, synth.sample_seeds(m.n_v, 32, 40 + i), 100000)
    t0 = time.monotonic()
    srv.close()
    assert time.monotonic() - t0 < 30.0


def test_server_lloyd_rounds_and_dual_mesh_match_the_job_alone(lf):
    # two jobs asking for Lloyd-like rounds and the dual mesh, batched with a
    # plain one: seeds, labels and triangles equal those of the same calls
    # on the job alone (lf_step, lf_lloyd, lf_extract_dual)
    jobs = [(synth.planar_grid(41, seed=3), 16, 1, 120, 2, True), (synth.noisy_torus(40), 24, 5, 150, 1, True),
            (synth.planar_grid(33, seed=7), 24, 9, 90, 0, False)]
    with lf.Server(chunk_steps=50) as srv:
        ids = [srv.submit(m.V, m.F, synth.sample_seeds(m.n_v, k, sid), n, lloyd_rounds=r, extract_dual=d)
               for m, k, sid, n, r, d in jobs]
        assert srv.drain(120.0) == lf.LF_OK
        for jid, (m, k, sid, n, r, d) in zip(ids, jobs):
            status, info, labels = srv.wait(jid, 0.0, n_v=m.n_v)
            assert status == lf.LF_OK and info["lloyd_done"] == r == info["lloyd_rounds"]
            with lf.Mesh(m.V, m.F) as mesh:
                mesh.seed(synth.sample_seeds(m.n_v, k, sid))
                mesh.step(n)
                total = mesh.stats()["skeleton_total"]
                for _ in range(r):
                    mesh.lloyd(1, n)
                    total += mesh.stats()["skeleton_total"]
                assert np.array_equal(labels, mesh.labels())
                assert info["skeleton_total"] == total
                if d:
                    tri = srv.dual_mesh(jid)
                    assert info["dual_triangles"] == len(tri) > 0
                    assert np.array_equal(tri, mesh.extract_dual())
                else:
                    assert info["dual_triangles"] == -1
                    with pytest.raises(lf.LFError) as ei:
                        srv.dual_mesh(jid)
                    assert ei.value.status == lf.LF_ERR_STATE


def test_server_job_matches_the_oracle(lf, oracle_mod):
    """A job through the server against the FP64 oracle directly (not only
    against the same job alone): icosphere level 3, 16 seeds, 300 steps,
    served beside two other jobs.  Labels must equal the oracle's on every
    vertex where a second oracle run, rounded to FP32 after every step, gives
    the same label (and on its 1-ring): ties aside, bit-exact."""
    from parity_util import one_ring, to_f32
    m = synth.icosphere(3)
    seeds = synth.sample_seeds(m.n_v, 16, 1)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = Fr = oracle_mod.seed(m.n_v, seeds)
    for _ in range(300):
        F, _ = oracle_mod.step(L, F)
        Fr, _ = oracle_mod.step(L, to_f32(Fr, oracle_mod))
    lab_o = oracle_mod.labels(F)
    stable = ~one_ring(L.rowptr, L.col, lab_o != oracle_mod.labels(Fr))
    others = [synth.noisy_torus(40), synth.planar_grid(33, seed=7)]
    with lf.Server(max_active=3, chunk_steps=64) as srv:
        ids = [srv.submit(o.V, o.F, synth.sample_seeds(o.n_v, 20, 3 + j), 250) for j, o in enumerate(others)]
        jid = srv.submit(m.V, m.F, seeds, 300)
        assert srv.drain(120.0) == lf.LF_OK
        status, info, labels = srv.wait(jid, 0.0, n_v=m.n_v, release=True)
        for x in ids:
            srv.wait(x, 0.0, release=True)
    assert status == lf.LF_OK
    assert stable.mean() > 0.8
    assert np.array_equal(labels[stable], lab_o[stable])
    assert np.mean(labels == lab_o) > 0.95

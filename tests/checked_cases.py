"""Cases that test_gpu_checked runs in a child process, once per library build.

``python tests/checked_cases.py OUT.npz`` runs a set of step-kernel cases
through whatever library LF_LIBRARY names (the plain or the bounds-checked
build) and saves every result; the test compares the two files bit for bit.
``python tests/checked_cases.py --bad-index`` (checked build only) feeds
lf_step_noalloc an operator whose first column is one past the last vertex
and prints the status it returns: the checked kernel must catch the index
before using it.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "tests")):
    if p not in sys.path:
        sys.path.insert(0, p)

import synth  # noqa: E402
from test_gpu_parity import random_field  # noqa: E402


def run_cases(out):
    from paper_1804_09152_gb300 import _lib as lf
    res = {}

    def keep(name, mesh):
        rp, lay, val = mesh.get_field()
        res[name + "_rp"], res[name + "_lay"], res[name + "_val"] = rp, lay, val
        res[name + "_labels"] = mesh.labels()
        st = mesh.stats()
        res[name + "_stats"] = np.array([st["skeleton_total"], st["nnz_io_total"], st["retries"]], np.int64)

    g = synth.planar_grid(61, seed=2)
    for sched in ("ctas4", "hot", "lean"):                             # register tier, ragged last tile
        with lf.Mesh(g.V, g.F) as mesh:                                # (and the lean schedules' gather)
            mesh.set_schedule(sched)
            mesh.seed(synth.sample_seeds(g.n_v, 64, 3))
            mesh.step(300)
            keep("grid" if sched == "ctas4" else f"grid_{sched}", mesh)
    t = synth.noisy_torus(40)
    with lf.Mesh(t.V, t.F, field_dtype="bf16", initial_capacity=t.n_v) as mesh:   # growth and re-runs
        mesh.seed(synth.sample_seeds(t.n_v, 32, 5))
        mesh.step(200)
        keep("torus_bf16", mesh)
    small = synth.planar_grid(20, seed=6)
    for per_row, n_layers in ((5, 200), (14, 400)):                    # shared-memory and storage-free tiers
        for sched in ("ctas4", "hot", "lean"):                         # (hot: every tile takes the full step)
            rng = np.random.default_rng(per_row)
            with lf.Mesh(small.V, small.F) as mesh:
                mesh.set_schedule(sched)
                mesh.set_field(*random_field(small.n_v, n_layers, per_row, rng), n_layers)
                mesh.step(1)
                keep(f"unions{per_row}" + ("" if sched == "ctas4" else f"_{sched}"), mesh)
    meshes = [lf.Mesh(m.V, m.F, field_dtype=d) for m, d in ((g, "f32"), (t, "bf16"), (synth.icosphere(3), "f16"))]
    for k, mesh in enumerate(meshes):
        mesh.seed(synth.sample_seeds(mesh.n_v, 16 + 8 * k, 7 + k))
    lf.lf_step_batch(meshes, [150, 90, 120])                           # one launch per step and storage type
    for k, mesh in enumerate(meshes):
        keep(f"batch{k}", mesh)
    for k, (mesh, sched) in enumerate(zip(meshes, ("hot", "lean", "hot"))):
        mesh.set_schedule(sched)                                       # the lean schedules in a batch
        mesh.seed(synth.sample_seeds(mesh.n_v, 16 + 8 * k, 7 + k))
    lf.lf_step_batch(meshes, [150, 90, 120])
    for k, mesh in enumerate(meshes):
        keep(f"batch{k}_lean", mesh)
        mesh.close()
    rng = np.random.default_rng(11)
    mats = [0.2 * rng.random((31, 31)) for _ in range(3)]
    with lf.Mesh(g.V, g.F) as mesh:                                    # general coefficient matrices
        mesh.seed(synth.sample_seeds(g.n_v, 30, 4))
        mesh.set_coefficients(*[M.astype(np.float32) for M in mats])
        mesh.step(60)
        keep("general", mesh)
    with lf.Mesh(g.V, g.F) as mesh:                                    # region seeds
        mesh.seed_regions(synth.sample_seeds(g.n_v, 40, 8), 1)
        mesh.step(40)
        keep("regions", mesh)
    np.savez(out, **res)


def bad_index():
    import torch
    from paper_1804_09152_gb300 import _lib as lf
    from test_zz_no_alloc import TILE, segment
    m = synth.planar_grid(33, seed=7)
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed(synth.sample_seeds(m.n_v, 16, 1))
        mesh.step(10)
        state = mesh.get_field()
        rp, col, val = mesh.get_operator()
    colval = np.empty((col.size, 2), np.int32)
    colval[:, 0] = col
    colval[:, 1] = val.view(np.int32)
    colval[0, 0] = m.n_v                                               # one past the last vertex
    cap = 768
    tiles = (m.n_v + TILE - 1) // TILE
    dev = torch.device("cuda", 0)
    d_rp = torch.from_numpy(rp.astype(np.int32)).to(dev)
    d_cv = torch.from_numpy(colval.reshape(-1)).to(dev)
    bufs = [(torch.zeros((m.n_v, 2), dtype=torch.int32, device=dev),
             torch.zeros((m.n_v, 4), dtype=torch.int32, device=dev),
             torch.zeros(tiles * cap, dtype=torch.int16, device=dev),
             torch.zeros(tiles * cap, dtype=torch.float32, device=dev)) for _ in range(2)]
    rows, head, ids, vals = segment(*state, m.n_v, cap)
    for dst, src in zip(bufs[0], (rows, head, ids.view(np.int16), vals)):
        dst.copy_(torch.from_numpy(src))
    stream = torch.cuda.current_stream().cuda_stream
    try:
        lf.lf_step_noalloc(stream, m.n_v, 17, d_rp.data_ptr(), d_cv.data_ptr(),
                           *[x.data_ptr() for x in bufs[0]], *[x.data_ptr() for x in bufs[1]], cap)
        print("status 0")
    except lf.LFError as e:
        print(f"status {e.status} {e}")
    torch.cuda.synchronize()


if __name__ == "__main__":
    if sys.argv[1] == "--bad-index":
        bad_index()
    else:
        run_cases(sys.argv[1])

"""lf_step_noalloc against lf_step.

lf_step_noalloc serves callers that own all device memory and cannot let the
library allocate (a framework with its own memory pool, a service that
allocates only at start-up, code running where allocation is not allowed).
Here the test allocates every buffer itself, runs two steps in a row through
lf_step_noalloc (the output of the first is the input of the second) and
checks each against lf_step on the same state, with the tolerance of the
other parity tests.  The file is named to be collected last.
"""
import numpy as np
import pytest

import synth
from parity_util import FIELD_TOL

pytestmark = pytest.mark.gpu

TILE = 256


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


def segment(rp, lay, val, n_v, cap):
    """Plain CSR -> tile-segmented arrays: rows as (start, count) int32 pairs,
    head records as (count, id0 | id1 << 16, bits of value 0, bits of value 1)."""
    tiles = (n_v + TILE - 1) // TILE
    rows = np.zeros((n_v, 2), np.int32)
    head = np.zeros((n_v, 4), np.int32)
    ids = np.zeros(tiles * cap, np.uint16)
    vals = np.zeros(tiles * cap, np.float32)
    for i in range(n_v):
        t = i // TILE
        start = t * cap + int(rp[i] - rp[t * TILE])
        n = int(rp[i + 1] - rp[i])
        rows[i] = (start, n)
        ids[start:start + n] = lay[rp[i]:rp[i + 1]]
        vals[start:start + n] = val[rp[i]:rp[i + 1]]
        head[i, 0] = n
        if n > 0:
            head[i, 1] = int(lay[rp[i]])
            head[i, 2] = np.float32(val[rp[i]]).view(np.int32)
        if n > 1:
            head[i, 1] |= int(lay[rp[i] + 1]) << 16
            head[i, 3] = np.float32(val[rp[i] + 1]).view(np.int32)
    return rows, head, ids, vals


def unsegment(rows, ids, vals):
    counts = rows[:, 1].astype(np.int64)
    rp = np.concatenate([[0], np.cumsum(counts)])
    idx = np.concatenate([np.arange(s, s + n) for s, n in rows]) if rp[-1] else np.zeros(0, np.int64)
    return rp, ids[idx].astype(np.int32), vals[idx]


def test_noalloc_matches_lf_step_on_two_calls(lf, oracle_mod):
    import torch
    m = synth.planar_grid(61, seed=2)                       # 3721 vertices: a ragged last tile
    seeds = synth.sample_seeds(m.n_v, 64, 3)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    rows_of = np.repeat(np.arange(m.n_v), np.diff(L.rowptr))
    off = L.col != rows_of
    rp_off = np.concatenate([[0], np.cumsum(np.bincount(rows_of[off], minlength=m.n_v))]).astype(np.int32)
    colval = np.empty((int(off.sum()), 2), np.int32)
    colval[:, 0] = L.col[off]
    colval[:, 1] = L.val[off].astype(np.float32).view(np.int32)

    ref = lf.Mesh(csr=(L.rowptr, L.col, L.val))             # the same operator through lf_create_mesh_csr
    ref.seed(seeds)
    ref.step(20)
    state = ref.get_field()

    cap = 768
    dev = torch.device("cuda", 0)
    d_rp = torch.from_numpy(rp_off).to(dev)
    d_cv = torch.from_numpy(colval.reshape(-1)).to(dev)
    tiles = (m.n_v + TILE - 1) // TILE
    bufs = []
    for _ in range(2):
        bufs.append((torch.zeros((m.n_v, 2), dtype=torch.int32, device=dev),
                     torch.zeros((m.n_v, 4), dtype=torch.int32, device=dev),
                     torch.zeros(tiles * cap, dtype=torch.int16, device=dev),
                     torch.zeros(tiles * cap, dtype=torch.float32, device=dev)))
    rows, head, ids, vals = segment(*state, m.n_v, cap)
    bufs[0][0].copy_(torch.from_numpy(rows))
    bufs[0][1].copy_(torch.from_numpy(head))
    bufs[0][2].copy_(torch.from_numpy(ids.view(np.int16)))
    bufs[0][3].copy_(torch.from_numpy(vals))
    stream = torch.cuda.current_stream().cuda_stream

    for call in range(2):
        src, dst = bufs[call % 2], bufs[(call + 1) % 2]
        nnz, _ = lf.lf_step_noalloc(stream, m.n_v, 65, d_rp.data_ptr(), d_cv.data_ptr(),
                                    *[x.data_ptr() for x in src], *[x.data_ptr() for x in dst], cap)
        out = unsegment(dst[0].cpu().numpy(), dst[2].cpu().numpy().view(np.uint16), dst[3].cpu().numpy())
        # the output's head records describe its rows
        want_head = segment(*out, m.n_v, cap)[1]
        assert np.array_equal(dst[1].cpu().numpy(), want_head), f"head records, call {call}"
        ref.step(1)
        want = ref.get_field()
        assert nnz == want[0][-1]
        assert np.array_equal(out[0], want[0]) and np.array_equal(out[1], want[1]), f"pattern, call {call}"
        assert np.abs(out[2] - want[2]).max() <= FIELD_TOL, f"values, call {call}"
    ref.close()


def test_noalloc_reports_small_segments_and_bad_sizes(lf, oracle_mod):
    import torch
    m = synth.icosphere(2)                                  # 162 vertices: one tile
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    rows_of = np.repeat(np.arange(m.n_v), np.diff(L.rowptr))
    off = L.col != rows_of
    rp_off = np.concatenate([[0], np.cumsum(np.bincount(rows_of[off], minlength=m.n_v))]).astype(np.int32)
    colval = np.empty((int(off.sum()), 2), np.int32)
    colval[:, 0] = L.col[off]
    colval[:, 1] = L.val[off].astype(np.float32).view(np.int32)
    # one layer per vertex, different at neighbouring vertices, and no exclusion
    # penalty: every layer of a neighbour enters with a positive value, so the
    # output holds several entries per vertex and outgrows 256-entry segments
    n_layers = 64
    rp = np.arange(m.n_v + 1, dtype=np.int64)
    lay = ((np.arange(m.n_v) * 7) % (n_layers - 1)).astype(np.int32)
    val = np.ones(m.n_v, np.float32)
    cap = TILE
    rows, head, ids, vals = segment(rp, lay, val, m.n_v, cap)
    dev = torch.device("cuda", 0)
    d = [torch.from_numpy(x).to(dev) for x in (rp_off, colval.reshape(-1), rows, head, ids.view(np.int16), vals)]
    o = [torch.zeros_like(x) for x in d[2:]]
    stream = torch.cuda.current_stream().cuda_stream
    args = [x.data_ptr() for x in d] + [x.data_ptr() for x in o]
    free = lf.lf_default_params(w_cc=0.0, w_cb=0.0)
    with pytest.raises(lf.LFError) as ei:
        lf.lf_step_noalloc(stream, m.n_v, n_layers, *args, cap, free)
    assert ei.value.status == lf.LF_ERR_CAPACITY
    assert ei.value.need_tile_cap > cap
    assert "tile_cap" in lf.lf_last_error(None)
    with pytest.raises(lf.LFError) as ei:
        lf.lf_step_noalloc(stream, m.n_v, n_layers, *args, 100)     # not a multiple of 16, below 256
    assert ei.value.status == lf.LF_ERR_INVALID
    with pytest.raises(lf.LFError) as ei:
        lf.lf_step_noalloc(stream, m.n_v, n_layers, *args, cap, lf.lf_default_params(field_dtype="bf16"))
    assert ei.value.status == lf.LF_ERR_INVALID

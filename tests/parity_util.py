"""Comparison helpers for the GPU-vs-oracle parity tests (no method arithmetic).

Fields are compared element by element over the union of both patterns (an
entry missing on one side counts as 0).  A row whose discrete decisions sit
within rounding of flipping (oracle margins: the irows test or the clamp to
zero, relative distance below ``TAU_DECISION``) is a tie: either outcome is
correct.  Every row is compared:

* a row that is not a tie must have the oracle's pattern and every value
  within ``FIELD_TOL``;
* a tie row may differ in pattern only by entries of at most ``FIELD_TOL``
  (an entry clamped to zero on one side and kept at a tiny value on the
  other); a row whose values differ by more -- the flip changed the row --
  counts as value-disagreeing, and those rows stay a small, stated fraction.

Most tie rows are entries entering or leaving at a tiny value (the base
layer re-entering a vertex from a neighbour's small tail): the margin of the
clamp is taken relative to the magnitude sums of the terms, which are O(1)
while the value is small, so such rows count as ties although both outcomes
agree far within ``FIELD_TOL``.
"""
import numpy as np

from oracle import TIE_MARGIN

FIELD_TOL = 1e-5              # FP32 field error bound (absolute; values lie in [0, 1])
TAU_DECISION = TIE_MARGIN     # ~800 FP32 ulps of relative distance from a flip
VALUE_ROWS_FRAC = 0.01        # bound on value-disagreeing (tie) rows per comparison


def coo(rowptr, ids, n_layers):
    rows = np.repeat(np.arange(rowptr.size - 1, dtype=np.int64), np.diff(rowptr))
    return rows * n_layers + ids.astype(np.int64)


def field_from_lib(rp, lay, val, n_layers, oracle):
    return oracle.Field(rp.astype(np.int64), lay.astype(np.int32), val.astype(np.float64), n_layers)


def to_f32(F, oracle):
    """The oracle field rounded to the FP32 storage of the GPU (zeros dropped)."""
    v32 = F.vals.astype(np.float32).astype(np.float64)
    keep = v32 != 0.0
    rows = np.repeat(np.arange(F.n_v), np.diff(F.rowptr))[keep]
    rp = np.zeros(F.n_v + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return oracle.Field(np.cumsum(rp), F.ids[keep].copy(), v32[keep], F.n_layers)


def ambiguous_rows(margins, tau=TAU_DECISION):
    return (margins[:, 0] < tau) | (margins[:, 1] < tau)


def compare(Fo, Fg, amb=None, oracle=None):
    """Element-wise comparison over the union of both patterns.

    A row disagrees when its patterns differ or an entry differs by more than
    FIELD_TOL.  ``unexplained`` counts disagreeing rows that are not ties: it
    must be 0.  ``value_rows`` counts rows with an entry differing by more
    than FIELD_TOL (a missing entry counts as 0), ties included.  With
    ``oracle`` given, the oracle output is first rounded to FP32 storage: an
    entry too small for FP32 is absent from any FP32 result.
    """
    if oracle is not None:
        Fo = to_f32(Fo, oracle)
    NL = Fo.n_layers
    ko = coo(Fo.rowptr, Fo.ids, NL)
    kg = coo(Fg.rowptr, Fg.ids, NL)
    allk = np.union1d(ko, kg)
    vo = np.zeros(allk.size)
    vg = np.zeros(allk.size)
    io = np.searchsorted(allk, ko)
    ig = np.searchsorted(allk, kg)
    vo[io] = Fo.vals
    vg[ig] = Fg.vals
    in_o = np.zeros(allk.size, bool)
    in_g = np.zeros(allk.size, bool)
    in_o[io] = True
    in_g[ig] = True
    rows = allk // NL
    if amb is None:
        amb = np.zeros(Fo.n_v, bool)
    err = np.abs(vo - vg)
    bad_entry = (in_o != in_g) | (err > FIELD_TOL)
    bad_rows = np.zeros(Fo.n_v, bool)
    bad_rows[rows[bad_entry]] = True
    value_rows = np.zeros(Fo.n_v, bool)
    value_rows[rows[err > FIELD_TOL]] = True
    ok = ~amb[rows]
    return {
        "max_err": float(err[ok].max()) if ok.any() else 0.0,
        "max_err_all": float(err.max()) if err.size else 0.0,
        "pattern_mismatch": int((in_o != in_g)[ok].sum()),
        "pattern_mismatch_all": int((in_o != in_g).sum()),
        "disagreeing_rows": int(bad_rows.sum()),
        "value_rows": int(value_rows.sum()),
        "unexplained": int((bad_rows & ~amb).sum()),
        "tie_rows": int(amb.sum()),
        "rows": int(Fo.n_v),
    }


def check_compare(r, value_rows_frac=VALUE_ROWS_FRAC):
    """The parity bar on one ``compare`` result: non-tie rows exact in pattern
    and within FIELD_TOL; value-disagreeing rows (ties whose flip moved the
    row) at most ``value_rows_frac`` of the rows, plus two."""
    assert r["unexplained"] == 0, r
    assert r["max_err"] <= FIELD_TOL, r
    assert r["pattern_mismatch"] == 0, r
    assert r["value_rows"] <= value_rows_frac * r["rows"] + 2, r


def lloyd_differences_explained(got, want, seeds, cand, ties):
    """Whether every cell whose new seed differs between the GPU (``got``) and
    the oracle (``want``) is explained by a decision tie.

    A cell that is not a tie has the same candidate vertex on both sides, so
    it can end differently only by losing or winning a conflict over that
    candidate that went otherwise on the other side.  That needs another
    contender for the vertex that differs: a tie cell, or a cell already
    explained (it may return to its old seed on one side only).  Starting
    from the tie cells, a differing cell is explained when its candidate is
    among the vertices the explained cells chose, were given or hold as old
    seeds on either side; repeated until nothing changes.  Returns the cells
    left unexplained (empty when the result is accepted)."""
    bad = set(np.flatnonzero(got != want).tolist())
    explained = set(int(c) for c in ties)
    verts = set()
    for c in explained:
        verts |= {int(got[c]), int(want[c]), int(cand[c]), int(seeds[c])}
    changed = True
    while changed:
        changed = False
        for c in sorted(bad - explained):
            if int(cand[c]) in verts:
                explained.add(c)
                verts |= {int(got[c]), int(want[c]), int(cand[c]), int(seeds[c])}
                changed = True
    return sorted(bad - explained)


def row_max_err(Fa, Fb):
    """Per row, the largest absolute difference between two fields over the
    union of their patterns (an entry missing on one side counts as 0)."""
    NL = Fa.n_layers
    ka = coo(Fa.rowptr, Fa.ids, NL)
    kb = coo(Fb.rowptr, Fb.ids, NL)
    allk = np.union1d(ka, kb)
    va = np.zeros(allk.size)
    vb = np.zeros(allk.size)
    va[np.searchsorted(allk, ka)] = Fa.vals
    vb[np.searchsorted(allk, kb)] = Fb.vals
    out = np.zeros(Fa.n_v)
    np.maximum.at(out, allk // NL, np.abs(va - vb))
    return out


def one_ring(rowptr, col, mask):
    """mask grown by one ring of the operator's pattern (rows with an entry
    in a masked column)."""
    rows = np.repeat(np.arange(rowptr.size - 1), np.diff(rowptr))
    out = mask.copy()
    np.logical_or.at(out, rows, mask[col])
    return out

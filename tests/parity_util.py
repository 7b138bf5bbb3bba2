"""Comparison helpers for the GPU-vs-oracle parity tests (no method arithmetic).

Fields are compared element by element over the union of both patterns (an
entry missing on one side counts as 0).  A row whose discrete decisions sit
within rounding of flipping (oracle margins: the irows test or the clamp to
zero, relative distance below ``TAU_DECISION``) is a tie: either outcome is
correct.  Every row is compared; a row that disagrees must be a tie.
"""
import numpy as np

FIELD_TOL = 1e-5          # FP32 field error bound (absolute; values lie in [0, 1])
TAU_DECISION = 1e-4       # ~800 FP32 ulps of relative distance from a flip


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
    must be 0.  With ``oracle`` given, the oracle output is first rounded to
    FP32 storage: an entry too small for FP32 is absent from any FP32 result.
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
    ok = ~amb[rows]
    return {
        "max_err": float(err[ok].max()) if ok.any() else 0.0,
        "max_err_all": float(err.max()) if err.size else 0.0,
        "pattern_mismatch": int((in_o != in_g)[ok].sum()),
        "pattern_mismatch_all": int((in_o != in_g).sum()),
        "disagreeing_rows": int(bad_rows.sum()),
        "unexplained": int((bad_rows & ~amb).sum()),
        "tie_rows": int(amb.sum()),
        "rows": int(Fo.n_v),
    }

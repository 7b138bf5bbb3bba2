"""Comparison helpers for the GPU-vs-oracle parity tests (no method arithmetic).

Fields are compared element by element over the union of both patterns (an
entry missing on one side counts as 0).  A row whose discrete decisions sit
within rounding of flipping (oracle margins: the irows test or the clamp to
zero, relative distance below ``TAU_DECISION``) is a tie: either outcome is
correct, so it is counted and left out of the value comparison.
"""
import numpy as np

FIELD_TOL = 1e-5          # FP32 field error bound (absolute; values lie in [0, 1])
TAU_DECISION = 1e-3       # ~8000 FP32 ulps of relative distance from a flip


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


def compare(Fo, Fg, amb=None):
    """Max |difference| over rows that are not ties, plus pattern statistics."""
    NL = Fo.n_layers
    ko = coo(Fo.rowptr, Fo.ids, NL)
    kg = coo(Fg.rowptr, Fg.ids, NL)
    allk = np.union1d(ko, kg)
    vo = np.zeros(allk.size)
    vg = np.zeros(allk.size)
    vo[np.searchsorted(allk, ko)] = Fo.vals
    vg[np.searchsorted(allk, kg)] = Fg.vals
    rows = allk // NL
    in_o = np.zeros(allk.size, bool)
    in_g = np.zeros(allk.size, bool)
    in_o[np.searchsorted(allk, ko)] = True
    in_g[np.searchsorted(allk, kg)] = True
    if amb is None:
        amb = np.zeros(Fo.n_v, bool)
    ok = ~amb[rows]
    err = np.abs(vo - vg)
    mism = in_o != in_g
    return {
        "max_err": float(err[ok].max()) if ok.any() else 0.0,
        "max_err_all": float(err.max()) if err.size else 0.0,
        "pattern_mismatch": int(mism[ok].sum()),
        "pattern_mismatch_all": int(mism.sum()),
        "tie_rows": int(amb.sum()),
        "rows": int(Fo.n_v),
    }

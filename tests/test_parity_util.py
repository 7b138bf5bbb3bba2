"""The comparison rules of the parity tests, on hand-made inputs (CPU).

These rules decide what a GPU result may differ in; each case here is built
so that one rule, applied wrongly, flips the outcome.
"""
import numpy as np
import pytest

from parity_util import FIELD_TOL, check_compare, compare, lloyd_differences_explained


def field(oracle, rows, n_layers):
    rp, ids, vals = [0], [], []
    for r in rows:
        for l in sorted(r):
            ids.append(l)
            vals.append(r[l])
        rp.append(len(ids))
    return oracle.Field(np.array(rp, np.int64), np.array(ids, np.int32), np.array(vals, np.float64), n_layers)


def test_compare_counts_rows_by_kind(oracle_mod):
    want = field(oracle_mod, [{0: 1.0}, {0: 0.5, 1: 0.5}, {1: 1.0}, {0: 0.9, 2: 0.1}], 3)
    # row 1: a tiny extra entry (pattern differs, values within tolerance)
    # row 3: a value moved by 1e-3
    got = field(oracle_mod, [{0: 1.0}, {0: 0.5, 1: 0.5, 2: 1e-7}, {1: 1.0}, {0: 0.899, 2: 0.101}], 3)
    r = compare(want, got)
    assert r["disagreeing_rows"] == 2 and r["value_rows"] == 1 and r["unexplained"] == 2
    amb = np.array([False, True, False, True])
    r = compare(want, got, amb)
    assert r["unexplained"] == 0 and r["pattern_mismatch"] == 0 and r["max_err"] == 0.0
    check_compare(r, value_rows_frac=0.0)                 # one value row <= 0 * 4 + 2
    # a tie row whose values moved counts against the bound; a non-tie row fails outright
    with pytest.raises(AssertionError):
        check_compare(compare(want, got, np.array([False, True, False, False])))
    many = field(oracle_mod, [{0: 0.5, 1: 0.5}] * 400, 2)
    moved = field(oracle_mod, [{0: 0.5 + 2 * FIELD_TOL, 1: 0.5 - 2 * FIELD_TOL}] * 400, 2)
    r = compare(many, moved, np.ones(400, bool))
    assert r["value_rows"] == 400 and r["unexplained"] == 0
    with pytest.raises(AssertionError):
        check_compare(r)                                  # 400 > 1 % of 400 + 2


def test_lloyd_differences_need_a_tie():
    seeds = np.array([10, 20, 30, 40])
    cand = np.array([11, 21, 31, 41])
    want = cand.copy()
    # cell 2 kept its old seed on the GPU side with no tie anywhere: unexplained
    got = want.copy()
    got[2] = seeds[2]
    assert lloyd_differences_explained(got, want, seeds, cand, []) == [2]
    # cell 0 is a tie and took 31 on the GPU, so cell 2 (candidate 31) lost it there
    got = np.array([31, 21, 30, 41])
    assert lloyd_differences_explained(got, want, seeds, cand, [0]) == []
    # ... and cell 3, whose candidate is cell 2's old seed, along the chain
    cand3 = np.array([11, 21, 31, 30])
    want3 = cand3.copy()
    got3 = np.array([31, 21, 30, 40])
    assert lloyd_differences_explained(got3, want3, seeds, cand3, [0]) == []
    # a difference far from the tie stays unexplained
    got4 = np.array([31, 20, 30, 41])
    assert lloyd_differences_explained(got4, want, seeds, cand, [0]) == [1]


def test_row_errors_and_rings(oracle_mod):
    from parity_util import one_ring, row_max_err
    a = field(oracle_mod, [{0: 1.0}, {0: 0.5, 1: 0.5}, {1: 1.0}], 3)
    b = field(oracle_mod, [{0: 1.0}, {0: 0.4, 1: 0.5, 2: 0.1}, {2: 1.0}], 3)
    assert np.allclose(row_max_err(a, b), [0.0, 0.1, 1.0])
    # path 0 - 1 - 2 - 3: a mark at 3 spreads to 2 only
    rp = np.array([0, 2, 5, 8, 10])
    col = np.array([0, 1, 0, 1, 2, 1, 2, 3, 2, 3])
    assert one_ring(rp, col, np.array([False, False, False, True])).tolist() == [False, False, True, True]

"""Hand-worked time-iterations (tests/golden/hand_cases.json) through the
oracle (CPU) and through the CUDA library (GPU, FP32: within 1e-6).

Each case is a tiny operator and field whose next states were derived by
hand from Algorithm 1; the derivations sit beside the oracle tests of the
same name in test_oracle.py.
"""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = json.load(open(os.path.join(HERE, "golden", "hand_cases.json")))["cases"]


def field_arrays(rows):
    rp, ids, vals = [0], [], []
    for r in rows:
        for l in sorted(r, key=int):
            ids.append(int(l))
            vals.append(float(r[l]))
        rp.append(len(ids))
    return np.array(rp, np.int64), np.array(ids, np.int32), np.array(vals, np.float64)


def check_rows(rp, ids, vals, expect, tol):
    for i, want in enumerate(expect):
        got = {int(ids[p]): float(vals[p]) for p in range(rp[i], rp[i + 1])}
        assert set(got) == {int(k) for k in want}, (i, got, want)
        for k, v in want.items():
            assert abs(got[int(k)] - v) <= tol, (i, k, got[int(k)], v)


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_cases_on_the_oracle(oracle_mod, case):
    L = oracle_mod.operator_from_dense(np.array(case["operator"]))
    F = oracle_mod.Field(*field_arrays(case["field"]), case["n_layers"])
    for expect in case["expect"]:
        F, _ = oracle_mod.step(L, F)
        check_rows(F.rowptr, F.ids, F.vals, expect, 1e-14)


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_cases_on_the_gpu(oracle_mod, case):
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib as lf
    L = oracle_mod.operator_from_dense(np.array(case["operator"]))
    rp, ids, vals = field_arrays(case["field"])
    with lf.Mesh(csr=(L.rowptr, L.col, L.val)) as mesh:
        mesh.set_field(rp, ids, vals.astype(np.float32), case["n_layers"])
        for expect in case["expect"]:
            mesh.step(1)
            grp, gids, gvals = mesh.get_field()
            check_rows(grp, gids, gvals.astype(np.float64), expect, 1e-6)

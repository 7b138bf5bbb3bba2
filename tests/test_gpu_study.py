"""The Δt study (Sec. 6) through the library against the same study on the oracle.

Both sides run the same seeds at Δt = 0.1, 1, 5 and 10 for the same simulated
time and read the labels every unit of simulated time.  The final labels of
each Δt must agree with the oracle's at that Δt (the sphere's exact ties may
resolve either way, so not every vertex), and the study's own figures (label
agreement with Δt = 0.1, steps to converge) must match the oracle's.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

DTS = (0.1, 1.0, 5.0, 10.0)
HORIZON = 120.0


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


def oracle_sweep(oracle, m, seeds):
    L = oracle.cotan_laplacian(m.V, m.F)
    out = {}
    for dt in DTS:
        steps, every = int(round(HORIZON / dt)), max(1, int(round(1.0 / dt)))
        F = oracle.seed(m.n_v, seeds)
        done, last, prev = 0, 0, None
        while done < steps:
            n = min(every, steps - done)
            for _ in range(n):
                F, _ = oracle.step(L, F, dict(dt=dt))
            done += n
            lab = oracle.labels(F)
            if prev is None or not np.array_equal(lab, prev):
                last = done
            prev = lab
        out[dt] = dict(labels=prev, steps_to_converge=last, steps=steps, every=every)
    for r in out.values():
        r["agreement"] = float(np.mean(r["labels"] == out[DTS[0]]["labels"]))
    return out


def test_dt_sweep_matches_the_oracle(lf, oracle_mod):
    from paper_1804_09152_gb300 import study
    m = synth.icosphere(3)
    seeds = synth.sample_seeds(m.n_v, 16, 1)
    got = study.dt_sweep(m.V, m.F, seeds, DTS, horizon=HORIZON)
    want = oracle_sweep(oracle_mod, m, seeds)
    for dt in DTS:
        g, w = got[dt], want[dt]
        assert g["steps"] == w["steps"] and g["check_every"] == w["every"]
        assert np.mean(g["labels"] == w["labels"]) >= 0.95, dt
        assert abs(g["agreement"] - w["agreement"]) <= 0.05, (dt, g["agreement"], w["agreement"])
        assert g["steps_to_converge"] <= g["steps"]
        if dt >= 5.0:
            assert abs(g["steps_to_converge"] - w["steps_to_converge"]) <= 2 * w["every"], dt
    # the paper's observation: Δt up to 5 gives nearly the same partition
    assert got[1.0]["agreement"] >= 0.95 and got[5.0]["agreement"] >= 0.95

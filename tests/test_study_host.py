"""Host logic of the Δt study (paper_1804_09152_gb300.study) on a scripted
stand-in for the library mesh: how runs are split into label checks, when a
run counts as converged, and the agreement with the smallest Δt."""
import numpy as np
import pytest


class ScriptedMesh:
    """Stands in for lf.Mesh: labels change at scripted step counts."""
    script = {}

    def __init__(self, V, F, field_dtype="f32", dt=None, **kw):
        self.dt, self.done = dt, 0
        self.change_at, self.final = ScriptedMesh.script[dt]

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def seed(self, seeds):
        self.done = 0

    def step(self, n):
        self.done += n

    def labels(self):
        lab = np.zeros(6, np.int32)
        if self.done >= self.change_at:
            lab[:] = self.final
        return lab

    def stats(self):
        return {"skeleton_total": 10 * self.done}


@pytest.fixture
def study(monkeypatch):
    """The study module imported against the scripted mesh; every module and
    attribute it touches is put back afterwards."""
    import importlib
    import sys
    import types
    import paper_1804_09152_gb300 as pkg
    fake = types.SimpleNamespace(Mesh=ScriptedMesh)
    monkeypatch.setitem(sys.modules, "paper_1804_09152_gb300._lib", fake)
    monkeypatch.delitem(sys.modules, "paper_1804_09152_gb300.study", raising=False)
    monkeypatch.setattr(pkg, "_lib", fake, raising=False)
    monkeypatch.setattr(pkg, "study", None, raising=False)
    yield importlib.import_module("paper_1804_09152_gb300.study")


def test_steps_checks_convergence_and_agreement(study):
    # dt = 0.5: 20 steps, labels read every 2 steps, a change at step 7 (seen at 8)
    # dt = 2: 5 steps, read every step, a change at step 3, to other labels
    ScriptedMesh.script = {0.5: (7, [1, 1, 1, 2, 2, 2]), 2.0: (3, [1, 1, 2, 2, 2, 2])}
    r = study.dt_sweep(None, None, [0], dts=(2.0, 0.5), horizon=10.0, check_time=1.0)
    a, b = r[0.5], r[2.0]
    assert a["steps"] == 20 and a["check_every"] == 2 and a["steps_to_converge"] == 8
    assert b["steps"] == 5 and b["check_every"] == 1 and b["steps_to_converge"] == 3
    assert a["time_to_converge"] == 4.0 and b["time_to_converge"] == 6.0
    assert a["agreement"] == 1.0 and abs(b["agreement"] - 5 / 6) < 1e-12
    assert a["skeleton_total"] == 200 and a["base_left"] == 0


def test_a_run_that_never_changes_converges_at_its_first_check(study):
    ScriptedMesh.script = {1.0: (10 ** 9, 0)}
    r = study.dt_sweep(None, None, [0], dts=(1.0,), horizon=4.0, check_time=1.0)
    assert r[1.0]["steps_to_converge"] == 1 and r[1.0]["agreement"] == 1.0

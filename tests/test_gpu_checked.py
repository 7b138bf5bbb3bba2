"""The bounds-checked build (-DLF_CHECKED) against the plain one.

compute-sanitizer is not available to these tests, so the library has a
checked build of its own: every index the step kernel reads or writes
through is compared with its array's length, and one outside raises an error
bit instead of leaving the buffer.  The same cases (every tier of the step
kernel, under the default schedule and the two lean ones, growth with
re-runs, all three storage types, batches, general coefficient matrices,
region seeds) run in a child process against each build: no case may raise
the error, and every result must be bit-identical.
Then an operator entry one past the last vertex, given to the checked build
alone, must come back as an error status, not as a memory fault.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = os.path.join(HERE, "checked_cases.py")


def run_child(lib, *args):
    env = dict(os.environ, LF_LIBRARY=lib)
    r = subprocess.run([sys.executable, CASES, *args], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return r.stdout


def test_checked_build_finds_no_bad_index_and_gives_the_same_bits(tmp_path):
    from paper_1804_09152_gb300 import native
    plain = native.build()
    checked = native.build(checked=True)
    run_child(plain, str(tmp_path / "plain.npz"))
    run_child(checked, str(tmp_path / "checked.npz"))
    a = np.load(tmp_path / "plain.npz")
    b = np.load(tmp_path / "checked.npz")
    assert sorted(a.files) == sorted(b.files) and len(a.files) > 40
    for k in a.files:
        assert a[k].dtype == b[k].dtype and np.array_equal(a[k], b[k]), k
    assert a["torus_bf16_stats"][2] > 0                  # the growth path ran
    for k in a.files:                                    # the schedules give the same bits
        for sched in ("_hot", "_lean"):                  # (retries depend on the capacity left by earlier runs)
            if sched in k and not k.endswith("_stats"):
                assert np.array_equal(a[k], a[k.replace(sched, "")]), k


def test_checked_build_reports_an_index_past_the_end():
    from paper_1804_09152_gb300 import native
    out = run_child(native.build(checked=True), "--bad-index")
    assert "status 5" in out and "index left its array" in out, out

"""Whole trajectories at the benchmark's sizes against the FP64 oracle.

Over a whole trajectory the iteration amplifies rounding: a vertex tied
between two cells is an unstable equilibrium (the w_cc term doubles a
deviation from the tie every step), and the base layer keeps re-entering
band vertices from neighbours' small tails, kept at a tiny value on one side
and clamped to zero on the other, which moves later values nearby.  The
oracle shows the size of this by itself: the same FP64 run with its state
rounded to FP32 storage after every step ends, on the 512^2 grid after 2000
steps, with 0.67 % of the labels changed (nearly all on cell boundaries) and
values changed by up to 7e-5 four rings inside the cells.  The GPU computes
in FP32 and so parts from the FP64 oracle in the same way; it is held to
that spread:

* label agreement: the GPU's labels differ from the FP64 oracle's on at most
  three times as many vertices (plus 0.2 % of them) as the FP32-rounded
  oracle run does -- the GPU rounds every operation to FP32, not only the
  stored state (measured: 0.91 % against 0.67 % on the grid, 1.66 % against
  0.71 % on the torus, whose parametric cells sit near the explicit
  stability limit at dt = 5);
* the differences are tie-breaks between neighbouring cells: at least 95 %
  of the differing vertices lie on a cell boundary (a neighbour carries
  another label) of the oracle's or the GPU's partition, and the same cells
  are alive;
* values: five rings and more inside the cells of both partitions, where
  the two oracle runs agree within FIELD_TOL, the GPU's FP32 field agrees
  within 10 FIELD_TOL.

Single steps at these sizes are compared entry by entry at FIELD_TOL in
test_gpu_parity / test_gpu_fullsize.  BF16 and FP16 storage are stated, not
gated: label agreement and field error against the same FP64 trajectory.

Workloads: 512 x 512 jittered grid, 1024 seeds, 2000 steps (FP32 storage);
1024 x 1024 noisy torus, 8192 seeds, 3000 steps, FP32 / BF16 / FP16.  The
oracle runs on every host core (orc_step_threads, identical to the
single-thread step).
"""
import time

import numpy as np
import pytest

import synth
from parity_util import FIELD_TOL, field_from_lib, one_ring, row_max_err, to_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


def boundary(L, lab):
    """Vertices with a neighbour of another label."""
    rows = np.repeat(np.arange(L.rowptr.size - 1), np.diff(L.rowptr))
    b = np.zeros(lab.size, bool)
    np.logical_or.at(b, rows, lab[L.col] != lab[rows])
    return b


def interior(L, B, rings):
    d = B.copy()
    for _ in range(rings):
        d = one_ring(L.rowptr, L.col, d)
    return ~d


def trajectory_report(lf, oracle, m, seeds, steps, dtypes):
    t0 = time.perf_counter()
    L = oracle.cotan_laplacian(m.V, m.F)
    F = oracle.seed(m.n_v, seeds)
    Fr = F
    for _ in range(steps):
        F, _ = oracle.step(L, F, threads=0)
        Fr, _ = oracle.step(L, to_f32(Fr, oracle), threads=0)
    lab_o = oracle.labels(F)
    lab_r = oracle.labels(Fr)
    err_r = row_max_err(F, Fr)
    t_oracle = time.perf_counter() - t0
    pair = {"mismatch": float(np.mean(lab_o != lab_r))}
    Bo = boundary(L, lab_o)
    deep_r = interior(L, Bo | boundary(L, lab_r), 4)
    pair["max_err_deep"] = float(err_r[deep_r].max())
    print(f"\n{m.n_v} vertices, {len(seeds)} seeds, {steps} steps ({t_oracle:.0f} s of oracle): the FP32-rounded "
          f"oracle run changes {pair['mismatch']:.3%} of the labels; five rings inside the cells "
          f"({deep_r.mean():.1%} of the vertices) its values differ by {pair['max_err_deep']:.2e} at most")
    out = {}
    for dt in dtypes:
        with lf.Mesh(m.V, m.F, field_dtype=dt) as mesh:
            mesh.seed(seeds)
            mesh.step(steps)
            lab = mesh.labels()
            Fg = field_from_lib(*mesh.get_field(), F.n_layers, oracle)
        err = row_max_err(F, Fg)
        mis = lab != lab_o
        on_b = Bo | boundary(L, lab)
        deep = interior(L, on_b, 4)
        out[dt] = {"mismatch": float(mis.mean()), "on_boundary": float(on_b[mis].mean()) if mis.any() else 1.0,
                   "cells_same": set(np.unique(lab[lab >= 0]).tolist()) == set(np.unique(lab_o[lab_o >= 0]).tolist()),
                   "deep": float(deep.mean()), "max_err_deep": float(err[deep].max()) if deep.any() else 0.0,
                   "mean_err": float(err.mean())}
        r = out[dt]
        print(f"  {dt}: labels differ from the FP64 oracle on {r['mismatch']:.3%} of the vertices "
              f"({r['on_boundary']:.1%} of them on a cell boundary); five rings inside the cells "
              f"({r['deep']:.1%} of the vertices) the values differ by {r['max_err_deep']:.2e} at most; "
              f"mean row error {r['mean_err']:.2e}")
    return pair, out


def check_fp32(pair, r):
    assert r["mismatch"] <= 3 * pair["mismatch"] + 0.002, (pair, r)
    assert r["on_boundary"] >= 0.95, (pair, r)
    assert r["cells_same"], r
    if pair["max_err_deep"] <= FIELD_TOL:
        assert r["max_err_deep"] <= 10 * FIELD_TOL, (pair, r)


def test_grid512_2000_steps(lf, oracle_mod):
    m = synth.planar_grid(512, jitter=0.2, seed=2)
    pair, out = trajectory_report(lf, oracle_mod, m, synth.sample_seeds(m.n_v, 1024, 3), 2000, ["f32"])
    check_fp32(pair, out["f32"])


def test_torus1024_3000_steps_precision(lf, oracle_mod):
    m = synth.noisy_torus(1024)
    pair, out = trajectory_report(lf, oracle_mod, m, synth.sample_seeds(m.n_v, 8192, 5), 3000,
                                  ["f32", "bf16", "f16"])
    check_fp32(pair, out["f32"])
    for dt in ("bf16", "f16"):
        assert out[dt]["mismatch"] < 0.1, (dt, out[dt])

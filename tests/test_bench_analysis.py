"""CPU checks of the analysis bench.py reports beside its rates: dual-mesh
triangle quality and cell-area statistics, on cases worked by hand."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_dual_quality_of_known_triangles():
    V = np.array([[0, 0, 0], [1, 0, 0], [0.5, math.sqrt(3) / 2, 0], [0, 1, 0], [2, 0, 0], [1, 0.1, 0]])
    eq = bench.dual_quality(V, np.array([[0, 1, 2]]))
    assert abs(eq["mean_quality"] - 1.0) < 1e-12 and abs(eq["min_angle"] - 60.0) < 1e-9
    assert eq["angles_below_30_pct"] == 0.0
    # right isosceles: r_in = (2 - sqrt 2) / 2, r_circ = sqrt 2 / 2
    ri = bench.dual_quality(V, np.array([[0, 1, 3]]))
    assert abs(ri["mean_quality"] - (2 - math.sqrt(2)) / (math.sqrt(2) / 2)) < 1e-12
    assert abs(ri["mean_min_angle"] - 45.0) < 1e-9
    # a flat triangle: two of its three angles are below 30 degrees
    fl = bench.dual_quality(V, np.array([[0, 4, 5]]))
    assert abs(fl["angles_below_30_pct"] - 200.0 / 3.0) < 1e-9 and fl["mean_quality"] < 0.2
    both = bench.dual_quality(V, np.array([[0, 1, 2], [0, 1, 3]]))
    assert both["triangles"] == 2 and abs(both["min_quality"] - ri["mean_quality"]) < 1e-12


def test_cell_areas_of_a_split_grid():
    # unit-spaced 11 x 11 grid: total area 100; the left five columns and the
    # right six columns as two cells (a vertex carries a third of its faces)
    m = synth.planar_grid(11, jitter=0.0)
    x = m.V[:, 0]
    labels = np.where(x < x.min() + 4.5 * (x.max() - x.min()) / 10, 0, 1).astype(np.int32)
    st = bench.cell_area_stats(m, labels, 2)
    P = m.V[m.F]
    fa = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    va = np.zeros(m.n_v)
    for c in range(3):
        np.add.at(va, m.F[:, c], fa / 3)
    a = np.array([va[labels == 0].sum(), va[labels == 1].sum()])
    assert abs(a.sum() - fa.sum()) < 1e-9
    assert abs(st["cv"] - a.std() / a.mean()) < 1e-12
    assert st["empty_cells"] == 0 and st["base_vertices"] == 0 and sum(st["hist"]) == 2


def test_cell_areas_closed_cases():
    m = synth.planar_grid(11, jitter=0.0)
    extent = np.ptp(m.V[:, 0]) * np.ptp(m.V[:, 1])
    one = bench.cell_area_stats(m, np.zeros(m.n_v, np.int32), 1)
    assert one["cv"] == 0.0 and one["min_rel"] == one["max_rel"] == 1.0 and one["hist"][4] == 1
    # the lumped vertex areas cover the grid's rectangle exactly
    P = m.V[m.F]
    assert abs(0.5 * np.abs(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])[:, 2]).sum() - extent) < 1e-9
    lab = np.zeros(m.n_v, np.int32)
    lab[0] = -1                                    # a base-layer vertex is left out
    st = bench.cell_area_stats(m, lab, 3)          # cells 1 and 2 hold no vertex
    assert st["base_vertices"] == 1 and st["empty_cells"] == 2

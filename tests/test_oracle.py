"""Pins for the FP64 oracle: each test ties it to something other than itself.

* operator: textbook cases of the cotangent Laplacian (5-point stencil on the
  right-triangle grid, equilateral weights, linear precision on planar meshes,
  mean-curvature normal on the sphere), symmetry and zero row sums;
* L_t: the dense matrix product (numpy) on small meshes;
* interest skeleton: dense brute-force evaluation of the irows predicate;
* update: hand-derived special cases of Algorithm 1 (two-vertex operator,
  isolated two-layer vertices, the single-layer fixed point), the literal
  triple loop against the closed form;
* invariants of the iteration: partition of unity, range (0, 1], support
  growth of at most one ring per step, monotone single-seed growth and full
  coverage, mirror symmetry of the partition;
* semantic sanity: agreement with the nearest-seed Voronoi partition on the
  sphere (Sec. 3.1 reports the two as quasi-similar) and insensitivity of the
  partition to the time step (Sec. 6).
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ----------------------------------------------------------------------------
# helpers (no layered-field arithmetic here)
# ----------------------------------------------------------------------------

def adjacency(L):
    n = L.n_v
    A = np.zeros((n, n), bool)
    rows = np.repeat(np.arange(n), np.diff(L.rowptr))
    A[rows, L.col] = True
    return A


def make_field(oracle, rows, n_layers):
    """rows: list of dicts {layer: value}"""
    rp = [0]
    ids, vals = [], []
    for r in rows:
        for l in sorted(r):
            ids.append(l)
            vals.append(r[l])
        rp.append(len(ids))
    return oracle.Field(np.array(rp, np.int64), np.array(ids, np.int32), np.array(vals, np.float64), n_layers)


def row_dict(F, i):
    return {int(F.ids[p]): float(F.vals[p]) for p in range(F.rowptr[i], F.rowptr[i + 1])}


def clamp(v):
    v = 1.0 if v > 1.0 else v
    return 0.0 if v <= 0.0 else v


def normalise(d):
    s = sum(d.values())
    return {k: v / s for k, v in d.items() if v != 0.0}


# ----------------------------------------------------------------------------
# operator
# ----------------------------------------------------------------------------

def test_cotan_right_triangle_grid_is_five_point_stencil(oracle_mod):
    n = 7
    m = synth.planar_grid(n, jitter=0.0)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    D = L.dense()
    A = adjacency(L)
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            v = j * n + i
            assert D[v, v] == -4.0
            for di, dj, w in [(1, 0, 1.0), (-1, 0, 1.0), (0, 1, 1.0), (0, -1, 1.0)]:
                assert D[v, (j + dj) * n + i + di] == w
            # diagonal edges of the split carry the cotangent of a right angle: 0,
            # yet stay structural entries
            diag = [(j + dj) * n + i + di for di, dj in [(1, 1), (-1, -1), (1, -1), (-1, 1)]]
            present = [u for u in diag if A[v, u]]
            assert len(present) in (0, 4)
            for u in present:
                assert D[v, u] == 0.0
    # vertex (i+j) even has all four diagonals, odd none (alternating split)
    assert A[1 * n + 1, 2 * n + 2] and not A[1 * n + 2, 2 * n + 3]


def test_cotan_equilateral_triangle(oracle_mod):
    V = np.array([[0, 0, 0], [1, 0, 0], [0.5, math.sqrt(3) / 2, 0]], float)
    L = oracle_mod.cotan_laplacian(V, np.array([[0, 1, 2]], np.int32))
    D = L.dense()
    w = 0.5 / math.sqrt(3.0)           # (cot 60 deg) / 2, one triangle per edge
    for i in range(3):
        for j in range(3):
            expect = -2 * w if i == j else w
            assert abs(D[i, j] - expect) < 1e-15


@pytest.mark.parametrize("mesh", ["grid", "ico", "torus"])
def test_cotan_symmetric_zero_rowsum(oracle_mod, mesh):
    m = {"grid": lambda: synth.planar_grid(20), "ico": lambda: synth.icosphere(2),
         "torus": lambda: synth.noisy_torus(16)}[mesh]()
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    D = L.dense()
    assert np.abs(D - D.T).max() < 1e-14
    assert np.abs(D.sum(axis=1)).max() < 1e-13
    assert np.abs(D @ np.ones(m.n_v)).max() < 1e-13       # L const = 0


def test_cotan_linear_precision_on_planar_jittered_grid(oracle_mod):
    n = 16
    m = synth.planar_grid(n, jitter=0.2, seed=11)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    D = L.dense()
    interior = [j * n + i for j in range(1, n - 1) for i in range(1, n - 1)]
    for c in range(2):
        r = D @ m.V[:, c]
        assert np.abs(r[interior]).max() < 1e-12
    # jitter makes some angles obtuse: negative off-diagonal weights exist
    off = D[~np.eye(m.n_v, dtype=bool)]
    assert off.min() < 0.0


def test_cotan_sphere_mean_curvature_normal(oracle_mod):
    m = synth.icosphere(3)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    LX = L.dense() @ m.V
    # Laplace-Beltrami of the position on the unit sphere is -2 x (H = 1)
    cosang = np.einsum("ij,ij->i", LX, -m.V) / np.linalg.norm(LX, axis=1)
    assert cosang.min() > 0.999
    # integrated: sum_i |(L X)_i| ~ 2 * area (area of the polyhedron ~ 4 pi)
    tri = m.V[m.F]
    area = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1).sum()
    assert abs(np.linalg.norm(LX, axis=1).sum() / (2 * area) - 1.0) < 0.02


def test_cotan_rejects_degenerate(oracle_mod):
    V = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], float)
    with pytest.raises(ValueError):
        oracle_mod.cotan_laplacian(V, np.array([[0, 1, 2]], np.int32))
    with pytest.raises(ValueError):
        oracle_mod.cotan_laplacian(V, np.array([[0, 1, 1]], np.int32))


# ----------------------------------------------------------------------------
# initialisation and L_t
# ----------------------------------------------------------------------------

def test_seed_layout(oracle_mod):
    F = oracle_mod.seed(6, np.array([4, 1], np.int32))
    D = F.dense()
    assert F.n_layers == 3
    expect = np.zeros((6, 3))
    expect[:, 2] = 1.0
    expect[4] = [1, 0, 0]
    expect[1] = [0, 1, 0]
    assert np.array_equal(D, expect)
    with pytest.raises(ValueError):
        oracle_mod.seed(6, np.array([1, 1], np.int32))
    with pytest.raises(ValueError):
        oracle_mod.seed(6, np.array([6], np.int32))


def random_field(oracle, n_v, n_layers, rng, density=0.3):
    D = rng.random((n_v, n_layers)) * (rng.random((n_v, n_layers)) < density)
    D[np.arange(n_v), rng.integers(0, n_layers, n_v)] += 0.1
    D /= D.sum(axis=1, keepdims=True)
    rows = [{l: D[i, l] for l in range(n_layers) if D[i, l] > 0} for i in range(n_v)]
    return make_field(oracle, rows, n_layers), D


@pytest.mark.parametrize("mesh", ["ico1", "grid6", "torus6"])
def test_lt_matches_dense_product(oracle_mod, mesh):
    m = {"ico1": lambda: synth.icosphere(1), "grid6": lambda: synth.planar_grid(6),
         "torus6": lambda: synth.noisy_torus(6)}[mesh]()
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    rng = np.random.default_rng(7)
    F, D = random_field(oracle_mod, m.n_v, 9, rng)
    G = oracle_mod.lt(L, F)
    ref = L.dense() @ D
    assert np.abs(G.dense() - ref).max() < 1e-13
    # pattern: exactly the layers present somewhere in the closed neighbourhood
    A = adjacency(L)
    struct = (A.astype(int) @ (D > 0).astype(int)) > 0
    pat = np.zeros_like(struct)
    rows = np.repeat(np.arange(m.n_v), np.diff(G.rowptr))
    pat[rows, G.ids] = True
    assert np.array_equal(pat, struct)


def test_skeleton_matches_dense_brute_force(oracle_mod):
    m = synth.planar_grid(8)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    rng = np.random.default_rng(3)
    F, D = random_field(oracle_mod, m.n_v, 7, rng, density=0.2)
    G = L.dense() @ D
    irows = (D > 0) | ((D == 0) & (G > 0))          # Algorithm 1, irows line
    _, sk, mg = oracle_mod.step(L, F, margins=True)
    assert np.array_equal(mg[:, 2].astype(int), irows.sum(axis=1))
    assert sk == irows.sum()


# ----------------------------------------------------------------------------
# the update: hand-derived special cases
# ----------------------------------------------------------------------------

PARAM_SETS = [
    {},                                                     # defaults
    dict(dt=1.0, mu=0.7, w_cb=0.05, a_cb=0.3, e_cb=0.9, e_bc=-0.4),
    dict(dt=5.0, mu=1.0, w_cc=0.2, w_cb=0.2, a_cc=1.0, a_cb=1.0, e_cc=0.2, e_cb=0.2, e_bc=0.2),
]


@pytest.mark.parametrize("params", PARAM_SETS)
@pytest.mark.parametrize("c", [1.0, 0.3])
def test_two_vertex_front(oracle_mod, params, c):
    """Operator [[-c, c], [c, -c]]; vertex 0 holds cell 0, vertex 1 the base.

    At vertex 1 the cell enters (G = c > 0) and at vertex 0 the base enters.
    By hand from Algorithm 1 with irows = {cell, base}, n = 2:
      d_cell(1) = (mu/2)(a_cb c - w_cb),  d_base(1) = -d_cell(1),
      d_cell(0) = -(mu/2)(a_cb c - w_cb), d_base(0) = -d_cell(0);
    the e terms vanish because one of the two values is 0.
    """
    p = dict(oracle_mod.DEFAULT_PARAMS)
    p.update(params)
    L = oracle_mod.operator_from_dense(np.array([[-c, c], [c, -c]]))
    F = make_field(oracle_mod, [{0: 1.0}, {1: 1.0}], 2)
    out, sk = oracle_mod.step(L, F, params)
    assert sk == 4
    g = (p["mu"] / 2) * (p["a_cb"] * c - p["w_cb"])
    v0 = normalise({0: clamp(1.0 - p["dt"] * g), 1: clamp(0.0 + p["dt"] * g)})
    v1 = normalise({0: clamp(0.0 + p["dt"] * g), 1: clamp(1.0 - p["dt"] * g)})
    for i, ref in enumerate([v0, v1]):
        got = row_dict(out, i)
        assert set(got) == set(ref)
        for l in ref:
            assert abs(got[l] - ref[l]) < 1e-14


def test_two_vertex_front_second_step_defaults(oracle_mod):
    """Second step of the case above with the default parameters and c = 1.

    After step 1: vertex 0 = {cell .9, base .1}, vertex 1 = {cell .1, base .9}.
    Step 2 by hand (a_cb = .04, w_cb = 0, e_cb = -e_bc = .5, mu = 1, dt = 5):
      vertex 0: G = (-.8, .8); d_cell = -.016 + .25 sqrt(.09) = .059 -> 1.195
                clamps to 1, the base to 0 and is dropped;
      vertex 1: G = (.8, -.8); d_cell = .016 + .075 = .091 -> .555, base .445.
    """
    L = oracle_mod.operator_from_dense(np.array([[-1.0, 1.0], [1.0, -1.0]]))
    F = make_field(oracle_mod, [{0: 1.0}, {1: 1.0}], 2)
    F, _ = oracle_mod.step(L, F)
    F, sk = oracle_mod.step(L, F)
    assert sk == 4
    assert row_dict(F, 0) == {0: 1.0}
    got = row_dict(F, 1)
    assert abs(got[0] - 0.555) < 1e-14 and abs(got[1] - 0.445) < 1e-14


@pytest.mark.parametrize("p_", [0.6, 0.25, 0.5])
@pytest.mark.parametrize("params", PARAM_SETS)
def test_isolated_vertex_two_cells(oracle_mod, p_, params):
    """One vertex, no neighbours (G = 0), cells 0 and 1 with values p, 1 - p.

    By hand: d_0 = -(mu/2) w_cc (1 - 2p) + (mu/2) e_cc sqrt(p (1 - p)) and the
    same with p -> 1 - p for cell 1.
    """
    p = dict(oracle_mod.DEFAULT_PARAMS)
    p.update(params)
    L = oracle_mod.operator_from_dense(np.zeros((1, 1)))
    F = make_field(oracle_mod, [{0: p_, 1: 1 - p_}], 3)
    out, _ = oracle_mod.step(L, F, params)
    s = math.sqrt(p_ * (1 - p_))
    d0 = -(p["mu"] / 2) * p["w_cc"] * (1 - 2 * p_) + (p["mu"] / 2) * p["e_cc"] * s
    d1 = -(p["mu"] / 2) * p["w_cc"] * (1 - 2 * (1 - p_)) + (p["mu"] / 2) * p["e_cc"] * s
    ref = normalise({0: clamp(p_ + p["dt"] * d0), 1: clamp(1 - p_ + p["dt"] * d1)})
    got = row_dict(out, 0)
    assert set(got) == set(ref)
    for l in ref:
        assert abs(got[l] - ref[l]) < 1e-14


@pytest.mark.parametrize("p_", [0.6, 0.1])
@pytest.mark.parametrize("params", PARAM_SETS)
def test_isolated_vertex_cell_and_base(oracle_mod, p_, params):
    """One vertex with cell 0 at p and the base at 1 - p, G = 0.

    By hand: d_cell = -(mu/2) w_cb (1 - 2p) + (mu/2) e_cb sqrt(p (1 - p)),
             d_base = -(mu/2) w_cb (2p - 1) + (mu/2) e_bc sqrt(p (1 - p)).
    """
    p = dict(oracle_mod.DEFAULT_PARAMS)
    p.update(params)
    L = oracle_mod.operator_from_dense(np.zeros((1, 1)))
    F = make_field(oracle_mod, [{0: p_, 1: 1 - p_}], 2)
    out, _ = oracle_mod.step(L, F, params)
    s = math.sqrt(p_ * (1 - p_))
    dc = -(p["mu"] / 2) * p["w_cb"] * (1 - 2 * p_) + (p["mu"] / 2) * p["e_cb"] * s
    db = -(p["mu"] / 2) * p["w_cb"] * (2 * p_ - 1) + (p["mu"] / 2) * p["e_bc"] * s
    ref = normalise({0: clamp(p_ + p["dt"] * dc), 1: clamp(1 - p_ + p["dt"] * db)})
    got = row_dict(out, 0)
    assert set(got) == set(ref)
    for l in ref:
        assert abs(got[l] - ref[l]) < 1e-14


def test_general_matrices_three_layers_by_hand(oracle_mod):
    """Dense coefficient matrices on an isolated vertex with three layers, G = 0.

    With G = 0 Algorithm 1 gives d_j = -(mu/3) sum_k [sum_l (w_jl - w_kl) F_l
    - e_jk sqrt(F_j F_k)]; evaluated here for one hand-picked matrix pair.
    """
    W = np.array([[0, .1, .3], [.1, 0, .2], [.3, .2, 0]])
    E = np.array([[0, .5, -.2], [-.5, 0, .4], [.2, -.4, 0]])
    Fv = np.array([.5, .3, .2])
    L = oracle_mod.operator_from_dense(np.zeros((1, 1)))
    F = make_field(oracle_mod, [{0: .5, 1: .3, 2: .2}], 3)
    out, _ = oracle_mod.step(L, F, dict(dt=1.0, mu=1.0), W=W, A=np.zeros((3, 3)), E=E)
    WF = W @ Fv                                   # sum_l w_jl F_l
    d = np.array([-(1 / 3) * sum((WF[j] - WF[k]) - E[j, k] * math.sqrt(Fv[j] * Fv[k]) for k in range(3))
                  for j in range(3)])
    ref = normalise({j: clamp(Fv[j] + d[j]) for j in range(3)})
    got = row_dict(out, 0)
    for l in ref:
        assert abs(got[l] - ref[l]) < 1e-14


def test_general_a_matrix_and_interest_layer_by_hand(oracle_mod):
    """The a_jl term and a layer entering through G > 0, on a two-vertex path.

    With L = [[-1, 1], [1, -1]], vertex 0 holds {0: .6, 1: .4} and vertex 1
    {0: .2, 2: .8}: at vertex 0, G = F_1 - F_0 = (-.4, -.4, .8), so layer 2
    joins the skeleton with F = 0.  With W = E = 0 the update of layer j is
    d_j = -(mu/n) sum_k (1/2) (A G)_j - (A G)_k over the skeleton, written
    here with matrix products over the skeleton only.
    """
    rng = np.random.default_rng(4)
    A = rng.random((3, 3))
    L = oracle_mod.operator_from_dense(np.array([[-1.0, 1.0], [1.0, -1.0]]))
    F = make_field(oracle_mod, [{0: .6, 1: .4}, {0: .2, 2: .8}], 3)
    dt, mu = 0.5, 1.0
    out, _ = oracle_mod.step(L, F, dict(dt=dt, mu=mu), W=np.zeros((3, 3)), A=A, E=np.zeros((3, 3)))
    Fv = np.array([.6, .4, 0.0])
    G = np.array([-.4, -.4, .8])
    AG = A @ G                                    # all three layers are in the skeleton
    n = 3
    d = -(mu / n) * 0.5 * (n * AG - AG.sum())
    ref = normalise({j: clamp(Fv[j] + dt * d[j]) for j in range(3)})
    got = row_dict(out, 0)
    assert set(got) == {j for j in ref if ref[j] > 0}
    for l in got:
        assert abs(got[l] - ref[l]) < 1e-14


def test_class_rule_as_matrices_equals_the_class_step(oracle_mod):
    """The class coefficients written out as dense matrices give the class step."""
    m = synth.planar_grid(14, seed=3)
    k = 6
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = oracle_mod.seed(m.n_v, synth.sample_seeds(m.n_v, k, 2))
    for _ in range(15):
        F, _ = oracle_mod.step(L, F)
    n = k + 1
    p = oracle_mod.DEFAULT_PARAMS
    cell = np.arange(n) < k
    both = np.outer(cell, cell)
    W = np.where(both, p["w_cc"], p["w_cb"])
    A = np.where(both, p["a_cc"], p["a_cb"])
    E = np.where(both, p["e_cc"], 0.0)
    E[cell, k] = p["e_cb"]
    E[k, cell] = p["e_bc"]
    for M in (W, A, E):
        np.fill_diagonal(M, 0.0)
    a, ska = oracle_mod.step(L, F)
    b, skb = oracle_mod.step(L, F, W=W, A=A, E=E)
    assert ska == skb and np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.ids, b.ids)
    assert np.abs(a.vals - b.vals).max() < 1e-15


def test_single_layer_is_fixed_point(oracle_mod):
    m = synth.planar_grid(12)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = make_field(oracle_mod, [{3: 1.0}] * m.n_v, 5)
    out, sk = oracle_mod.step(L, F)
    assert sk == m.n_v
    assert np.array_equal(out.rowptr, F.rowptr) and np.array_equal(out.ids, F.ids)
    assert np.array_equal(out.vals, F.vals)


# ----------------------------------------------------------------------------
# decision margins (the tie classifier of the GPU parity tests)
# ----------------------------------------------------------------------------
#
# orc_step reports per vertex how far its two discrete decisions are from
# flipping: [0] the irows test on an entry with F = 0 (|G| over the sum of the
# magnitudes of the products that make G), [1] the clamp at zero (|F + d dt|
# over |F| plus dt times the sum of the magnitudes of the terms of d, each G
# counted by its magnitude sum).  The parity tests exclude a row as a tie
# when either is below the tie threshold, so both are pinned here by hand.

def three_vertex_cancellation_operator():
    """L = [[0, .5, -.5], [.5, -.5, 0], [-.5, 0, .5]]: rows sum to zero and
    vertex 0 sees its two neighbours with opposite weights (a negative
    cotangent weight, as on jittered meshes)."""
    return np.array([[0.0, 0.5, -0.5], [0.5, -0.5, 0.0], [-0.5, 0.0, 0.5]])


@pytest.mark.parametrize("x1,x2,want", [(0.75, 0.25, 0.5), (0.25, 0.75, 0.5), (0.9, 0.1, 0.8), (0.5, 0.5, 0.0)])
def test_irows_margin_by_hand(oracle_mod, x1, x2, want):
    """Vertex 0 holds the base layer only; vertices 1 and 2 hold cell 0 at x1
    and x2 (the base layer at the rest).  Cell 0 is absent at vertex 0, so its
    irows test is on G(0, cell) = .5 x1 - .5 x2, whose magnitude sum is
    .5 x1 + .5 x2: margin |x1 - x2| / (x1 + x2).  With x1 = x2 the two
    products cancel exactly: margin 0, and the cell stays out of irows.
    Vertices 1 and 2 hold every layer of their neighbourhood: no such entry."""
    L = oracle_mod.operator_from_dense(three_vertex_cancellation_operator())
    F = make_field(oracle_mod, [{1: 1.0}, {0: x1, 1: 1 - x1}, {0: x2, 1: 1 - x2}], 2)
    _, _, mg = oracle_mod.step(L, F, margins=True)
    assert abs(mg[0, 0] - want) < 1e-15
    assert mg[1, 0] == math.inf and mg[2, 0] == math.inf
    assert mg[0, 2] == (2 if x1 > x2 else 1)          # the cell enters irows iff G > 0


def test_clamp_margin_with_cancelling_g_by_hand(oracle_mod):
    """The case above with x1 = .75, x2 = .25 and the default parameters
    (a_cb = .04, w_cb = 0, e_cb = -e_bc = .5, mu = 1, dt = 5).

    At vertex 0: G_cell = .25 (magnitude sum .5), G_base = .125 - .375 = -.25
    (magnitude sum .5); irows = {cell, base}, n = 2.
      cell: sum_{cell,base} = 1/2 (0 - a_cb) G_cell + 1/2 (a_cb - 0) G_base = -.01,
            its magnitude sum .02 (.02 * .5 twice), e term 0 (F_cell = 0):
            d = .005, d dt = .025, scale 0 + 5 * (.02 / 2) = .05 -> margin .5;
      base: sum = +.01, d = -.005, value .975, scale 1 + .05 -> margin .975 / 1.05.
    Counting G by |G| (.25) instead of its magnitude sum (.5) would give 1.
    """
    L = oracle_mod.operator_from_dense(three_vertex_cancellation_operator())
    F = make_field(oracle_mod, [{1: 1.0}, {0: 0.75, 1: 0.25}, {0: 0.25, 1: 0.75}], 2)
    out, _, mg = oracle_mod.step(L, F, margins=True)
    assert abs(mg[0, 1] - 0.5) < 1e-14
    got = row_dict(out, 0)
    assert abs(got[0] - 0.025) < 1e-14 and abs(got[1] - 0.975) < 1e-14


def test_two_vertex_front_margins_by_hand(oracle_mod):
    """Operator [[-1, 1], [1, -1]], vertex 0 = {cell 1.0}, vertex 1 = {base 1.0},
    default parameters.  Vertex 1: the cell enters with G = 1 from one product
    (margin 1); irows = {cell, base}; cell: sum = -.02 - .02 = -.04 over a
    magnitude sum .04, d = .02, value .1 over scale 5 * .02 = .1 -> 1;
    base: value .9 over scale 1.1 -> 9/11.  Vertex 0 is the mirror image."""
    L = oracle_mod.operator_from_dense(np.array([[-1.0, 1.0], [1.0, -1.0]]))
    F = make_field(oracle_mod, [{0: 1.0}, {1: 1.0}], 2)
    _, _, mg = oracle_mod.step(L, F, margins=True)
    for i in range(2):
        assert abs(mg[i, 0] - 1.0) < 1e-15
        assert abs(mg[i, 1] - 9.0 / 11.0) < 1e-14
        assert mg[i, 2] == 2


@pytest.mark.parametrize("p_,want", [(0.6, 1.0 / 3.0), (0.3, 0.125), (0.75, 0.0), (0.25, 0.0)])
def test_isolated_two_cells_clamp_margin_by_hand(oracle_mod, p_, want):
    """One vertex, G = 0, cells at p and 1 - p, default parameters (w_cc = .2,
    e_cc = 0, mu = 1, dt = 5).  For cell 0 the double sum is w (1 - 2p) with
    magnitude sum w, so d = -(w/2)(1 - 2p) and the scale is p + dt w / 2;
    cell 1 likewise with p -> 1 - p.
      p = .6:  cell 0 .7 / 1.1, cell 1 .3 / .9 = 1/3;
      p = .3:  cell 0 (.3 - .2) / (.3 + .5) = .125, cell 1 .9 / 1.2;
      p = .75: cell 1 lands exactly on the clamp, .25 - .25 = 0 (p = .25: cell 0)."""
    L = oracle_mod.operator_from_dense(np.zeros((1, 1)))
    F = make_field(oracle_mod, [{0: p_, 1: 1 - p_}], 3)
    _, _, mg = oracle_mod.step(L, F, margins=True)
    assert abs(mg[0, 1] - want) < 1e-14
    assert mg[0, 0] == math.inf                       # no entry with F = 0
    assert mg[0, 2] == 2


def test_isolated_cell_and_base_clamp_margin_by_hand(oracle_mod):
    """One vertex, G = 0, cell 0 at .6 and the base at .4, default parameters.
    Only the band terms act (w_cb = 0): cell d = +(1/2) e_cb s, base
    d = -(1/2) e_cb s with s = sqrt(.24); the cell's margin is 1 (one term),
    the base's |.4 - 1.25 s| / (.4 + 1.25 s)."""
    L = oracle_mod.operator_from_dense(np.zeros((1, 1)))
    F = make_field(oracle_mod, [{0: 0.6, 1: 0.4}], 2)
    _, _, mg = oracle_mod.step(L, F, margins=True)
    s = math.sqrt(0.24)
    assert abs(mg[0, 1] - (1.25 * s - 0.4) / (0.4 + 1.25 * s)) < 1e-14


def brute_force_margins(Ld, D, params, base):
    """Margins of one step from the dense operator and field, written from the
    definitions: every layer of the closed neighbourhood, Algorithm 1's double
    sum per interest entry with every term replaced by its magnitude (G by the
    magnitude sum of its products) for the scale."""
    p = params
    n_v, K = D.shape

    def coef(cc, cb, j, l):
        if j == l:
            return 0.0
        return cb if (j == base or l == base) else cc

    def ecoef(j, k):
        if j == k:
            return 0.0
        if j == base:
            return p["e_bc"]
        return p["e_cb"] if k == base else p["e_cc"]

    G = Ld @ D
    Ga = np.abs(Ld) @ D
    struct = (np.abs(Ld) > 0).astype(int) @ (D > 0).astype(int) > 0
    out = np.full((n_v, 3), math.inf)
    for i in range(n_v):
        cand = [l for l in range(K) if D[i, l] == 0 and struct[i, l] and Ga[i, l] > 0]
        if cand:
            out[i, 0] = min(abs(G[i, l]) / Ga[i, l] for l in cand)
        S = [l for l in range(K) if D[i, l] > 0 or (D[i, l] == 0 and struct[i, l] and G[i, l] > 0)]
        n = len(S)
        out[i, 2] = n
        for j in S:
            d = dabs = 0.0
            for k in S:
                s = sa = 0.0
                for l in S:
                    ca = 0.5 * (coef(p["a_cc"], p["a_cb"], j, l) - coef(p["a_cc"], p["a_cb"], k, l))
                    tw = (coef(p["w_cc"], p["w_cb"], j, l) - coef(p["w_cc"], p["w_cb"], k, l)) * D[i, l]
                    s += ca * G[i, l] + tw
                    sa += abs(ca) * Ga[i, l] + abs(tw)
                te = ecoef(j, k) * math.sqrt(D[i, j] * D[i, k])
                d += -(p["mu"] / n) * (s - te)
                dabs += (p["mu"] / n) * (sa + abs(te))
            v = D[i, j] + d * p["dt"]
            scale = D[i, j] + p["dt"] * dabs
            if scale > 0:
                out[i, 1] = min(out[i, 1], abs(v) / scale)
    return out


@pytest.mark.parametrize("params", PARAM_SETS)
@pytest.mark.parametrize("mesh", ["grid5", "torus5"])
def test_margins_match_brute_force(oracle_mod, params, mesh):
    m = {"grid5": lambda: synth.planar_grid(5, jitter=0.2, seed=2), "torus5": lambda: synth.noisy_torus(5)}[mesh]()
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    rng = np.random.default_rng(11)
    F, D = random_field(oracle_mod, m.n_v, 6, rng, density=0.35)
    p = dict(oracle_mod.DEFAULT_PARAMS)
    p.update(params)
    _, _, mg = oracle_mod.step(L, F, params, margins=True)
    want = brute_force_margins(L.dense(), D, p, base=5)
    assert np.array_equal(mg[:, 2], want[:, 2])
    for c in (0, 1):
        fin = np.isfinite(want[:, c])
        assert np.array_equal(fin, np.isfinite(mg[:, c]))
        assert np.abs(mg[fin, c] - want[fin, c]).max() < 1e-12


# ----------------------------------------------------------------------------
# literal triple loop vs closed form
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("params", PARAM_SETS + [dict(w_cc=0.35, w_cb=0.02, a_cc=0.07, a_cb=0.05,
                                                      e_cc=0.3, e_cb=0.8, e_bc=-0.1)])
@pytest.mark.parametrize("mesh", ["ico3", "grid24", "torus24"])
def test_literal_matches_closed_form(oracle_mod, params, mesh):
    m, k = {"ico3": (synth.icosphere(3), 16), "grid24": (synth.planar_grid(24), 20),
            "torus24": (synth.noisy_torus(24), 20)}[mesh]
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = oracle_mod.seed(m.n_v, synth.sample_seeds(m.n_v, k, 1))
    for t in range(40):
        a, ska = oracle_mod.step(L, F, params)
        b, skb = oracle_mod.step_closed(L, F, params)
        assert ska == skb
        assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.ids, b.ids)
        assert np.abs(a.vals - b.vals).max() < 1e-12
        F = a


# ----------------------------------------------------------------------------
# invariants of the iteration
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("mesh", ["ico3", "grid32", "torus32"])
def test_invariants_along_trajectory(oracle_mod, mesh):
    m, k = {"ico3": (synth.icosphere(3), 16), "grid32": (synth.planar_grid(32), 24),
            "torus32": (synth.noisy_torus(32), 24)}[mesh]
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    A = adjacency(L).astype(np.int32)
    F = oracle_mod.seed(m.n_v, synth.sample_seeds(m.n_v, k, 2))
    for t in range(120):
        Fn, _ = oracle_mod.step(L, F)
        # partition of unity (Eq. 1) and range
        rs = np.add.reduceat(Fn.vals, Fn.rowptr[:-1])
        assert np.abs(rs - 1.0).max() < 1e-12
        assert Fn.vals.min() > 0.0 and Fn.vals.max() <= 1.0
        # ids sorted, unique per row
        for i in range(0, m.n_v, 17):
            r = Fn.ids[Fn.rowptr[i]:Fn.rowptr[i + 1]]
            assert np.all(np.diff(r) > 0)
        # a layer reaches at most the 1-ring of its support per step
        before = F.dense() > 0
        reach = (A @ before.astype(np.int32)) > 0
        after = Fn.dense() > 0
        assert not np.any(after & ~reach)
        F = Fn
    lab = oracle_mod.labels(F)
    if mesh == "torus32":
        # the square (u, v) grid of the torus has cells of aspect ratio ~4, so
        # cotangent weights reach ~4 and dt = 5 sits above the explicit
        # diffusion limit there: the base layer lingers at a few vertices
        assert np.mean(lab >= 0) > 0.99
    else:
        assert np.all(lab >= 0)                  # the base layer is gone
    assert len(set(lab[lab >= 0].tolist())) == k  # every cell survives


def test_single_seed_grows_monotonically_and_covers(oracle_mod):
    m = synth.icosphere(3)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = oracle_mod.seed(m.n_v, np.array([5], np.int32))
    supp = F.dense()[:, 0] > 0
    covered_at = None
    for t in range(400):
        F, _ = oracle_mod.step(L, F)
        s = F.dense()[:, 0] > 0
        assert np.all(s[supp]), f"support shrank at step {t}"
        assert s.sum() > supp.sum() or s.all(), f"support stalled at step {t}"
        supp = s
        if supp.all() and covered_at is None:
            covered_at = t
        if np.all(oracle_mod.labels(F) == 0):
            break
    # one ring per step: the support reaches the antipode after ~ graph diameter steps
    assert covered_at is not None and covered_at < 40
    assert np.all(oracle_mod.labels(F) == 0)


def test_mirror_symmetric_seeds_give_mirror_partition(oracle_mod):
    m = synth.icosphere(3)
    key = {tuple(np.round(v, 9)): i for i, v in enumerate(m.V)}
    pi = np.array([key[tuple(np.round(v * np.array([-1, 1, 1]), 9))] for v in m.V])
    assert np.array_equal(pi[pi], np.arange(m.n_v))
    right = [v for v in synth.sample_seeds(m.n_v, 60, 9) if m.V[v, 0] > 0.1][:8]
    seeds = np.array(right + [pi[v] for v in right], np.int32)
    h = len(right)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = oracle_mod.seed(m.n_v, seeds)
    F, _ = oracle_mod.run(L, F, 150)
    lab = oracle_mod.labels(F)
    sigma = lambda l: -1 if l < 0 else (l + h) % (2 * h)
    # vertices on the mirror plane are fixed by the mirror: there the two mirrored
    # cells tie exactly, the sharpening term makes that tie unstable and rounding
    # picks a side; every other vertex must map onto its mirror image
    on_plane = np.abs(m.V[:, 0]) < 1e-12
    bad = [v for v in range(m.n_v) if not on_plane[v] and lab[pi[v]] != sigma(lab[v])]
    assert not bad
    assert len(set(lab.tolist())) == 2 * h


# ----------------------------------------------------------------------------
# labels
# ----------------------------------------------------------------------------

def test_labels_ties_and_base(oracle_mod):
    F = make_field(oracle_mod, [{0: .5, 2: .5}, {1: .3, 3: .7}, {2: .5, 3: .5}, {3: 1.0}, {1: .6, 2: .4}], 4)
    lab, mx = oracle_mod.labels(F, with_max=True)
    assert lab.tolist() == [0, -1, 2, -1, 1]
    assert mx.tolist() == [.5, .7, .5, 1.0, .6]


# ----------------------------------------------------------------------------
# semantic sanity (the paper's qualitative claims)
# ----------------------------------------------------------------------------

def test_sphere_partition_close_to_voronoi(oracle_mod):
    m = synth.icosphere(3)
    seeds = synth.sample_seeds(m.n_v, 16, 1)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F, _ = oracle_mod.run(L, oracle_mod.seed(m.n_v, seeds), 300)
    vor = np.argmin(((m.V[:, None, :] - m.V[seeds][None]) ** 2).sum(-1), axis=1)
    assert np.mean(oracle_mod.labels(F) == vor) > 0.93


def test_partition_insensitive_to_time_step(oracle_mod):
    m = synth.icosphere(3)
    seeds = synth.sample_seeds(m.n_v, 16, 1)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F5, _ = oracle_mod.run(L, oracle_mod.seed(m.n_v, seeds), 120, dict(dt=5.0))
    F1, _ = oracle_mod.run(L, oracle_mod.seed(m.n_v, seeds), 400, dict(dt=1.0))
    assert np.mean(oracle_mod.labels(F5) == oracle_mod.labels(F1)) > 0.95


# ----------------------------------------------------------------------------
# the threaded step (the timed CPU baseline) is the literal step
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("threads", [2, 3, 7, 0])
@pytest.mark.parametrize("params", PARAM_SETS[:2])
def test_threaded_step_is_identical(oracle_mod, threads, params):
    """Several threads over vertex ranges give the single-thread step's
    arrays bit for bit, margins and skeleton size included, along a
    trajectory with growing and shrinking rows."""
    m = synth.noisy_torus(20)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F = oracle_mod.seed(m.n_v, synth.sample_seeds(m.n_v, 24, 2))
    for _ in range(25):
        a, ska, ma = oracle_mod.step(L, F, params, margins=True)
        b, skb, mb = oracle_mod.step(L, F, params, margins=True, threads=threads)
        assert ska == skb
        for x, y in ((a.rowptr, b.rowptr), (a.ids, b.ids), (a.vals, b.vals), (ma, mb)):
            assert np.array_equal(x, y)
        F = a


def test_threaded_step_with_matrices_and_tiny_meshes(oracle_mod):
    rng = np.random.default_rng(5)
    m = synth.planar_grid(7, jitter=0.2, seed=2)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    F, _ = random_field(oracle_mod, m.n_v, 5, rng, density=0.4)
    W, A, E = (rng.random((5, 5)) * 0.3 for _ in range(3))
    a, ska = oracle_mod.step(L, F, W=W, A=A, E=E)
    b, skb = oracle_mod.step(L, F, W=W, A=A, E=E, threads=4)
    assert ska == skb and np.array_equal(a.vals, b.vals) and np.array_equal(a.ids, b.ids)
    # more threads than vertices
    L1 = oracle_mod.operator_from_dense(np.array([[-1.0, 1.0], [1.0, -1.0]]))
    F1 = make_field(oracle_mod, [{0: 1.0}, {1: 1.0}], 2)
    a, _ = oracle_mod.step(L1, F1)
    b, _ = oracle_mod.step(L1, F1, threads=8)
    assert np.array_equal(a.vals, b.vals) and np.array_equal(a.rowptr, b.rowptr)


def test_band_term_is_what_separates_the_fields(oracle_mod):
    """Sec. 3.1 states that dropping the band term g would remove the
    separation between the fields.  Under the readings used here (the band
    term acts between a cell and the base layer, e_cb = -e_bc = e), e = 0
    leaves every vertex to the base layer after 400 steps, the cells spread
    thin and never dominate anywhere, while e = .5 (and already e = .1)
    gives a partition: nearly every vertex belongs to a cell, most with a
    dominant value above .9."""
    m = synth.planar_grid(40, jitter=0.2, seed=2)
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    seeds = synth.sample_seeds(m.n_v, 12, 4)
    res = {}
    for e in (0.0, 0.1, 0.5):
        F, _ = oracle_mod.run(L, oracle_mod.seed(m.n_v, seeds), 400, dict(e_cb=e, e_bc=-e))
        lab, mx = oracle_mod.labels(F, with_max=True)
        res[e] = (np.mean(lab >= 0), np.mean(mx > 0.9))
    assert res[0.0] == (0.0, 0.0)
    for e in (0.1, 0.5):
        assert res[e][0] > 0.99 and res[e][1] > 0.7, res

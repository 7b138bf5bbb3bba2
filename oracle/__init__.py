"""Layered-field oracle: plain FP64 CPU reference (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_1804_09152_gb300``; the library never imports it.

The arithmetic lives in ``lf_oracle.c`` (compiled here with gcc, no fast-math,
no FMA contraction); this module only marshals numpy arrays.  Every function
follows a passage of Zayer et al., "Layered Fields for Natural Tessellations
on Surfaces" (arXiv 1804.09152), cited in the C source:

* ``cotan_laplacian`` -- the precomputed mesh Laplacian (Sec. 3.2),
* ``seed``            -- initialisation with seeds and the base layer (Sec. 3.1, 3.2),
* ``seed_regions``    -- the same with a seed's immediate neighbours (Sec. 3.2),
* ``lt``              -- the product L_t = Phi L^T of Algorithm 1 (Sec. 4),
* ``step``            -- one time-iteration of Algorithm 1 (Eq. 11-13, Sec. 4),
                         on one thread or, with the same result, on several
* ``step_closed``     -- the same update through its closed form for the
                         class coefficients (cross-check only),
* ``labels``          -- sharp labels, the layer of largest value (Sec. 6),
* ``lloyd_seeds``     -- one Lloyd-like seed update (Sec. 5), in ``tessellation.py``.

A field is a vertex-major CSR triple ``(rowptr int64[n_v+1], ids int32[nnz],
vals float64[nnz])``; row i lists the layers present at vertex i with ids
ascending, layers 0..k-1 for the seeds and k for the base layer.
"""
import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblf_oracle.so")
_lib = None

# Parameters of the update (see the coefficient block of lf_oracle.c):
# dt from Sec. 7; w = 0.2 and a = w / 5 from Sec. 3.1; mu and e are not given
# by the paper (mu = 1; e = 0.5 between a cell and the base layer).
DEFAULT_PARAMS = dict(dt=5.0, mu=1.0, w_cc=0.2, w_cb=0.0, a_cc=0.04, a_cb=0.04,
                      e_cc=0.0, e_cb=0.5, e_bc=-0.5)
_COEF_ORDER = ("dt", "mu", "w_cc", "w_cb", "a_cc", "a_cb", "e_cc", "e_cb", "e_bc")

# Relative decision margin (``step(..., margins=True)``) below which a parity
# check treats a vertex's discrete decision as a tie that rounding may flip:
# about 800 FP32 ulps.  The tests, the smoke check and the documentation use
# this one value.
TIE_MARGIN = 1e-4


def build(force=False):
    """Compile the oracle into ``oracle/_build/liblf_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int32
        lib.orc_cotan_laplacian.restype = i64
        lib.orc_cotan_laplacian.argtypes = [i64, P, i64, P, P, P, P]
        lib.orc_seed.restype = ctypes.c_int
        lib.orc_seed.argtypes = [i64, i32, P, P, P, P]
        lib.orc_lt.restype = i64
        lib.orc_lt.argtypes = [i64, i32, P, P, P, P, P, P, i64, P, P, P]
        lib.orc_step.restype = i64
        lib.orc_step.argtypes = [i64, i32, P, P, P, P, P, P, P, P, P, P, i64, P, P, P, P, P]
        lib.orc_step_threads.restype = i64
        lib.orc_step_threads.argtypes = [i32, i64, i32, P, P, P, P, P, P, P, P, P, P, i64, P, P, P, P, P]
        lib.orc_step_closed.restype = i64
        lib.orc_step_closed.argtypes = [i64, i32, P, P, P, P, P, P, P, i64, P, P, P, P]
        lib.orc_labels.restype = ctypes.c_int
        lib.orc_labels.argtypes = [i64, i32, P, P, P, P, P]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Field:
    rowptr: np.ndarray   # int64 [n_v + 1]
    ids: np.ndarray      # int32 [nnz]
    vals: np.ndarray     # float64 [nnz]
    n_layers: int        # k + 1

    @property
    def n_v(self):
        return self.rowptr.size - 1

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def dense(self):
        D = np.zeros((self.n_v, self.n_layers))
        rows = np.repeat(np.arange(self.n_v), np.diff(self.rowptr))
        D[rows, self.ids] = self.vals
        return D

    def copy(self):
        return Field(self.rowptr.copy(), self.ids.copy(), self.vals.copy(), self.n_layers)


@dataclass
class Operator:
    rowptr: np.ndarray   # int64 [n_v + 1]
    col: np.ndarray      # int32
    val: np.ndarray      # float64

    @property
    def n_v(self):
        return self.rowptr.size - 1

    def dense(self):
        n = self.n_v
        D = np.zeros((n, n))
        rows = np.repeat(np.arange(n), np.diff(self.rowptr))
        np.add.at(D, (rows, self.col), self.val)
        return D


def cotan_laplacian(V, F):
    """Cotangent Laplacian of a triangle mesh (FP64 CSR with explicit diagonal)."""
    lib = _load()
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    n_v, n_f = V.shape[0], F.shape[0]
    rp = np.zeros(n_v + 1, np.int64)
    cap = n_v + 6 * n_f
    col = np.zeros(max(cap, 1), np.int32)
    val = np.zeros(max(cap, 1), np.float64)
    nnz = lib.orc_cotan_laplacian(n_v, _p(V), n_f, _p(F), _p(rp), _p(col), _p(val))
    if nnz < 0:
        raise ValueError(f"orc_cotan_laplacian failed ({nnz})")
    return Operator(rp, col[:nnz].copy(), val[:nnz].copy())


def operator_from_dense(D):
    """CSR of a dense symmetric operator, keeping the diagonal structurally."""
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    rp = [0]
    cols, vals = [], []
    for i in range(n):
        for j in range(n):
            if D[i, j] != 0.0 or i == j:
                cols.append(j)
                vals.append(D[i, j])
        rp.append(len(cols))
    return Operator(np.array(rp, np.int64), np.array(cols, np.int32), np.array(vals, np.float64))


def seed(n_v, seeds):
    """Initial field: seed s carries layer s, every other vertex the base layer k."""
    lib = _load()
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    k = seeds.size
    rp = np.zeros(n_v + 1, np.int64)
    ids = np.zeros(n_v, np.int32)
    vals = np.zeros(n_v, np.float64)
    rc = lib.orc_seed(n_v, k, _p(seeds), _p(rp), _p(ids), _p(vals))
    if rc != 0:
        raise ValueError(f"orc_seed failed ({rc})")
    return Field(rp, ids, vals, k + 1)


def seed_regions(L, seeds, rings=1):
    """Initial field with region seeds (Sec. 3.2, "Initialization": a vertex
    and its immediate neighbours set to 1).  Layer c goes to seed vertex
    seeds[c] and, with rings = 1, to its neighbours in L; a vertex reached by
    several seeds keeps its own seed's layer if it is a seed, else takes the
    lowest seed id; all other vertices hold the base layer k."""
    seeds = [int(x) for x in seeds]
    k = len(seeds)
    n_v = L.rowptr.size - 1
    owner = [None] * n_v
    seed_set = set(seeds)
    for c, v in enumerate(seeds):
        owner[v] = c                                   # seed vertices first
    if rings == 1:
        for c, v in enumerate(seeds):
            for q in range(L.rowptr[v], L.rowptr[v + 1]):
                j = int(L.col[q])
                if j == v or j in seed_set:
                    continue
                if owner[j] is None or c < owner[j]:
                    owner[j] = c
    ids = np.array([k if o is None else o for o in owner], np.int32)
    return Field(np.arange(n_v + 1, dtype=np.int64), ids, np.ones(n_v), k + 1)


def _coefs(params):
    p = dict(DEFAULT_PARAMS)
    for key, v in (params or {}).items():
        if key not in p:
            raise KeyError(f"unknown parameter {key!r}")
        p[key] = v
    return np.array([p[k] for k in _COEF_ORDER], np.float64)


def lt(L, F):
    """L_t of Algorithm 1 in vertex-major form: G = L F with the structural pattern."""
    lib = _load()
    cap = max(8 * (F.nnz + F.n_v), 64)
    while True:
        rp = np.zeros(F.n_v + 1, np.int64)
        ids = np.zeros(cap, np.int32)
        vals = np.zeros(cap, np.float64)
        r = lib.orc_lt(F.n_v, F.n_layers, _p(L.rowptr), _p(L.col), _p(L.val),
                       _p(F.rowptr), _p(F.ids), _p(F.vals), cap, _p(rp), _p(ids), _p(vals))
        if r <= -16:
            cap = int(-(r + 16)) + 16
            continue
        if r < 0:
            raise RuntimeError(f"orc_lt failed ({r})")
        return Field(rp, ids[:r].copy(), vals[:r].copy(), F.n_layers)


def _mat(M, n):
    if M is None:
        return None
    M = np.ascontiguousarray(M, dtype=np.float64)
    assert M.shape == (n, n)
    return M


def step(L, F, params=None, W=None, A=None, E=None, margins=False, threads=1):
    """One time-iteration of Algorithm 1 (literal triple loop).

    Returns ``(F_next, skeleton)`` or ``(F_next, skeleton, margins)`` where
    ``margins`` is (n_v, 3): the relative distance of the irows test and of
    the clamp to zero from flipping (see lf_oracle.c), and n_i.
    ``threads`` other than 1 runs the same per-vertex arithmetic on that many
    threads (0: every core; ``orc_step_threads``), with an identical result.
    """
    lib = _load()
    co = _coefs(params)
    n = F.n_layers
    Wm, Am, Em = _mat(W, n), _mat(A, n), _mat(E, n)
    cap = max(2 * F.nnz + 16, 64)
    sk = np.zeros(1, np.int64)
    mg = np.zeros((F.n_v, 3), np.float64) if margins else None
    while True:
        # written in full up to the returned count by the C side
        rp = np.empty(F.n_v + 1, np.int64)
        ids = np.empty(cap, np.int32)
        vals = np.empty(cap, np.float64)
        args = (F.n_v, n, _p(L.rowptr), _p(L.col), _p(L.val),
                _p(F.rowptr), _p(F.ids), _p(F.vals), _p(co), _p(Wm), _p(Am), _p(Em),
                cap, _p(rp), _p(ids), _p(vals), _p(sk), _p(mg))
        r = lib.orc_step(*args) if threads == 1 else lib.orc_step_threads(int(threads), *args)
        if r <= -16:
            cap = int(-(r + 16)) + 16
            continue
        if r < 0:
            raise RuntimeError(f"orc_step failed ({r})")
        out = Field(rp, ids[:r].copy(), vals[:r].copy(), n)
        return (out, int(sk[0]), mg) if margins else (out, int(sk[0]))


def step_closed(L, F, params=None):
    """Same step through the closed form (class coefficients only)."""
    lib = _load()
    co = _coefs(params)
    cap = max(2 * F.nnz + 16, 64)
    sk = np.zeros(1, np.int64)
    while True:
        rp = np.zeros(F.n_v + 1, np.int64)
        ids = np.zeros(cap, np.int32)
        vals = np.zeros(cap, np.float64)
        r = lib.orc_step_closed(F.n_v, F.n_layers, _p(L.rowptr), _p(L.col), _p(L.val),
                                _p(F.rowptr), _p(F.ids), _p(F.vals), _p(co),
                                cap, _p(rp), _p(ids), _p(vals), _p(sk))
        if r <= -16:
            cap = int(-(r + 16)) + 16
            continue
        if r < 0:
            raise RuntimeError(f"orc_step_closed failed ({r})")
        return Field(rp, ids[:r].copy(), vals[:r].copy(), F.n_layers), int(sk[0])


def run(L, F, n_steps, params=None, closed=False, callback=None, threads=1):
    """``n_steps`` time-iterations; returns the final field and sum of |skeleton|."""
    total = 0
    for t in range(n_steps):
        F, sk = (step_closed(L, F, params) if closed else step(L, F, params, threads=threads))
        total += sk
        if callback is not None:
            callback(t, F)
    return F, total


def labels(F, with_max=False):
    """Per-vertex layer of largest value (ties: lowest id); base layer -> -1."""
    lib = _load()
    lab = np.zeros(F.n_v, np.int32)
    mx = np.zeros(F.n_v, np.float64)
    lib.orc_labels(F.n_v, F.n_layers, _p(F.rowptr), _p(F.ids), _p(F.vals), _p(lab), _p(mx))
    return (lab, mx) if with_max else lab

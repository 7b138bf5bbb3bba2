"""ctypes binding of the C ABI in ``include/lf.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
layered-field arithmetic: the work runs in ``_build/liblf.so`` (or the build of
the same sources that LF_LIBRARY names).  Importing this module raises if the
library has not been built; there is no fallback.

Device memory and streams may come from PyTorch: ``torch_device()`` returns an
``lf_device`` that allocates through the caching allocator of the current
device and runs on its current stream.
"""
import ctypes
import os

import numpy as np

from .native import LIB as _DEFAULT_LIB

# LF_LIBRARY selects another build of the same sources (the bounds-checked
# test build); there is no other implementation to fall back to.
LIB = os.environ.get("LF_LIBRARY") or _DEFAULT_LIB
if not os.path.exists(LIB):
    raise ImportError(f"CUDA library {LIB} is missing: run paper_1804_09152_gb300.build() first")

_lib = ctypes.CDLL(LIB)

LF_OK, LF_ERR_INVALID, LF_ERR_OOM, LF_ERR_CUDA, LF_ERR_TIMEOUT, LF_ERR_STATE, LF_ERR_CAPACITY = range(7)
LF_F32, LF_BF16, LF_F16 = 0, 1, 2
DTYPES = {"f32": LF_F32, "bf16": LF_BF16, "f16": LF_F16}

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class lf_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("mu", ctypes.c_double),
                ("w_cc", ctypes.c_double), ("w_cb", ctypes.c_double),
                ("a_cc", ctypes.c_double), ("a_cb", ctypes.c_double),
                ("e_cc", ctypes.c_double), ("e_cb", ctypes.c_double), ("e_bc", ctypes.c_double),
                ("iso", ctypes.c_double),
                ("field_dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("initial_capacity", ctypes.c_int64)]


class lf_device(ctypes.Structure):
    _fields_ = [("cuda_stream", ctypes.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN),
                ("user", ctypes.c_void_p)]


class lf_stats_t(ctypes.Structure):
    _fields_ = [("n_v", ctypes.c_int64), ("n_layers", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("capacity", ctypes.c_int64), ("operator_nnz", ctypes.c_int64),
                ("skeleton_total", ctypes.c_uint64), ("nnz_io_total", ctypes.c_uint64),
                ("device_bytes", ctypes.c_int64), ("retries", ctypes.c_int32), ("map_slots", ctypes.c_int32),
                ("field_dtype", ctypes.c_int32), ("value_bytes", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lf_server_params(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("chunk_steps", ctypes.c_int32)]


class lf_job_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("n_v", ctypes.c_int64),
                ("steps", ctypes.c_int64), ("steps_done", ctypes.c_int64), ("arrival_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("finish_ns", ctypes.c_int64), ("skeleton_total", ctypes.c_uint64),
                ("device_bytes", ctypes.c_int64), ("lloyd_rounds", ctypes.c_int32), ("lloyd_done", ctypes.c_int32),
                ("dual_triangles", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class lf_server_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "done", "failed", "queued", "running", "bytes_in_use",
                                              "peak_bytes", "peak_running", "batches", "busy_ns")] + \
               [("skeleton_total", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


LF_JOB_QUEUED, LF_JOB_RUNNING, LF_JOB_DONE, LF_JOB_FAILED = range(4)

_P = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_lib.lf_default_params.argtypes = [ctypes.POINTER(lf_params)]
_lib.lf_default_params.restype = None
_lib.lf_create_mesh.argtypes = [ctypes.POINTER(lf_device), _P, _i64, _P, _i64, ctypes.POINTER(lf_params),
                                ctypes.POINTER(_P)]
_lib.lf_create_mesh.restype = ctypes.c_int
_lib.lf_create_mesh_csr.argtypes = [ctypes.POINTER(lf_device), _i64, _P, _P, _P, ctypes.POINTER(lf_params),
                                    ctypes.POINTER(_P)]
_lib.lf_create_mesh_csr.restype = ctypes.c_int
_lib.lf_seed_regions.argtypes = [_P, _P, _i32, _i32]
_lib.lf_seed_regions.restype = ctypes.c_int
_lib.lf_set_coefficients.argtypes = [_P, _i32, _P, _P, _P]
_lib.lf_set_coefficients.restype = ctypes.c_int
_lib.lf_seed.argtypes = [_P, _P, _i32]
_lib.lf_seed.restype = ctypes.c_int
_lib.lf_step.argtypes = [_P, _i32]
_lib.lf_step.restype = ctypes.c_int
_lib.lf_labels.argtypes = [_P, _P, _P]
_lib.lf_labels.restype = ctypes.c_int
_lib.lf_get_operator.argtypes = [_P, _P, _P, _P, _i64, ctypes.POINTER(_i64)]
_lib.lf_get_operator.restype = ctypes.c_int
_lib.lf_get_field.argtypes = [_P, _P, _P, _P, _i64, ctypes.POINTER(_i64)]
_lib.lf_get_field.restype = ctypes.c_int
_lib.lf_set_field.argtypes = [_P, _P, _P, _P, _i64, _i32]
_lib.lf_set_field.restype = ctypes.c_int
_lib.lf_stats.argtypes = [_P, ctypes.POINTER(lf_stats_t)]
_lib.lf_stats.restype = ctypes.c_int
_lib.lf_destroy_mesh.argtypes = [_P]
_lib.lf_destroy_mesh.restype = None
_lib.lf_status_string.argtypes = [ctypes.c_int]
_lib.lf_status_string.restype = ctypes.c_char_p
_lib.lf_last_error.argtypes = [_P]
_lib.lf_last_error.restype = ctypes.c_char_p
_lib.lf_step_batch.argtypes = [ctypes.POINTER(_P), _i32, ctypes.POINTER(_i32)]
_lib.lf_step_batch.restype = ctypes.c_int
_lib.lf_set_schedule.argtypes = [_P, _i32]
_lib.lf_set_schedule.restype = ctypes.c_int
_lib.lf_schedule.argtypes = [_P]
_lib.lf_schedule.restype = _i32
_lib.lf_tune.argtypes = [_P, _i32, ctypes.POINTER(_i32)]
_lib.lf_tune.restype = ctypes.c_int
_lib.lf_step_noalloc.argtypes = [_P, _i32, _i32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _i32,
                                 ctypes.POINTER(lf_params), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
_lib.lf_step_noalloc.restype = ctypes.c_int
_lib.lf_extract_dual.argtypes = [_P, _P, _i64, ctypes.POINTER(_i64)]
_lib.lf_extract_dual.restype = ctypes.c_int
_lib.lf_lloyd.argtypes = [_P, _i32, _i32, _P]
_lib.lf_lloyd.restype = ctypes.c_int
_lib.lf_server_default_params.argtypes = [ctypes.POINTER(lf_server_params)]
_lib.lf_server_default_params.restype = None
_lib.lf_server_create.argtypes = [ctypes.POINTER(lf_device), ctypes.POINTER(lf_server_params), ctypes.POINTER(_P)]
_lib.lf_server_create.restype = ctypes.c_int
_lib.lf_server_submit.argtypes = [_P, _P, _i64, _P, _i64, _P, _i32, _i32, _i32, _i32, ctypes.POINTER(lf_params),
                                  _i64, ctypes.POINTER(_i64)]
_lib.lf_server_dual_mesh.argtypes = [_P, _i64, _P, _i64, ctypes.POINTER(_i64)]
_lib.lf_server_dual_mesh.restype = ctypes.c_int
_lib.lf_server_submit.restype = ctypes.c_int
_lib.lf_server_wait.argtypes = [_P, _i64, ctypes.c_double, ctypes.POINTER(lf_job_info), _P, _i32]
_lib.lf_server_wait.restype = ctypes.c_int
_lib.lf_server_drain.argtypes = [_P, ctypes.c_double]
_lib.lf_server_drain.restype = ctypes.c_int
_lib.lf_server_stats.argtypes = [_P, ctypes.POINTER(lf_server_stats_t)]
_lib.lf_server_stats.restype = ctypes.c_int
_lib.lf_server_destroy.argtypes = [_P]
_lib.lf_server_destroy.restype = None

EXPORTED = ["lf_default_params", "lf_create_mesh", "lf_create_mesh_csr", "lf_seed", "lf_seed_regions",
            "lf_set_coefficients", "lf_step", "lf_labels",
            "lf_get_operator", "lf_get_field", "lf_set_field", "lf_stats", "lf_destroy_mesh", "lf_status_string", "lf_last_error",
            "lf_step_noalloc", "lf_step_batch", "lf_set_schedule", "lf_schedule", "lf_tune", "lf_lloyd", "lf_extract_dual", "lf_server_default_params", "lf_server_create",
            "lf_server_submit", "lf_server_wait", "lf_server_dual_mesh", "lf_server_drain", "lf_server_stats", "lf_server_destroy"]


class LFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.lf_status_string(status).decode()}: {msg}")
        self.status = status


def _check(status, mesh=None):
    if status != LF_OK:
        raise LFError(status, _lib.lf_last_error(mesh).decode(errors="replace"))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def lf_default_params(**overrides):
    p = lf_params()
    _lib.lf_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "field_dtype" and isinstance(v, str):
            v = DTYPES[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def torch_device(stream=None):
    """lf_device running on a torch stream with torch's caching allocator."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    dev_index = s.device.index if s.device.index is not None else torch.cuda.current_device()

    def _alloc(nbytes, cuda_stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev_index, s)
        except Exception:
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    d = lf_device()
    d.cuda_stream = s.cuda_stream
    d.alloc = _ALLOC_FN(_alloc)
    d.free = _FREE_FN(_free)
    d.user = None
    d._keep = (d.alloc, d.free, s)      # the callbacks must outlive the mesh
    return d


def lf_create_mesh(V, F, params=None, device=None):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    out = _P()
    st = _lib.lf_create_mesh(ctypes.byref(device) if device is not None else None, _ptr(V), V.shape[0], _ptr(F),
                             F.shape[0], ctypes.byref(params) if params is not None else None, ctypes.byref(out))
    _check(st)
    return out


def lf_create_mesh_csr(rowptr, col, val, params=None, device=None):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    out = _P()
    st = _lib.lf_create_mesh_csr(ctypes.byref(device) if device is not None else None, rowptr.size - 1,
                                 _ptr(rowptr), _ptr(col), _ptr(val),
                                 ctypes.byref(params) if params is not None else None, ctypes.byref(out))
    _check(st)
    return out


def lf_seed(mesh, seeds):
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    _check(_lib.lf_seed(mesh, _ptr(seeds), seeds.size), mesh)


def lf_seed_regions(mesh, seeds, rings):
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    _check(_lib.lf_seed_regions(mesh, _ptr(seeds), seeds.size, int(rings)), mesh)


def lf_set_coefficients(mesh, n_layers, W=None, A=None, E=None):
    """Dense FP32 coefficient matrices (None: class rule for that one)."""
    mats = []
    for M in (W, A, E):
        if M is None:
            mats.append(None)
            continue
        M = np.ascontiguousarray(M, dtype=np.float32)
        if M.shape != (n_layers, n_layers):
            raise ValueError(f"coefficient matrix must be {n_layers}x{n_layers}, got {M.shape}")
        mats.append(M)
    ptrs = [None if M is None else _ptr(M) for M in mats]
    _check(_lib.lf_set_coefficients(mesh, int(n_layers), *ptrs), mesh)


def lf_step(mesh, n_iters):
    _check(_lib.lf_step(mesh, int(n_iters)), mesh)


# the step kernel's resident CTAs per SM; the lean register-tier path with the
# full step for the tiles outside its shape; the lean gather with the other
# tiers per vertex
SCHEDULES = {"ctas4": 0, "ctas5": 1, "ctas3": 2, "hot": 3, "lean": 4}


def lf_set_schedule(mesh, schedule):
    _check(_lib.lf_set_schedule(mesh, SCHEDULES.get(schedule, schedule)), mesh)


def lf_schedule(mesh):
    return int(_lib.lf_schedule(mesh))


def lf_tune(mesh, trial_steps):
    out = _i32(-1)
    _check(_lib.lf_tune(mesh, int(trial_steps), ctypes.byref(out)), mesh)
    return int(out.value)


def lf_step_batch(meshes, n_iters):
    """Advances meshes[a] by n_iters[a] steps (or every mesh by one int) in shared launches."""
    arr = (_P * len(meshes))(*[m.h if isinstance(m, Mesh) else m for m in meshes])
    counts = [int(n_iters)] * len(meshes) if np.isscalar(n_iters) else [int(x) for x in n_iters]
    if len(counts) != len(meshes):
        raise ValueError("n_iters needs one count per mesh")
    cnt = (_i32 * max(1, len(counts)))(*counts)
    st = _lib.lf_step_batch(arr, len(meshes), cnt)
    if st != LF_OK:
        msgs = [_lib.lf_last_error(h).decode(errors="replace") for h in arr if h]
        msg = next((x for x in msgs if x), "") or _lib.lf_last_error(None).decode(errors="replace")
        raise LFError(st, msg)


def lf_lloyd(mesh, rounds, steps_per_round, k):
    """Lloyd-like rounds; returns the k seeds afterwards."""
    out = np.empty(k, np.int32)
    _check(_lib.lf_lloyd(mesh, int(rounds), int(steps_per_round), _ptr(out)), mesh)
    return out


def lf_extract_dual(mesh):
    """Oriented dual triangles over seed vertex ids, (n, 3) int32."""
    n = _i64()
    _check(_lib.lf_extract_dual(mesh, None, 0, ctypes.byref(n)), mesh)
    out = np.empty((n.value, 3), np.int32)
    _check(_lib.lf_extract_dual(mesh, _ptr(out), n.value, ctypes.byref(n)), mesh)
    return out


def lf_labels(mesh, n_v, with_max=False):
    lab = np.empty(n_v, np.int32)
    mx = np.empty(n_v, np.float32) if with_max else None
    _check(_lib.lf_labels(mesh, _ptr(lab), _ptr(mx)), mesh)
    return (lab, mx) if with_max else lab


def lf_get_field(mesh, n_v):
    """Returns (rowptr int64, layer int32, val float32)."""
    nnz = _i64()
    rp = np.empty(n_v + 1, np.int64)
    _check(_lib.lf_get_field(mesh, _ptr(rp), None, None, 0, ctypes.byref(nnz)), mesh)
    lay = np.empty(max(nnz.value, 1), np.int32)
    val = np.empty(max(nnz.value, 1), np.float32)
    _check(_lib.lf_get_field(mesh, _ptr(rp), _ptr(lay), _ptr(val), lay.size, ctypes.byref(nnz)), mesh)
    return rp, lay[:nnz.value].copy(), val[:nnz.value].copy()


def lf_get_operator(mesh, n_v):
    """Returns the stored off-diagonal operator (rowptr int64, col int32, val float32)."""
    nnz = _i64()
    rp = np.empty(n_v + 1, np.int64)
    _check(_lib.lf_get_operator(mesh, _ptr(rp), None, None, 0, ctypes.byref(nnz)), mesh)
    col = np.empty(max(nnz.value, 1), np.int32)
    val = np.empty(max(nnz.value, 1), np.float32)
    _check(_lib.lf_get_operator(mesh, _ptr(rp), _ptr(col), _ptr(val), col.size, ctypes.byref(nnz)), mesh)
    return rp, col[:nnz.value].copy(), val[:nnz.value].copy()


def lf_set_field(mesh, rowptr, layer, val, n_layers):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    layer = np.ascontiguousarray(layer, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float32)
    _check(_lib.lf_set_field(mesh, _ptr(rowptr), _ptr(layer), _ptr(val), layer.size, int(n_layers)), mesh)


def lf_stats(mesh):
    s = lf_stats_t()
    _check(_lib.lf_stats(mesh, ctypes.byref(s)), mesh)
    return s.as_dict()


def lf_destroy_mesh(mesh):
    _lib.lf_destroy_mesh(mesh)


def lf_step_noalloc(stream, n_v, n_layers, L_rowptr, L_colval, rows_in, head_in, ids_in, vals_in, rows_out,
                    head_out, ids_out, vals_out, tile_cap, params=None):
    """One step on caller-owned device buffers (integer device addresses).

    Returns (nnz_out, need_tile_cap); raises LFError on failure.
    """
    nnz = _i64(0)
    need = _i64(0)
    st = _lib.lf_step_noalloc(stream, n_v, n_layers, L_rowptr, L_colval, rows_in, head_in, ids_in, vals_in,
                              rows_out, head_out, ids_out, vals_out, tile_cap,
                              ctypes.byref(params) if params is not None else None,
                              ctypes.byref(nnz), ctypes.byref(need))
    if st != LF_OK:
        err = LFError(st, _lib.lf_last_error(None).decode(errors="replace"))
        err.need_tile_cap = need.value
        raise err
    return nnz.value, need.value


def lf_status_string(status):
    return _lib.lf_status_string(status).decode()


def lf_last_error(mesh=None):
    return _lib.lf_last_error(mesh).decode(errors="replace")


class Mesh:
    """Owns one lf_mesh handle; each method calls the entry point of the same name."""

    def __init__(self, V=None, F=None, params=None, device=None, csr=None, **overrides):
        if params is None:
            params = lf_default_params(**overrides)
        self.params = params
        self.device = device
        if csr is not None:
            self.n_v = len(csr[0]) - 1
            self.h = lf_create_mesh_csr(*csr, params=params, device=device)
        else:
            self.n_v = int(np.asarray(V).shape[0])
            self.h = lf_create_mesh(V, F, params=params, device=device)

    def seed(self, seeds):
        lf_seed(self.h, seeds)

    def seed_regions(self, seeds, rings=1):
        lf_seed_regions(self.h, seeds, rings)

    def set_coefficients(self, W=None, A=None, E=None):
        n = self.stats()["n_layers"]
        lf_set_coefficients(self.h, n, W, A, E)

    def step(self, n):
        lf_step(self.h, n)

    def set_schedule(self, schedule):
        """0 / "ctas4" (the default), 1 / "ctas5", 2 / "ctas3", 3 / "hot" or 4 / "lean": the same bits."""
        lf_set_schedule(self.h, schedule)

    @property
    def schedule(self):
        return lf_schedule(self.h)

    def tune(self, trial_steps=128):
        """The autotuner: times each schedule on this job (advancing it) and keeps the fastest."""
        return lf_tune(self.h, trial_steps)

    def labels(self, with_max=False):
        return lf_labels(self.h, self.n_v, with_max)

    def extract_dual(self):
        return lf_extract_dual(self.h)

    def lloyd(self, rounds, steps_per_round):
        return lf_lloyd(self.h, rounds, steps_per_round, self.stats()["n_layers"] - 1)

    def get_field(self):
        return lf_get_field(self.h, self.n_v)

    def get_operator(self):
        return lf_get_operator(self.h, self.n_v)

    def set_field(self, rowptr, layer, val, n_layers):
        lf_set_field(self.h, rowptr, layer, val, n_layers)

    def stats(self):
        return lf_stats(self.h)

    def close(self):
        if self.h:
            lf_destroy_mesh(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lf_server_default_params(**overrides):
    p = lf_server_params()
    _lib.lf_server_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def lf_server_create(params=None):
    out = _P()
    _check(_lib.lf_server_create(None, ctypes.byref(params) if params is not None else None, ctypes.byref(out)))
    return out


def lf_server_submit(server, V, F, seeds, n_iters, params=None, arrival_ns=0, lloyd_rounds=0, extract_dual=False):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    jid = _i64()
    _check(_lib.lf_server_submit(server, _ptr(V), V.shape[0], _ptr(F), F.shape[0], _ptr(seeds), seeds.size,
                                 int(n_iters), int(lloyd_rounds), 1 if extract_dual else 0,
                                 ctypes.byref(params) if params is not None else None,
                                 int(arrival_ns), ctypes.byref(jid)))
    return jid.value


def lf_server_dual_mesh(server, job_id):
    n = _i64()
    _check(_lib.lf_server_dual_mesh(server, int(job_id), None, 0, ctypes.byref(n)))
    out = np.empty((n.value, 3), np.int32)
    _check(_lib.lf_server_dual_mesh(server, int(job_id), _ptr(out), n.value, ctypes.byref(n)))
    return out


def lf_server_wait(server, job_id, timeout_s=0.0, n_v=None, release=False):
    """(status, info dict, labels or None); status LF_ERR_TIMEOUT while the job runs."""
    info = lf_job_info()
    labels = np.empty(n_v, np.int32) if n_v else None
    st = _lib.lf_server_wait(server, int(job_id), float(timeout_s), ctypes.byref(info), _ptr(labels),
                             1 if release else 0)
    if st == LF_ERR_INVALID:
        _check(st)
    return st, info.as_dict(), (labels if st == LF_OK else None)


def lf_server_drain(server, timeout_s):
    return _lib.lf_server_drain(server, float(timeout_s))


def lf_server_stats(server):
    s = lf_server_stats_t()
    _check(_lib.lf_server_stats(server, ctypes.byref(s)))
    return s.as_dict()


def lf_server_destroy(server):
    _lib.lf_server_destroy(server)


class Server:
    """Owns one lf_server handle; each method calls the entry point of the same name."""

    def __init__(self, **overrides):
        self.h = lf_server_create(lf_server_default_params(**overrides))

    def submit(self, V, F, seeds, n_iters, params=None, arrival_ns=0, lloyd_rounds=0, extract_dual=False,
               **overrides):
        if params is None and overrides:
            params = lf_default_params(**overrides)
        return lf_server_submit(self.h, V, F, seeds, n_iters, params, arrival_ns, lloyd_rounds, extract_dual)

    def dual_mesh(self, job_id):
        return lf_server_dual_mesh(self.h, job_id)

    def wait(self, job_id, timeout_s=0.0, n_v=None, release=False):
        return lf_server_wait(self.h, job_id, timeout_s, n_v, release)

    def drain(self, timeout_s):
        return lf_server_drain(self.h, timeout_s)

    def stats(self):
        return lf_server_stats(self.h)

    def close(self):
        if self.h:
            lf_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

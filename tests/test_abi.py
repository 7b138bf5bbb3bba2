"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
declared in include/lf.h, and rejects invalid arguments before any CUDA call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_09152_gb300 import native
    native.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(lf_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["lf_create_mesh", "lf_create_mesh_csr", "lf_seed", "lf_step", "lf_labels", "lf_get_field",
              "lf_set_field", "lf_stats", "lf_destroy_mesh", "lf_status_string", "lf_last_error",
              "lf_default_params"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    so = ctypes.CDLL(lib.LIB)
    for n in names:
        assert hasattr(so, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(lf_\w+)", out))
    assert set(names) <= exported
    assert set(lib.EXPORTED) <= exported


def test_default_params(lib):
    p = lib.lf_default_params()
    assert (p.dt, p.mu, p.w_cc, p.w_cb, p.a_cc, p.a_cb) == (5.0, 1.0, 0.2, 0.0, 0.04, 0.04)
    assert (p.e_cc, p.e_cb, p.e_bc, p.iso, p.field_dtype, p.initial_capacity) == (0.0, 0.5, -0.5, 0.25, 0, 0)


def test_default_params_match_oracle(lib):
    import oracle
    p = lib.lf_default_params()
    for k, v in oracle.DEFAULT_PARAMS.items():
        assert getattr(p, k) == v, k


def test_status_strings(lib):
    assert lib.lf_status_string(0) == "LF_OK"
    assert lib.lf_status_string(6) == "LF_ERR_CAPACITY"


@pytest.mark.parametrize("case", ["few_vertices", "face_range", "face_repeat", "zero_area", "bad_dt",
                                  "bad_dtype", "nonfinite"])
def test_create_rejects_invalid_input_without_gpu(lib, case):
    m = synth.planar_grid(4)
    V, F = m.V.copy(), m.F.copy()
    params = None
    if case == "few_vertices":
        V, F = V[:2], F[:0]
    elif case == "face_range":
        F[3, 1] = 99
    elif case == "face_repeat":
        F[2, 2] = F[2, 0]
    elif case == "zero_area":
        V[F[0, 1]] = V[F[0, 0]]
    elif case == "bad_dt":
        params = lib.lf_default_params(dt=0.0)
    elif case == "bad_dtype":
        params = lib.lf_default_params(field_dtype=7)
    elif case == "nonfinite":
        V[5, 0] = np.nan
    with pytest.raises(lib.LFError) as ei:
        lib.lf_create_mesh(V, F, params=params)
    assert ei.value.status == lib.LF_ERR_INVALID
    assert lib.lf_last_error(None)


def test_csr_create_rejects_invalid_input_without_gpu(lib):
    rp = np.array([0, 2, 1, 3], np.int64)           # not monotone
    with pytest.raises(lib.LFError):
        lib.lf_create_mesh_csr(rp, np.array([1, 2, 0], np.int32), np.ones(3))
    rp = np.array([0, 1, 2, 3], np.int64)
    with pytest.raises(lib.LFError):
        lib.lf_create_mesh_csr(rp, np.array([1, 5, 0], np.int32), np.ones(3))


def test_package_fails_loudly_without_library(tmp_path):
    code = ("import paper_1804_09152_gb300.native as b; b.LIB = '/nonexistent/liblf.so'\n"
            "try:\n    import paper_1804_09152_gb300._lib\nexcept ImportError as e:\n    print('RAISED', e)\n")
    out = subprocess.run(["python", "-c", code], capture_output=True, text=True, cwd=ROOT)
    assert "RAISED" in out.stdout


def test_server_and_batch_reject_invalid_input_without_gpu(lib):
    p = lib.lf_server_default_params()
    assert (p.hbm_budget_bytes, p.max_active, p.chunk_steps) == (150_000_000_000, 64, 256)
    out = ctypes.c_void_p()
    for bad in (dict(max_active=0), dict(max_active=65), dict(chunk_steps=0), dict(hbm_budget_bytes=0)):
        sp = lib.lf_server_default_params(**bad)
        assert lib._lib.lf_server_create(None, ctypes.byref(sp), ctypes.byref(out)) == lib.LF_ERR_INVALID, bad
        assert lib.lf_last_error(None)
    assert lib._lib.lf_server_create(None, None, None) == lib.LF_ERR_INVALID
    assert lib._lib.lf_server_wait(None, 1, 0.0, None, None, 0) == lib.LF_ERR_INVALID
    assert lib._lib.lf_server_drain(None, 0.0) == lib.LF_ERR_INVALID
    lib._lib.lf_server_destroy(None)
    cnt = (ctypes.c_int32 * 1)(3)
    assert lib._lib.lf_step_batch(None, 1, cnt) == lib.LF_ERR_INVALID
    arr = (ctypes.c_void_p * 1)(None)
    assert lib._lib.lf_step_batch(arr, 0, cnt) == lib.LF_ERR_INVALID
    assert lib._lib.lf_step_batch(arr, 1, cnt) == lib.LF_ERR_INVALID      # null mesh


def test_mesh_calls_reject_a_null_handle_without_gpu(lib):
    # every per-mesh entry point checks its handle before any CUDA call
    n = ctypes.c_int64()
    seeds = np.array([0, 1], np.int32)
    L = lib._lib
    assert L.lf_seed(None, lib._ptr(seeds), 2) == lib.LF_ERR_INVALID
    assert L.lf_seed_regions(None, lib._ptr(seeds), 2, 1) == lib.LF_ERR_INVALID
    assert L.lf_set_coefficients(None, 3, None, None, None) == lib.LF_ERR_INVALID
    assert L.lf_step(None, 1) == lib.LF_ERR_INVALID
    assert L.lf_labels(None, None, None) == lib.LF_ERR_INVALID
    assert L.lf_get_operator(None, None, None, None, 0, ctypes.byref(n)) == lib.LF_ERR_INVALID
    assert L.lf_get_field(None, None, None, None, 0, ctypes.byref(n)) == lib.LF_ERR_INVALID
    assert L.lf_lloyd(None, 1, 1, None) == lib.LF_ERR_INVALID
    assert L.lf_extract_dual(None, None, 0, ctypes.byref(n)) == lib.LF_ERR_INVALID
    st = lib.lf_stats_t()
    assert L.lf_stats(None, ctypes.byref(st)) == lib.LF_ERR_INVALID
    rp = np.array([0, 1], np.int64)
    lay = np.array([0], np.int32)
    val = np.array([1.0], np.float32)
    assert L.lf_set_field(None, lib._ptr(rp), lib._ptr(lay), lib._ptr(val), 1, 2) == lib.LF_ERR_INVALID
    assert L.lf_set_schedule(None, 0) == lib.LF_ERR_INVALID
    assert L.lf_schedule(None) == -1
    assert L.lf_tune(None, 8, None) == lib.LF_ERR_INVALID
    L.lf_destroy_mesh(None)                    # a no-op


def test_checked_build_compiles_and_exports_the_same_symbols():
    # the bounds-checked variant (-DLF_CHECKED) that the GPU tests compare
    # with the plain build: same sources, same entry points
    from paper_1804_09152_gb300 import native
    path = native.build(checked=True)
    so = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(so, n), n


def test_noalloc_validates_its_arguments_before_any_cuda_call(lib):
    # the addresses below are never dereferenced: every case fails a check
    # that comes before the first CUDA call
    A = 1 << 20                                    # a 16-byte aligned stand-in address

    def call(n_v=1000, n_layers=3, ptrs=None, tile_cap=768, params=None):
        p = [A] * 10 if ptrs is None else ptrs
        return lib._lib.lf_step_noalloc(None, n_v, n_layers, *p, tile_cap,
                                        ctypes.byref(params) if params is not None else None, None, None)

    assert call(ptrs=[A] * 9 + [None]) == lib.LF_ERR_INVALID
    assert call(n_v=0) == lib.LF_ERR_INVALID
    assert call(n_layers=1) == lib.LF_ERR_INVALID and call(n_layers=65537) == lib.LF_ERR_INVALID
    assert call(tile_cap=128) == lib.LF_ERR_INVALID and call(tile_cap=264) == lib.LF_ERR_INVALID
    assert call(n_v=2 ** 31 - 300, tile_cap=512) == lib.LF_ERR_CAPACITY
    assert call(ptrs=[A, A + 4] + [A] * 8) == lib.LF_ERR_INVALID           # colval not 8-byte aligned
    assert call(ptrs=[A] * 3 + [A + 8] + [A] * 6) == lib.LF_ERR_INVALID    # head record not 16-byte aligned
    assert call(params=lib.lf_default_params(field_dtype="bf16")) == lib.LF_ERR_INVALID
    assert call(params=lib.lf_default_params(dt=0.0)) == lib.LF_ERR_INVALID
    assert "dt" in lib.lf_last_error(None)
    for bad in (dict(dt=float("inf")), dict(mu=float("nan")), dict(w_cc=float("nan")), dict(e_bc=-float("inf")),
                dict(a_cb=1e300), dict(dt=1e39)):
        assert call(params=lib.lf_default_params(**bad)) == lib.LF_ERR_INVALID, bad
    bad = lib.lf_default_params()
    bad.reserved = 1
    assert call(params=bad) == lib.LF_ERR_INVALID


def test_the_product_never_reaches_the_oracle():
    # the oracle is test infrastructure: the package has no path to it, and
    # bench.py imports it only inside the function that times the CPU baseline
    import ast
    pkg = os.path.join(ROOT, "paper_1804_09152_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            src = open(os.path.join(pkg, name)).read()
            assert "oracle" not in src, name
    for name in os.listdir(os.path.join(pkg, "csrc")):
        assert "oracle" not in open(os.path.join(pkg, "csrc", name)).read(), name
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                    users.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any("oracle" in ast.dump(n) for n in top)
    assert users == {"oracle_sample"}

"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/hspgemm.h (no compute call: this runs without a GPU)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hspgemm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_operations():
    names = declared_functions()
    for must in ("hs_spgemm", "hs_spref", "hs_spasgn", "hs_sparse", "hs_mat_free", "hs_strerror"):
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_1109_3739_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in hspgemm.h but not exported"


def test_status_strings_without_gpu():
    from paper_1109_3739_gb300 import hspgemm as H
    L = H.library()
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert L.hs_strerror(code)
    assert L.hs_version() >= 100


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1109_3739_gb300 import hspgemm as H
    monkeypatch.setattr(H, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(H, "_L", None)
    with pytest.raises(RuntimeError):
        H.library()


def test_tuning_round_trip_without_gpu():
    from paper_1109_3739_gb300 import hspgemm as H
    H.set_tuning(None)
    d = H.get_tuning()
    assert d == {"warp_s_max": 128, "mid_s_max": 1024, "large_s_max": 4096, "sym_mid_s_max": 1024,
                 "sym_heavy_from": 0, "sort_max": 1024, "sort_pct": 50, "spa_max": 0, "heavy_part_kb": 16, "num_heavy_from": 0}
    H.set_tuning({"mid_s_max": 512, "sym_heavy_from": 6144})
    d2 = H.get_tuning()
    assert d2["mid_s_max"] == 512 and d2["sym_heavy_from"] == 6144 and d2["warp_s_max"] == 128
    H.set_tuning(None)
    assert H.get_tuning() == d


def test_sparse_argument_checks_without_gpu():
    """hs_sparse rejects bad requests before any CUDA call (no GPU needed)."""
    from paper_1109_3739_gb300 import hspgemm as H
    L = H.library()
    L.hs_sparse.restype = ctypes.c_int
    vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.hs_sparse.argtypes = [vp, vp, vp, i64, i64, i64, ci, ci, ctypes.POINTER(H.hs_mat), vp, vp, ctypes.c_uint32]
    c = H.hs_mat()
    dummy = ctypes.c_int32(0)
    p = ctypes.addressof(dummy)  # never dereferenced: every call below fails its checks first
    PT, MP, OR, SEL = H.SEMIRING["plus_times"], H.SEMIRING["min_plus"], H.SEMIRING["or_and"], H.SEMIRING["select2nd"]
    F64, F32, I32, I64, BOOL = (H.DTYPE[k] for k in ("f64", "f32", "i32", "i64", "bool"))
    cases = [
        ((p, p, p, -1, 4, 4, F64, PT), -1),        # negative count
        ((p, p, p, 1, 4, 4, F64, SEL), -1),        # selector semirings combine nothing
        ((p, p, p, 1, 4, 4, I32, PT), -1),         # no int32 sum
        ((p, p, p, 1, 4, 4, F64, MP), -1),         # no f64 min
        ((p, p, p, 1, 4, 4, F32, OR), -1),         # or needs bool
        ((None, p, p, 1, 4, 4, F64, PT), -1),      # missing i
        ((p, p, None, 1, 4, 4, I64, PT), -1),      # missing values
        ((p, p, p, 1 << 31, 4, 4, F64, PT), -7),   # more tuples than int32 ids
        ((p, p, p, 1, 4, 1 << 31, BOOL, OR), -7),  # more columns than int32 ids
    ]
    for args, want in cases:
        got = L.hs_sparse(*args, ctypes.byref(c), None, None, 0)
        assert got == want, (args, got)
        assert not c.ptr and not c.idx and not c.val  # nothing left allocated


def test_noalloc_argument_checks_without_gpu():
    """hs_spgemm_noalloc rejects missing input arrays with HS_EINVAL before any
    CUDA call (a null offset or column array would otherwise be read by its
    first kernel), the same checks hs_spgemm makes."""
    from paper_1109_3739_gb300 import hspgemm as H
    L = H.library()
    L.hs_spgemm_noalloc.restype = ctypes.c_int
    L.hs_spgemm_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(H.hs_mat), ctypes.POINTER(H.hs_mat),
                                    ctypes.POINTER(H.hs_mat), ctypes.c_int64, ctypes.c_void_p]
    dummy = (ctypes.c_int64 * 8)()
    p = ctypes.addressof(dummy)  # never dereferenced: every call below fails its checks first
    PT, F32 = H.SEMIRING["plus_times"], H.DTYPE["f32"]

    def mat(m, n, nnz, ptr=p, idx=p, val=p):
        x = H.hs_mat()
        x.fmt, x.dtype, x.m, x.n, x.nnz = 0, F32, m, n, nnz  # HS_CSR
        x.ptr, x.idx, x.val = ptr, idx, val
        return x

    cases = [
        (mat(4, 4, 3, ptr=None), mat(4, 4, 3)),   # A without offsets
        (mat(4, 4, 3, idx=None), mat(4, 4, 3)),   # A without column ids
        (mat(4, 4, 3), mat(4, 4, 3, ptr=None)),   # B without offsets
        (mat(4, 4, 3), mat(4, 4, 3, idx=None)),   # B without column ids
        (mat(4, 4, 3, val=None), mat(4, 4, 3)),   # (+,x) without values
        (mat(4, 4, 3), mat(5, 4, 3)),             # inner dimensions differ
    ]
    for A, B in cases:
        C = mat(0, 0, 0)
        got = L.hs_spgemm_noalloc(PT, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), 16, None)
        assert got == -1, got
    # a missing C->ptr, and C->idx with a capacity
    A, B = mat(4, 4, 3), mat(4, 4, 3)
    for C in (mat(0, 0, 0, ptr=None), mat(0, 0, 0, idx=None)):
        assert L.hs_spgemm_noalloc(PT, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), 16, None) == -1

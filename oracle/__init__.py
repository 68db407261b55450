"""CPU oracle for SpGEMM / SpRef / SpAsgn (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It is a plain C implementation (``oracle.c``) of the
definitions in Buluc & Gilbert, driven through ctypes, plus a pure-Python dense
brute force (``brute.py``) for tiny inputs.  It shares no code with the CUDA
library and never imports it.

Pinned against: dense brute force on tiny inputs, identity and permutation
products, transpose and associativity identities, the Galerkin closed form,
the SpRef/SpAsgn identities of Section 3, the DCSC worked example of
Section 2.2, and for sparse(): SciPy's COO->CSR duplicate summation, a
pure-Python dictionary build and the SpRef identity with sparse()-built
selection matrices (see tests/test_oracle_*.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SEMIRINGS = {"plus_times": 0, "or_and": 1, "min_plus": 2, "select2nd": 3, "select1st": 4}
TYPES = {"f64": 0, "f32": 1, "i32": 2, "i64": 3, "bool": 4}
_NP = {"f64": np.float64, "f32": np.float32, "i32": np.int32, "i64": np.int64}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, no FMA contraction, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-Wall", "-o", tmp, src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _ocsr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("p", ctypes.c_void_p), ("j", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("t", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, vp, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            P = ctypes.POINTER(_ocsr)
            lib.oracle_flops.restype = i64
            lib.oracle_flops.argtypes = [P, P, i64, i64, vp]
            lib.oracle_spgemm_symbolic.restype = i64
            lib.oracle_spgemm_symbolic.argtypes = [P, P, i64, i64, vp, ci]
            lib.oracle_spgemm_numeric.restype = ci
            lib.oracle_spgemm_numeric.argtypes = [ci, P, P, i64, i64, vp, vp, vp, vp, ci]
            lib.oracle_spref.restype = i64
            lib.oracle_spref.argtypes = [P, vp, i64, vp, i64, vp, vp, vp, vp]
            lib.oracle_spasgn.restype = i64
            lib.oracle_spasgn.argtypes = [P, vp, i64, vp, i64, P, ci, ci, vp, vp, vp, vp]
            lib.oracle_sparse.restype = i64
            lib.oracle_sparse.argtypes = [vp, vp, vp, i64, i64, i64, ci, ci, vp, vp, vp, vp, vp]
            lib.oracle_doubly_compress.restype = i64
            lib.oracle_doubly_compress.argtypes = [vp, i64, vp, vp]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Mat:
    """Keeps the numpy arrays alive while C sees them."""

    def __init__(self, A):
        self.rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(A.col, dtype=np.int32)
        self.val = None if A.val is None else np.ascontiguousarray(A.val)
        t = "bool" if A.val is None else A.dtype
        self.s = _ocsr(A.m, A.n, _ptr(self.rowptr), _ptr(self.col), _ptr(self.val), TYPES[t])
        self.ref = ctypes.byref(self.s)


class OCSR:
    """Result container: rowptr int64[m+1], col int32[nnz], val or None, dtype name."""

    def __init__(self, m, n, rowptr, col, val, dtype):
        self.m, self.n, self.rowptr, self.col, self.val, self.dtype = m, n, rowptr, col, val, dtype

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _csr(m, n, rowptr, col, val, dtype):
    return OCSR(m, n, rowptr, col, val, dtype)


def flops(A, B, r0: int = 0, r1: int | None = None):
    """(total, per-row) nonzero multiplications of A*B for rows r0..r1-1."""
    lib = _load()
    r1 = A.m if r1 is None else r1
    a, b = _Mat(A), _Mat(B)
    rf = np.zeros(max(r1 - r0, 0), dtype=np.int64)
    tot = lib.oracle_flops(a.ref, b.ref, r0, r1, _ptr(rf))
    return int(tot), rf


def out_type(sr: str, A, B) -> str:
    if sr == "or_and":
        return "bool"
    if sr == "select2nd":
        return B.dtype
    if sr == "select1st":
        return A.dtype
    return A.dtype


def spgemm(sr: str, A, B, r0: int = 0, r1: int | None = None, nthreads: int = 1,
           with_bound: bool = False):
    """C(r0:r1, :) = A(r0:r1, :) * B over semiring sr (row-wise Gustavson, dense SPA).

    Returns a CSR with r1-r0 rows (and the per-entry sum of |a||b| if with_bound).
    """
    if A.n != B.m:
        raise OracleError("inner dimensions differ")
    lib = _load()
    r1 = A.m if r1 is None else r1
    a, b = _Mat(A), _Mat(B)
    rows = max(r1 - r0, 0)
    rn = np.zeros(rows, dtype=np.int64)
    tot = lib.oracle_spgemm_symbolic(a.ref, b.ref, r0, r1, _ptr(rn), nthreads)
    if tot < 0:
        raise OracleError(f"symbolic failed: {tot}")
    cp = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(rn, out=cp[1:])
    ot = out_type(sr, A, B)
    cj = np.empty(tot, dtype=np.int32)
    cv = None if ot == "bool" else np.empty(tot, dtype=_NP[ot])
    bound = np.empty(tot, dtype=np.float64) if with_bound else None
    st = lib.oracle_spgemm_numeric(SEMIRINGS[sr], a.ref, b.ref, r0, r1, _ptr(cp), _ptr(cj),
                                   _ptr(cv), _ptr(bound), nthreads)
    if st != 0:
        raise OracleError(f"numeric failed: {st}")
    C = _csr(rows, B.n, cp, cj, cv, ot)
    return (C, bound) if with_bound else C


def spgemm_count(A, B, r0: int = 0, r1: int | None = None, nthreads: int = 1):
    """(nnz, per-row nnz) of C(r0:r1,:) = A*B (structure only)."""
    lib = _load()
    r1 = A.m if r1 is None else r1
    a, b = _Mat(A), _Mat(B)
    rn = np.zeros(max(r1 - r0, 0), dtype=np.int64)
    tot = lib.oracle_spgemm_symbolic(a.ref, b.ref, r0, r1, _ptr(rn), nthreads)
    if tot < 0:
        raise OracleError(f"symbolic failed: {tot}")
    return int(tot), rn


def spref(A, I, J):
    """B = A(I, J) by direct indexing (Section 3)."""
    lib = _load()
    a = _Mat(A)
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    rn = np.zeros(len(I), dtype=np.int64)
    tot = lib.oracle_spref(a.ref, _ptr(I), len(I), _ptr(J), len(J), _ptr(rn), None, None, None)
    if tot < 0:
        raise OracleError(f"spref failed: {tot}")
    cp = np.zeros(len(I) + 1, dtype=np.int64)
    np.cumsum(rn, out=cp[1:])
    cj = np.empty(tot, dtype=np.int32)
    cv = None if A.val is None else np.empty(tot, dtype=A.val.dtype)
    st = lib.oracle_spref(a.ref, _ptr(I), len(I), _ptr(J), len(J), _ptr(rn), _ptr(cp), _ptr(cj), _ptr(cv))
    if st < 0:
        raise OracleError(f"spref failed: {st}")
    return _csr(len(I), len(J), cp, cj, cv, A.dtype)


def spasgn(A, I, J, B, accumulate: bool = False, sr: str = "plus_times"):
    """C = A with A(I,J) = B (or A(I,J) += B with accumulate) by direct indexing (Section 3.1)."""
    lib = _load()
    a, b = _Mat(A), _Mat(B)
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    rn = np.zeros(A.m, dtype=np.int64)
    tot = lib.oracle_spasgn(a.ref, _ptr(I), len(I), _ptr(J), len(J), b.ref, int(accumulate),
                            SEMIRINGS[sr], _ptr(rn), None, None, None)
    if tot < 0:
        raise OracleError(f"spasgn failed: {tot}")
    cp = np.zeros(A.m + 1, dtype=np.int64)
    np.cumsum(rn, out=cp[1:])
    cj = np.empty(tot, dtype=np.int32)
    cv = None if A.val is None else np.empty(tot, dtype=A.val.dtype)
    st = lib.oracle_spasgn(a.ref, _ptr(I), len(I), _ptr(J), len(J), b.ref, int(accumulate),
                           SEMIRINGS[sr], _ptr(rn), _ptr(cp), _ptr(cj), _ptr(cv))
    if st < 0:
        raise OracleError(f"spasgn failed: {st}")
    return _csr(A.m, A.n, cp, cj, cv, A.dtype)


def sparse(i, j, v, m: int, n: int, sr: str = "plus_times", dtype: str | None = None,
           with_bound: bool = False):
    """C = sparse(i, j, v, m, n) (Section 2 notation), tuples sharing a position
    combined with sr's add in increasing tuple order (sum, min or or).

    v is None for dtype "bool".  With with_bound also returns, per entry of C,
    the sum of |v| over its tuples."""
    lib = _load()
    I = np.ascontiguousarray(i, dtype=np.int32)
    J = np.ascontiguousarray(j, dtype=np.int32)
    if len(I) != len(J):
        raise OracleError("i and j differ in length")
    if dtype is None:
        dtype = "bool" if v is None else {np.dtype(t): k for k, t in _NP.items()}[np.asarray(v).dtype]
    V = None if dtype == "bool" else np.ascontiguousarray(v, dtype=_NP[dtype])
    if V is not None and len(V) != len(I):
        raise OracleError("v differs in length")
    rn = np.zeros(max(m, 0), dtype=np.int64)
    tot = lib.oracle_sparse(_ptr(I), _ptr(J), _ptr(V), len(I), m, n, TYPES[dtype], SEMIRINGS[sr],
                            _ptr(rn), None, None, None, None)
    if tot < 0:
        raise OracleError(f"sparse failed: {tot}")
    cp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(rn, out=cp[1:])
    cj = np.empty(tot, dtype=np.int32)
    cv = None if dtype == "bool" else np.empty(tot, dtype=_NP[dtype])
    bound = np.empty(tot, dtype=np.float64)
    st = lib.oracle_sparse(_ptr(I), _ptr(J), _ptr(V), len(I), m, n, TYPES[dtype], SEMIRINGS[sr],
                           _ptr(rn), _ptr(cp), _ptr(cj), _ptr(cv), _ptr(bound))
    if st < 0:
        raise OracleError(f"sparse failed: {st}")
    C = _csr(m, n, cp, cj, cv, dtype)
    return (C, bound) if with_bound else C


def doubly_compress(ptr):
    """(JC, CP) of the doubly compressed form of a compressed-pointer array (Section 2.2)."""
    lib = _load()
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    dim = len(ptr) - 1
    nz = lib.oracle_doubly_compress(_ptr(ptr), dim, None, None)
    jc = np.empty(nz, dtype=np.int64)
    cp = np.empty(nz + 1, dtype=np.int64)
    lib.oracle_doubly_compress(_ptr(ptr), dim, _ptr(jc), _ptr(cp))
    return jc, cp

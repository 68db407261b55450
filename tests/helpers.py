"""Comparison helpers shared by the tests (no arithmetic of the method)."""
from __future__ import annotations

import numpy as np

from paper_1109_3739_gb300 import inputs as I

# per-entry tolerance factors: |c - c_ref| <= TOL[dtype] * sum |a||b|
TOL = {"f64": 1e-12, "f32": 1e-5}


def csr(m, n, rowptr, col, val, dtype):
    return I.CSR(m, n, np.asarray(rowptr, np.int64), np.asarray(col, np.int32), val, dtype)


def as_csr(X):
    """Any object with m, n, rowptr, col, val, dtype as an inputs.CSR."""
    return I.CSR(X.m, X.n, np.asarray(X.rowptr, np.int64), np.asarray(X.col, np.int32),
                 None if X.val is None else np.asarray(X.val), X.dtype)


def from_dense(D, dtype="f64", pattern=None):
    """CSR of a dense array; entries where pattern (default D != 0) holds are stored."""
    D = np.asarray(D)
    P = (D != 0) if pattern is None else np.asarray(pattern, bool)
    m, n = P.shape
    rows, cols = np.nonzero(P)
    rowptr = np.zeros(m + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=rowptr[1:])
    val = None if dtype == "bool" else D[rows, cols].astype(I.DTYPES[dtype])
    return I.CSR(m, n, rowptr, cols.astype(np.int32), val, dtype)


def transpose(A):
    """Aᵀ as CSR by a stable counting sort of the entries on their column."""
    rows = np.repeat(np.arange(A.m, dtype=np.int64), np.diff(A.rowptr))
    order = np.argsort(A.col, kind="stable")
    col = rows[order].astype(np.int32)
    rowptr = np.zeros(A.n + 1, np.int64)
    np.cumsum(np.bincount(A.col, minlength=A.n), out=rowptr[1:])
    val = None if A.val is None else A.val[order]
    return I.CSR(A.n, A.m, rowptr, col, val, A.dtype)


def assert_same_structure(C, R, what=""):
    assert C.m == R.m and C.n == R.n, f"{what}: shape {C.m}x{C.n} vs {R.m}x{R.n}"
    np.testing.assert_array_equal(np.asarray(C.rowptr), np.asarray(R.rowptr), err_msg=f"{what}: rowptr")
    np.testing.assert_array_equal(np.asarray(C.col), np.asarray(R.col), err_msg=f"{what}: col")


def assert_bitexact(C, R, what=""):
    assert_same_structure(C, R, what)
    if R.val is None:
        assert C.val is None or len(C.val) == len(R.col)
        return
    a = np.asarray(C.val)
    b = np.asarray(R.val)
    assert a.dtype == b.dtype, f"{what}: dtype {a.dtype} vs {b.dtype}"
    if a.dtype.kind == "f":
        same = (a.view(np.uint32 if a.itemsize == 4 else np.uint64) ==
                b.view(np.uint32 if b.itemsize == 4 else np.uint64))
        # +0 and -0 differ only in sign; treat them as equal
        same |= (a == 0) & (b == 0)
        bad = np.nonzero(~same)[0]
    else:
        bad = np.nonzero(a != b)[0]
    assert len(bad) == 0, f"{what}: {len(bad)} values differ, first at {bad[:5]}: {a[bad[:5]]} vs {b[bad[:5]]}"


def assert_within(C, R, bound, dtype, what=""):
    """Structure identical, values within TOL[dtype] * bound per entry."""
    assert_same_structure(C, R, what)
    a = np.asarray(C.val, dtype=np.float64)
    b = np.asarray(R.val, dtype=np.float64)
    err = np.abs(a - b)
    lim = TOL[dtype] * np.asarray(bound)
    bad = np.nonzero(err > lim)[0]
    assert len(bad) == 0, (f"{what}: {len(bad)} entries outside tolerance; worst ratio "
                           f"{(err / np.maximum(lim, 1e-300)).max():.3g} at {bad[:5]}")


def rand_sparse(m, n, density, seed, dtype, kind="signed"):
    """Random pattern with each entry present with the given probability."""
    u = I.uniform_f64(I.draws(seed, 11, 0, m * n)).reshape(m, n) if m * n else np.zeros((m, n))
    P = u < density
    vals = I.random_values(m * n, dtype, seed, stream=12, kind=kind)
    D = np.zeros((m, n)) if vals is None else vals.reshape(m, n)
    return from_dense(D, dtype, pattern=P)


def rows_of(C, rows):
    """CSR of the listed rows of C (host arrays)."""
    rp = np.asarray(C.rowptr)
    parts_j, parts_v, counts = [], [], []
    for r in rows:
        a, b = int(rp[r]), int(rp[r + 1])
        parts_j.append(np.asarray(C.col[a:b]))
        if C.val is not None:
            parts_v.append(np.asarray(C.val[a:b]))
        counts.append(b - a)
    rowptr = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = np.concatenate(parts_j) if parts_j else np.zeros(0, np.int32)
    val = None if C.val is None else (np.concatenate(parts_v) if parts_v else np.zeros(0))
    return I.CSR(len(rows), C.n, rowptr, col.astype(np.int32), val, C.dtype)

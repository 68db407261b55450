"""Pins of the oracle's sparse(i, j, v, m, n).

Section 2 defines sparse(i,j,v,m,n) as the m x n matrix with entry
(i(k), j(k)) = v(k); tuples naming one position are combined with the
semiring's add (sum, min or or).  Pinned against a pure-Python dictionary build
(brute.sparse), SciPy's COO->CSR conversion with duplicate summation, the
SpRef identity B = R*A*Q with R and Q built by sparse() as in the SpRef listing
of Section 3.1, and invariants that hold at any size: the total of the values
is kept, nnz(C) is the number of distinct positions, and
sparse(j,i,v) is the transpose of sparse(i,j,v).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact, assert_within, transpose

CASES = [("plus_times", "f64"), ("plus_times", "f32"), ("plus_times", "i64"),
         ("min_plus", "f32"), ("min_plus", "i32"), ("or_and", "bool")]


def _from_dict(d, m, n, dtype):
    keys = sorted(d)
    rowptr = np.zeros(m + 1, np.int64)
    for r, _ in keys:
        rowptr[r + 1] += 1
    np.cumsum(rowptr, out=rowptr)
    col = np.array([c for _, c in keys], np.int32)
    val = None if dtype == "bool" else np.array([d[k] for k in keys], dtype=I.DTYPES[dtype])
    return I.CSR(m, n, rowptr, col, val, dtype)


@pytest.mark.parametrize("sr,dt", CASES)
@pytest.mark.parametrize("m,n,nnz", [(7, 5, 60), (30, 40, 200), (1, 1, 9), (50, 3, 0)])
def test_sparse_vs_dictionary(sr, dt, m, n, nnz):
    i, j, v = I.random_tuples(m, n, nnz, seed=m * 1000 + nnz, dtype=dt)
    C, bound = oracle.sparse(i, j, v, m, n, sr, dtype=dt, with_bound=True)
    d, mag = brute.sparse(i, j, v, m, n, sr, with_bound=True)
    R = _from_dict(d, m, n, dt)
    # the dictionary folds in tuple order in Python floats (double) and so does the oracle
    assert_bitexact(C, R, f"{sr} {dt}")
    # the tolerance scale: per position, the sum of |v| over its tuples in
    # tuple order (double); the dictionary's keys sorted are C's entries
    ref_b = np.array([mag[key] for key in sorted(mag)], dtype=np.float64)
    np.testing.assert_array_equal(bound, ref_b, err_msg=f"bound {sr} {dt}")


def test_sparse_vs_scipy():
    sp = pytest.importorskip("scipy.sparse")
    m, n, nnz = 300, 200, 20000
    i, j, v = I.random_tuples(m, n, nnz, seed=5, dtype="f64")
    C, bound = oracle.sparse(i, j, v, m, n, with_bound=True)
    S = sp.coo_matrix((v, (i.astype(np.int64), j.astype(np.int64))), shape=(m, n)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    R = I.CSR(m, n, S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data, "f64")
    assert_within(C, R, bound, "f64", "vs scipy")
    # nonsquare and rows with no tuple
    assert np.count_nonzero(np.diff(C.rowptr)) <= m


@pytest.mark.parametrize("dt", ["f64", "i32", "bool"])
def test_sparse_builds_spref_selectors(dt):
    """R = sparse(1:len(I), I, 1, len(I), m), Q = sparse(J, 1:len(J), 1, n, len(J))
    and R*A*Q = A(I,J) (Section 3.1), with repeated indices in I and J."""
    A = I.er_matrix(45, 38, 4, seed=31, dtype=dt, kind="signed")
    Iv = I.random_sequence(45, 30, 7)
    Jv = I.random_sequence(38, 50, 8)
    R = oracle.sparse(np.arange(len(Iv)), Iv, None, len(Iv), A.m, "or_and", dtype="bool")
    Q = oracle.sparse(Jv, np.arange(len(Jv)), None, A.n, len(Jv), "or_and", dtype="bool")
    assert R.nnz == len(Iv) and Q.nnz == len(Jv)
    B = oracle.spgemm("select1st", oracle.spgemm("select2nd", R, A), Q)
    assert_bitexact(B, oracle.spref(A, Iv, Jv), f"R*A*Q {dt}")


@pytest.mark.parametrize("sr,dt", [("plus_times", "i64"), ("min_plus", "i32"), ("or_and", "bool")])
def test_sparse_invariants_rmat(sr, dt):
    i, j, v = I.rmat_tuples(10, 8, seed=3, dtype=dt, kind="signed")
    n = 1 << 10
    C = oracle.sparse(i, j, v, n, n, sr, dtype=dt)
    keys = np.unique(i.astype(np.int64) * n + j)
    assert C.nnz == len(keys)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(C.rowptr))
    np.testing.assert_array_equal(rows * n + C.col, keys)
    if sr == "plus_times":
        assert int(C.val.sum()) == int(v.sum())
    if sr == "min_plus":
        # every stored value is one of its position's tuples and none is smaller
        first = {}
        for k in range(len(i)):
            key = (int(i[k]), int(j[k]))
            first[key] = min(first.get(key, int(v[k])), int(v[k]))
        assert all(first[(int(r), int(c))] == int(x) for r, c, x in zip(rows, C.col, C.val))
    Ct = oracle.sparse(j, i, v, n, n, sr, dtype=dt)
    assert_bitexact(Ct, transpose(C), "sparse(j,i,v) = sparse(i,j,v)^T")


def test_sparse_keeps_cancellation_and_zero_values():
    # 1 + (-1) at (0,1) stays stored with value 0; an explicit 0 at (2,0) stays stored
    C = oracle.sparse([0, 2, 0], [1, 0, 1], np.array([1.0, 0.0, -1.0]), 3, 2)
    np.testing.assert_array_equal(C.rowptr, [0, 1, 1, 2])
    np.testing.assert_array_equal(C.col, [1, 0])
    np.testing.assert_array_equal(C.val, [0.0, 0.0])


def test_sparse_empty_and_errors():
    C = oracle.sparse([], [], np.zeros(0), 4, 3)
    assert C.m == 4 and C.n == 3 and C.nnz == 0 and list(C.rowptr) == [0] * 5
    C = oracle.sparse([], [], None, 0, 0, "or_and", dtype="bool")
    assert C.m == 0 and C.nnz == 0
    with pytest.raises(oracle.OracleError):
        oracle.sparse([0, 3], [0, 0], np.ones(2), 3, 1)
    with pytest.raises(oracle.OracleError):
        oracle.sparse([0], [-1], np.ones(1), 3, 1)
    with pytest.raises(oracle.OracleError):
        oracle.sparse([0], [0], np.ones(1, np.int32), 1, 1, "plus_times")  # no i32 sum
    with pytest.raises(oracle.OracleError):
        oracle.sparse([0], [0], np.ones(1), 1, 1, "select2nd")


def test_sparse_of_the_rmat_edge_list_is_the_rmat_matrix():
    """The edge list the sparse() workload starts from and the matrix the
    SpGEMM workload multiplies describe one graph: the oracle's or-combined
    construction has exactly rmat_matrix's structure."""
    i, j, _ = I.rmat_tuples(12, 8, seed=2, dtype="f32")
    C = oracle.sparse(i, j, None, 1 << 12, 1 << 12, "or_and", dtype="bool")
    R = I.rmat_matrix(12, 8, seed=2, dtype="f32")
    np.testing.assert_array_equal(C.rowptr, R.rowptr)
    np.testing.assert_array_equal(C.col, R.col)

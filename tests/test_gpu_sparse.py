"""GPU sparse(i, j, v, m, n) (hs_sparse through the C ABI) against the CPU oracle.

Structure, integer sums, minima and bool results are compared bit for bit;
floating-point sums, which the GPU forms in the value type (in input order,
runs of more than 32 tuples in 32 ordered slices), within TOL[dtype] x (sum
of |v| over the entry's tuples) per entry.  Shapes cover positions named
once, runs folded by one thread, runs of hundreds to 100000 tuples folded by a
warp, mostly distinct tuples with many empty rows, keys of 0 to 40 bits, and
the R-MAT edge lists of the paper's graph experiments (power-law rows,
repeated edges).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact, assert_within

pytestmark = pytest.mark.gpu

CASES = [("plus_times", "f64"), ("plus_times", "f32"), ("plus_times", "i64"),
         ("min_plus", "f32"), ("min_plus", "i32"), ("or_and", "bool")]


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


def check(i, j, v, m, n, sr, dt, what):
    got = H().sparse(i, j, v, m, n, add=sr, dtype=dt).to_host()
    ref, bound = oracle.sparse(i, j, v, m, n, sr, dtype=dt, with_bound=True)
    if sr == "plus_times" and dt in ("f64", "f32"):
        assert_within(got, ref, bound, dt, what)
    else:
        assert_bitexact(got, ref, what)


@pytest.mark.parametrize("sr,dt", CASES)
@pytest.mark.parametrize("m,n,nnz", [
    (7, 5, 60),             # every position repeated
    (300, 250, 5000),       # mixed
    (50000, 40000, 30000),  # mostly distinct, many empty rows
    (1000, 3, 20000),       # three columns: long runs of one position
    (5, 70000, 100000),     # five rows of ~20000 tuples
    (1, 1, 1),
    (2, 2, 5000),           # four positions of ~1250 tuples (runs folded by a warp each)
    (3, 40, 20000),         # 120 positions of ~170 tuples
    (1, 1, 100000),         # one position
])
def test_sparse_random(sr, dt, m, n, nnz):
    i, j, v = I.random_tuples(m, n, nnz, seed=m + n + nnz, dtype=dt)
    check(i, j, v, m, n, sr, dt, f"{sr} {dt} {m}x{n} nnz={nnz}")


@pytest.mark.parametrize("sr,dt", [("plus_times", "f32"), ("plus_times", "i64"), ("min_plus", "i32"),
                                   ("or_and", "bool")])
def test_sparse_rmat16_edges(sr, dt):
    i, j, v = I.rmat_tuples(16, 8, seed=4, dtype=dt, kind="signed")
    check(i, j, v, 1 << 16, 1 << 16, sr, dt, f"rmat16 {sr} {dt}")


def test_sparse_rmat20_edge_list():
    """The R-MAT scale-20 edge list (8 edges per vertex, duplicates kept) with
    f32 values, summed: the adjacency construction of the graph experiments."""
    i, j, v = I.rmat_tuples(20, 8, seed=2, dtype="f32")
    n = 1 << 20
    check(i, j, v, n, n, "plus_times", "f32", "rmat20 edge list")
    # its structure is the R-MAT matrix the SpGEMM experiments use
    S = H().sparse(i, j, None, n, n, add="or_and").to_host()
    R = I.rmat_matrix(20, 8, seed=2, dtype="f32")
    np.testing.assert_array_equal(np.asarray(S.rowptr), R.rowptr)
    np.testing.assert_array_equal(np.asarray(S.col), R.col)


def test_sparse_keeps_zero_sums_and_signed_zero():
    h = H()
    C = h.sparse([0, 2, 0], [1, 0, 1], np.array([1.0, 0.0, -1.0]), 3, 2).to_host()
    np.testing.assert_array_equal(np.asarray(C.rowptr), [0, 1, 1, 2])
    np.testing.assert_array_equal(np.asarray(C.col), [1, 0])
    np.testing.assert_array_equal(np.asarray(C.val), [0.0, 0.0])
    # (min,+) keeps -0.0 bit for bit: the selector value -0.0 leaves it unchanged
    C = h.sparse([0, 1], [0, 0], np.array([-0.0, 2.0], np.float32), 2, 1, add="min_plus").to_host()
    assert np.signbit(np.asarray(C.val)[0]) and np.asarray(C.val)[1] == 2.0


def test_sparse_empty_and_errors():
    h = H()
    C = h.sparse(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0), 4, 3).to_host()
    assert C.m == 4 and C.n == 3 and list(np.asarray(C.rowptr)) == [0] * 5
    C = h.sparse(np.zeros(0, np.int32), np.zeros(0, np.int32), None, 0, 0, add="or_and").to_host()
    assert C.m == 0 and C.nnz == 0
    for args, add in [(([0, 3], [0, 0], np.ones(2), 3, 1), "plus_times"),
                      (([0], [-1], np.ones(1), 3, 1), "plus_times"),
                      (([0], [0], np.ones(1, np.int32), 1, 1), "plus_times"),  # no i32 sum
                      (([0], [0], np.ones(1), 1, 1), "select2nd")]:
        with pytest.raises(h.HsError) as e:
            h.sparse(*args, add=add)
        assert e.value.code == -1

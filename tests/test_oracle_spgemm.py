"""Pins of the CPU oracle's SpGEMM against facts it does not compute itself.

- dense brute force over each semiring's definition (tiny shapes, empty cases)
- A*I = I*A = A and permutation products (row/column relabelling)
- flops = sum_k nnz(A(:,k)) * nnz(B(k,:)) and nnz(C) <= flops (Section 2)
- structure((+,x) on positive values) == structure((or,and))
- (A*B)^T == B^T * A^T and (A*B)*C == A*(B*C) where the semiring is exact
- SciPy's independent sparse product for (+,x) f64
- the Galerkin closed form R*A*R^T = 4 * Laplacian on the coarse grid
  (restriction experiments, Section 4.3.2), both parenthesisations
"""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import (assert_bitexact, assert_same_structure, assert_within, from_dense,
                           transpose)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SR_TYPES = [("plus_times", "f64"), ("plus_times", "f32"), ("plus_times", "i64"),
            ("or_and", "bool"), ("min_plus", "f32"), ("min_plus", "i32")]


def rand_sparse(m, n, density, seed, dtype, kind="signed"):
    """Random pattern with each entry present with the given probability."""
    u = I.uniform_f64(I.draws(seed, 11, 0, m * n)).reshape(m, n) if m * n else np.zeros((m, n))
    P = u < density
    vals = I.random_values(m * n, dtype, seed, stream=12, kind=kind)
    D = np.zeros((m, n)) if vals is None else vals.reshape(m, n)
    return from_dense(D, dtype, pattern=P)


SHAPES = [(0, 5, 4), (4, 0, 5), (5, 4, 0), (1, 7, 1), (7, 1, 7), (1, 1, 1), (6, 6, 6),
          (9, 13, 5), (16, 16, 16), (31, 17, 40)]


@pytest.mark.parametrize("sr,dt", SR_TYPES)
def test_brute_force(sr, dt):
    seed = 100
    for (m, k, n) in SHAPES:
        for dens in (0.0, 0.15, 0.5, 1.0):
            seed += 1
            A = rand_sparse(m, k, dens, seed, dt)
            B = rand_sparse(k, n, dens, seed + 5000, dt)
            C, bound = oracle.spgemm(sr, A, B, with_bound=True)
            pat, val, bnd = brute.spgemm(sr, A, B)
            np.testing.assert_array_equal(C.rowptr, np.concatenate([[0], np.cumsum(pat.sum(1))]))
            rows, cols = np.nonzero(pat)
            np.testing.assert_array_equal(C.col, cols)
            # the per-entry tolerance scale sum |a||b| of the floating-point
            # parity tests: same products, same ascending-k order of additions
            # in double, so equal; the exact semirings carry no scale
            if sr == "plus_times" and dt in ("f32", "f64"):
                ref_b = np.array([bnd[i][j] for i, j in zip(rows, cols)], dtype=np.float64)
                np.testing.assert_array_equal(bound, ref_b, err_msg=f"bound {dt} {m}x{k}x{n} d={dens}")
            else:
                assert not np.any(bound), f"{sr} {dt}: nonzero tolerance scale"
            if dt == "bool":
                assert C.val is None
                continue
            ref = np.array([val[i][j] for i, j in zip(rows, cols)], dtype=C.val.dtype)
            # same order of the same IEEE operations: equal, not merely close
            np.testing.assert_array_equal(C.val, ref, err_msg=f"{sr} {dt} {m}x{k}x{n} d={dens}")


def _identity_for(sr, dt, n):
    if sr == "or_and":
        return I.identity(n, "bool")
    E = I.identity(n, dt)
    if sr == "min_plus":  # multiplicative identity of (min,+) is 0
        E.val[:] = 0
    return E


@pytest.mark.parametrize("sr,dt", SR_TYPES)
def test_identity_products(sr, dt):
    A = rand_sparse(40, 40, 0.1, 7, dt)
    E = _identity_for(sr, dt, 40)
    assert_bitexact(oracle.spgemm(sr, A, E), A, "A*I")
    assert_bitexact(oracle.spgemm(sr, E, A), A, "I*A")


@pytest.mark.parametrize("dt", ["f64", "i64"])
def test_permutation_products(dt):
    A = I.er_matrix(300, 300, 6, seed=3, dtype=dt, kind="signed")
    p = I.random_permutation(300, seed=5)
    P = I.permutation_matrix(p, dt)
    # (P*A)(i,:) = A(p[i],:)
    PA = oracle.spgemm("plus_times", P, A)
    D = A.to_dense()
    pat = A.pattern()
    assert_bitexact(PA, from_dense(D[p, :], dt, pattern=pat[p, :]), "P*A")
    # (A*P)(:, p[k]) = A(:, k): column k moves to p[k]
    AP = oracle.spgemm("plus_times", A, P)
    D2 = np.zeros_like(D)
    pat2 = np.zeros_like(pat)
    D2[:, p] = D
    pat2[:, p] = pat
    assert_bitexact(AP, from_dense(D2, dt, pattern=pat2), "A*P")


def test_flops_and_nnz_bound():
    A = I.rmat_matrix(12, 8, seed=4, dtype="f64")
    B = I.er_matrix(4096, 4096, 5, seed=6, dtype="f64")
    tot, rf = oracle.flops(A, B)
    colcount = np.bincount(A.col, minlength=A.n)
    rowcount = np.diff(B.rowptr)
    assert tot == int((colcount.astype(np.int64) * rowcount).sum())
    nnz, rn = oracle.spgemm_count(A, B)
    assert nnz <= tot
    assert np.all(rn <= rf)


def test_structure_plus_times_equals_or_and():
    A = I.rmat_matrix(11, 8, seed=8, dtype="f64")  # values in [0,1): no cancellation
    C1 = oracle.spgemm("plus_times", A, A)
    C2 = oracle.spgemm("or_and", A.with_values("bool", 0), A.with_values("bool", 0))
    assert_same_structure(C1, C2, "structure")


@pytest.mark.parametrize("sr,dt", [("or_and", "bool"), ("plus_times", "i64"),
                                   ("min_plus", "f32"), ("min_plus", "i32")])
def test_transpose_identity(sr, dt):
    A = I.er_matrix(200, 150, 4, seed=9, dtype=dt, kind="signed")
    B = I.er_matrix(150, 220, 5, seed=10, dtype=dt, kind="signed")
    lhs = transpose(oracle.spgemm(sr, A, B))
    # B^T * A^T computes the same terms with the operands swapped; for (min,+)
    # a+b == b+a exactly, for the integer and boolean semirings everything is exact
    rhs = oracle.spgemm(sr, transpose(B), transpose(A))
    assert_bitexact(rhs, lhs, "(AB)^T vs B^T A^T")


@pytest.mark.parametrize("sr,dt", [("or_and", "bool"), ("plus_times", "i64"), ("min_plus", "i32")])
def test_associativity(sr, dt):
    A = I.er_matrix(120, 100, 3, seed=11, dtype=dt, kind="signed")
    B = I.er_matrix(100, 90, 4, seed=12, dtype=dt, kind="signed")
    C = I.er_matrix(90, 110, 3, seed=13, dtype=dt, kind="signed")
    lhs = oracle.spgemm(sr, oracle.spgemm(sr, A, B), C)
    rhs = oracle.spgemm(sr, A, oracle.spgemm(sr, B, C))
    assert_bitexact(lhs, rhs, "associativity")


def test_against_scipy_f64():
    sp = pytest.importorskip("scipy.sparse")
    A = I.er_matrix(4096, 4096, 8, seed=1, dtype="f64")
    C, bound = oracle.spgemm("plus_times", A, A, with_bound=True)
    S = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.m, A.n))
    R = (S @ S).tocsr()
    R.sort_indices()
    ref = I.CSR(R.shape[0], R.shape[1], R.indptr.astype(np.int64), R.indices.astype(np.int32),
                R.data, "f64")
    assert_within(C, ref, bound, "f64", "vs scipy")


def test_select_semirings_gather():
    A = I.er_matrix(50, 40, 4, seed=14, dtype="f64", kind="signed")
    rows = np.array([7, 2, 5, 7, 0], dtype=np.int32)
    R = I.CSR(5, 50, np.arange(6, dtype=np.int64), rows, None, "bool")
    RA = oracle.spgemm("select2nd", R, A)
    assert_bitexact(RA, from_dense(A.to_dense()[rows], "f64", pattern=A.pattern()[rows]), "R*A")
    cols = np.array([3, 3, 39, 0], dtype=np.int32)
    Q = I.CSR(40, 4, None, None, None, "bool")
    qrow = np.zeros(41, np.int64)
    order = np.argsort(cols, kind="stable")
    np.cumsum(np.bincount(cols, minlength=40), out=qrow[1:])
    Q = I.CSR(40, 4, qrow, order.astype(np.int32), None, "bool")
    AQ = oracle.spgemm("select1st", A, Q)
    assert_bitexact(AQ, from_dense(A.to_dense()[:, cols], "f64", pattern=A.pattern()[:, cols]), "A*Q")


def test_select_rejects_two_contributions():
    A = I.er_matrix(10, 10, 3, seed=15, dtype="f64")
    R = I.CSR(1, 10, np.array([0, 2], np.int64), np.array([1, 2], np.int32), None, "bool")
    B = I.CSR(10, 1, np.arange(11, dtype=np.int64), np.zeros(10, np.int32), np.ones(10), "f64")
    with pytest.raises(oracle.OracleError):
        oracle.spgemm("select2nd", R, B)


@pytest.mark.parametrize("nx", [8, 16])
def test_galerkin_closed_form(nx):
    A = I.laplacian7(nx, "f64")
    R = I.aggregation_R(nx, 2, "f64")
    RT = I.aggregation_RT(nx, 2, "f64")
    left = oracle.spgemm("plus_times", oracle.spgemm("plus_times", R, A), RT)
    right = oracle.spgemm("plus_times", R, oracle.spgemm("plus_times", A, RT))
    coarse = I.laplacian7(nx // 2, "f64")
    coarse.val = coarse.val * 4.0  # diag 24, off-diagonal -4
    assert_bitexact(left, coarse, "(R*A)*R^T")
    assert_bitexact(right, coarse, "R*(A*R^T)")


def test_oracle_threads_match_serial():
    A = I.rmat_matrix(12, 8, seed=16, dtype="f32")
    C1, b1 = oracle.spgemm("plus_times", A, A, with_bound=True, nthreads=1)
    C4, b4 = oracle.spgemm("plus_times", A, A, with_bound=True, nthreads=4)
    assert_bitexact(C4, C1, "threads")
    np.testing.assert_array_equal(b1, b4)


def test_row_block_equals_whole():
    A = I.rmat_matrix(11, 8, seed=17, dtype="f64")
    C = oracle.spgemm("plus_times", A, A)
    blk = oracle.spgemm("plus_times", A, A, r0=300, r1=900)
    a, b = C.rowptr[300], C.rowptr[900]
    np.testing.assert_array_equal(blk.rowptr, C.rowptr[300:901] - a)
    np.testing.assert_array_equal(blk.col, C.col[a:b])
    np.testing.assert_array_equal(blk.val, C.val[a:b])


@pytest.mark.slow
def test_rmat_table_scale21():
    """Table of R-MAT product statistics (Section 4.3.1) at scale 21, within 3 %."""
    g = json.load(open(os.path.join(GOLDEN, "rmat_product_stats.json")))
    row = [r for r in g["rows"] if r["scale"] == 21][0]
    A = I.rmat_matrix(21, g["edge_factor"], g["a"], g["b"], g["c"], seed=21, dtype="bool")
    B = I.rmat_matrix(21, g["edge_factor"], g["a"], g["b"], g["c"], seed=22, dtype="bool")
    mults, _ = oracle.flops(A, B)
    nnzc, _ = oracle.spgemm_count(A, B, nthreads=os.cpu_count() or 1)
    assert abs(A.nnz / 1e6 - row["nnzA_M"]) / row["nnzA_M"] < 0.03
    assert abs(B.nnz / 1e6 - row["nnzB_M"]) / row["nnzB_M"] < 0.03
    assert abs(2 * mults / 1e6 - row["flops_M"]) / row["flops_M"] < 0.03
    assert abs(nnzc / 1e6 - row["nnzC_M"]) / row["nnzC_M"] < 0.03

"""Pins of the oracle's SpRef / SpAsgn and of the doubly compressed format.

SpRef (Section 3): B = A(I,J) row t = A(I[t],:), column p = J[p], in index
order, duplicates allowed.  Pinned against dense fancy indexing, against the
triple product R*A*Q formed with the oracle's own SpGEMM and the Matlab
definitions of R and Q (Section 3.1 listing), the identity and inverse-
permutation round trips, flops(R*A) = nnz(R*A) <= nnz(A) (Section 3.1), and
the scatter figure of Section 3.2.

SpAsgn (Section 3.1): C = A + R*B*Q - S*A*T with the subtraction read as a
structural negation.  Pinned against dense assignment, the product form built
from the oracle's SpGEMM with the listing's R, Q, S, T, the round trips
spasgn(A,I,J,spref(A,I,J)) == A and spref(spasgn(A,I,J,B),I,J) == B, and
nnz(R*B*Q) = nnz(B) (proof of the SpAsgn theorem).
"""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import as_csr, assert_bitexact, from_dense, transpose

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sparse_bool(rows, cols, m, n):
    """sparse(rows, cols, 1, m, n) of the Matlab listings (distinct pairs), structure only."""
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    keys = np.sort(rows * n + cols)
    rowptr, col = I.csr_from_unique_sorted_keys(keys, m, n)
    return I.CSR(m, n, rowptr, col, None, "bool")


def spref_by_products(A, Iv, Jv):
    m, n = A.m, A.n
    R = sparse_bool(np.arange(len(Iv)), Iv, len(Iv), m)
    Q = sparse_bool(Jv, np.arange(len(Jv)), n, len(Jv))
    RA = oracle.spgemm("select2nd", R, A)
    return oracle.spgemm("select1st", RA, Q), RA


def dense_ref(A, Iv, Jv):
    D = A.to_dense()[np.ix_(Iv, Jv)]
    P = A.pattern()[np.ix_(Iv, Jv)]
    return from_dense(D, A.dtype, pattern=P)


@pytest.mark.parametrize("dt", ["f64", "f32", "i32", "i64", "bool"])
def test_spref_dense_and_products(dt):
    A = I.er_matrix(60, 50, 5, seed=21, dtype=dt, kind="signed")
    cases = [
        (I.random_subset_sorted(60, 20, 1), I.random_subset_sorted(50, 15, 2)),
        (I.random_unique_sequence(60, 25, 3), I.random_unique_sequence(50, 30, 4)),
        (I.random_sequence(60, 40, 5), I.random_sequence(50, 45, 6)),  # duplicates
        (np.zeros(0, np.int32), I.random_sequence(50, 5, 7)),
        (I.random_sequence(60, 5, 8), np.zeros(0, np.int32)),
        (np.arange(60, dtype=np.int32), np.arange(50, dtype=np.int32)),
    ]
    for Iv, Jv in cases:
        B = oracle.spref(A, Iv, Jv)
        assert_bitexact(B, dense_ref(A, Iv, Jv), "dense")
        Bp, RA = spref_by_products(A, Iv, Jv)
        assert_bitexact(B, Bp, "R*A*Q")
        # flops(R*A) = nnz(R*A) <= nnz(A) when I has no duplicates (Section 3.1)
        Rs = sparse_bool(np.arange(len(Iv)), Iv, len(Iv), A.m)
        f, _ = oracle.flops(Rs, A)
        assert f == RA.nnz
        if len(np.unique(Iv)) == len(Iv):
            assert RA.nnz <= A.nnz


def test_spref_identity_and_inverse_permutation():
    A = I.rmat_matrix(10, 8, seed=22, dtype="f64", kind="signed")
    n = A.n
    assert_bitexact(oracle.spref(A, np.arange(n), np.arange(n)), A, "identity")
    p = I.random_permutation(n, seed=23).astype(np.int32)
    inv = np.empty_like(p)
    inv[p] = np.arange(n, dtype=np.int32)
    Ap = oracle.spref(A, p, p)
    assert_bitexact(oracle.spref(Ap, inv, inv), A, "A(p,p)(p^-1,p^-1)")


def test_scatter_figure_R():
    g = json.load(open(os.path.join(GOLDEN, "scatter_R_example.json")))
    m = g["m"]
    Iv = np.array(g["I_1based"], np.int32) - 1
    R = sparse_bool(np.arange(len(Iv)), Iv, len(Iv), m)
    # R has one nonzero per row at column I[t]: R(t, I[t]) = 1
    np.testing.assert_array_equal(R.rowptr, np.arange(len(Iv) + 1))
    np.testing.assert_array_equal(R.col, Iv)
    A = I.er_matrix(m, m, 3, seed=24, dtype="f64")
    RA = oracle.spgemm("select2nd", R, A)
    rows = [A.row(int(i)) for i in Iv]
    np.testing.assert_array_equal(RA.col, np.concatenate([r[0] for r in rows]))
    np.testing.assert_array_equal(RA.val, np.concatenate([r[1] for r in rows]))


def dense_assign(A, Iv, Jv, B, accumulate=False, sr="plus_times"):
    D = A.to_dense().copy()
    P = A.pattern().copy()
    Bd, Bp = B.to_dense(), B.pattern()
    sub_d = D[np.ix_(Iv, Jv)]
    sub_p = P[np.ix_(Iv, Jv)]
    if accumulate:
        both = sub_p & Bp
        if sr == "min_plus":
            new = np.where(both, np.minimum(sub_d, Bd), np.where(Bp, Bd, sub_d))
        else:
            new = np.where(both, sub_d + Bd, np.where(Bp, Bd, sub_d))
        D[np.ix_(Iv, Jv)] = new
        P[np.ix_(Iv, Jv)] = sub_p | Bp
    else:
        D[np.ix_(Iv, Jv)] = Bd
        P[np.ix_(Iv, Jv)] = Bp
    return from_dense(D, A.dtype, pattern=P)


def spasgn_by_products(A, Iv, Jv, B):
    """C = A .* not(S*A*T) + R*B*Q with the listing's R, Q, S, T (Section 3.1)."""
    ma, na = A.m, A.n
    mb, nb = B.m, B.n
    R = sparse_bool(Iv, np.arange(mb), ma, mb)
    Q = sparse_bool(np.arange(nb), Jv, nb, na)
    S = sparse_bool(Iv, Iv, ma, ma)
    T = sparse_bool(Jv, Jv, na, na)
    RBQ = oracle.spgemm("select1st", oracle.spgemm("select2nd", R, B), Q)
    SAT = oracle.spgemm("select1st", oracle.spgemm("select2nd", S, A), T)
    assert RBQ.nnz == B.nnz  # nnz(R*B*Q) = nnz(B)
    RBQ, SAT = as_csr(RBQ), as_csr(SAT)
    keep = A.pattern() & ~SAT.pattern()
    D = np.where(keep, A.to_dense(), 0)
    P = keep | RBQ.pattern()
    D = np.where(RBQ.pattern(), RBQ.to_dense(), D)
    return from_dense(D, A.dtype, pattern=P)


@pytest.mark.parametrize("dt", ["f64", "f32", "i32", "i64", "bool"])
def test_spasgn_dense_and_products(dt):
    A = I.er_matrix(50, 45, 5, seed=25, dtype=dt, kind="signed")
    for s, (ni, nj) in enumerate([(10, 12), (1, 1), (50, 45), (0, 5), (7, 0)]):
        Iv = I.random_unique_sequence(50, ni, 30 + s)
        Jv = I.random_unique_sequence(45, nj, 40 + s)
        B = I.er_matrix(ni, nj, min(3, ni), seed=50 + s, dtype=dt, kind="signed") if nj and ni else \
            I.CSR(ni, nj, np.zeros(ni + 1, np.int64), np.zeros(0, np.int32),
                  I.random_values(0, dt, 1), dt)
        C = oracle.spasgn(A, Iv, Jv, B)
        assert_bitexact(C, dense_assign(A, Iv, Jv, B), "dense assign")
        assert_bitexact(C, spasgn_by_products(A, Iv, Jv, B), "product form")
        # round trips
        assert_bitexact(oracle.spref(C, Iv, Jv), B, "spref(spasgn(...))")
        assert_bitexact(oracle.spasgn(A, Iv, Jv, oracle.spref(A, Iv, Jv)), A, "spasgn(spref)")


@pytest.mark.parametrize("dt,sr", [("f64", "plus_times"), ("i64", "plus_times"), ("i32", "min_plus")])
def test_extend_add_dense(dt, sr):
    A = I.er_matrix(40, 40, 6, seed=26, dtype=dt, kind="signed")
    Iv = I.random_unique_sequence(40, 15, 60)
    Jv = I.random_unique_sequence(40, 12, 61)
    B = I.er_matrix(15, 12, 4, seed=62, dtype=dt, kind="signed")
    C = oracle.spasgn(A, Iv, Jv, B, accumulate=True, sr=sr)
    assert_bitexact(C, dense_assign(A, Iv, Jv, B, accumulate=True, sr=sr), "extend-add")


def test_spasgn_rejects_duplicates():
    A = I.er_matrix(20, 20, 3, seed=27, dtype="f64")
    B = I.er_matrix(2, 2, 1, seed=28, dtype="f64")
    with pytest.raises(oracle.OracleError):
        oracle.spasgn(A, np.array([3, 3], np.int32), np.array([1, 2], np.int32), B)


def test_entries_outside_block_unchanged():
    A = I.rmat_matrix(10, 8, seed=29, dtype="i64")
    Iv = I.random_unique_sequence(A.m, 100, 63)
    Jv = I.random_unique_sequence(A.n, 80, 64)
    B = I.er_matrix(100, 80, 2, seed=65, dtype="i64")
    C = oracle.spasgn(A, Iv, Jv, B)
    inI = np.zeros(A.m, bool)
    inI[Iv] = True
    inJ = np.zeros(A.n, bool)
    inJ[Jv] = True
    ra = np.repeat(np.arange(A.m), np.diff(A.rowptr))
    rc = np.repeat(np.arange(C.m), np.diff(C.rowptr))
    outside_a = ~(inI[ra] & inJ[A.col])
    outside_c = ~(inI[rc] & inJ[C.col])
    ka = ra[outside_a] * A.n + A.col[outside_a]
    kc = rc[outside_c] * C.n + C.col[outside_c]
    np.testing.assert_array_equal(ka, kc)
    np.testing.assert_array_equal(A.val[outside_a], C.val[outside_c])


def test_dcsc_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "dcsc_worked_example.json")))
    cp = np.array(g["csc_cp_1based"], np.int64) - 1
    jc, dcp = oracle.doubly_compress(cp)
    np.testing.assert_array_equal(jc, np.array(g["dcsc_jc_1based"]) - 1)
    np.testing.assert_array_equal(dcp, np.array(g["dcsc_cp_1based"]) - 1)
    # the CSC of A is the CSR of A^T: A^T row c holds IR entries of column c
    ir = np.array(g["csc_ir_1based"], np.int32) - 1
    AT = I.CSR(g["n"], g["m"], cp, ir, np.array(g["csc_num"]), "f64")
    A = transpose(AT)
    assert A.nnz == 4
    assert np.all(np.diff(A.rowptr) >= 0)

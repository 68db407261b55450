"""Output modes of hs_spgemm against the oracle: unsorted rows (HS_FLAG_UNSORTED:
the hash bins skip their sort, each row holds the same set of columns and
values in some order) and explicit-zero pruning (HS_FLAG_PRUNE_ZEROS: entries
whose (+,x) sum is exactly zero are removed)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact, assert_within

pytestmark = pytest.mark.gpu


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


def sort_rows(C):
    rp = np.asarray(C.rowptr)
    col = np.asarray(C.col).copy()
    val = None if C.val is None else np.asarray(C.val).copy()
    unsorted_rows = 0
    for r in range(C.m):
        a, b = int(rp[r]), int(rp[r + 1])
        if b - a > 1:
            o = np.argsort(col[a:b], kind="stable")
            if np.any(o != np.arange(b - a)):
                unsorted_rows += 1
            col[a:b] = col[a:b][o]
            if val is not None:
                val[a:b] = val[a:b][o]
    return I.CSR(C.m, C.n, rp.copy(), col, val, C.dtype), unsorted_rows


@pytest.mark.parametrize("dt", ["f64", "f32", "i64"])
def test_unsorted_rows_hold_the_product(dt):
    A = I.rmat_matrix(14, 8, seed=21, dtype=dt, kind="signed")
    h = H()
    dA = h.DeviceCSR.from_host(A)
    got, unsorted_rows = sort_rows(h.spgemm("plus_times", dA, dA, sorted_rows=False).to_host())
    ref, bound = oracle.spgemm("plus_times", A, A, with_bound=True)
    if dt == "i64":
        assert_bitexact(got, ref, "unsorted i64")
    else:
        assert_within(got, ref, bound, dt, f"unsorted {dt}")
    assert unsorted_rows > 0  # the hash bins did skip their sort


def test_unsorted_bool_and_min_plus():
    h = H()
    A = I.rmat_matrix(13, 8, seed=22, dtype="f32", kind="unit")
    dA = h.DeviceCSR.from_host(A)
    for sr in ("or_and", "min_plus"):
        got, _ = sort_rows(h.spgemm(sr, dA, dA, sorted_rows=False).to_host())
        assert_bitexact(got, oracle.spgemm(sr, A, A), f"unsorted {sr}")


def _pm1(A, dt):
    v = np.where(np.asarray(A.val) >= 0, 1, -1).astype(I.DTYPES[dt])
    return I.CSR(A.m, A.n, A.rowptr, A.col, v, dt)


def _drop_zeros(C):
    keep = np.asarray(C.val) != 0
    rows = np.repeat(np.arange(C.m), np.diff(C.rowptr))[keep]
    rp = np.zeros(C.m + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=C.m), out=rp[1:])
    return I.CSR(C.m, C.n, rp, np.asarray(C.col)[keep], np.asarray(C.val)[keep], C.dtype)


@pytest.mark.parametrize("dt", ["f64", "i64", "f32"])
def test_prune_zeros(dt):
    """Values +-1: many sums cancel exactly (every partial sum is a small
    integer, exact in every type); pruned = the oracle's product without its
    zero entries, bit for bit."""
    A = _pm1(I.er_matrix(3000, 4096, 6, seed=23, dtype="f64", kind="signed"), dt)
    B = _pm1(I.rmat_matrix(12, 8, seed=24, dtype="f64", kind="signed"), dt)
    h = H()
    dA, dB = h.DeviceCSR.from_host(A), h.DeviceCSR.from_host(B)
    ref = oracle.spgemm("plus_times", A, B)
    zeros = int(np.sum(np.asarray(ref.val) == 0))
    assert zeros > 0
    got = h.spgemm("plus_times", dA, dB, prune_zeros=True).to_host()
    assert_bitexact(got, _drop_zeros(ref), f"pruned {dt}")
    # other semirings ignore the flag
    got = h.spgemm("or_and", dA, dB, prune_zeros=True).to_host()
    assert_bitexact(got, oracle.spgemm("or_and", A, B), "or_and with the flag")

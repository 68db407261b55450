"""Tall-skinny products C = A*B of Section 4's last experiment on the GPU
against the CPU oracle: A an R-MAT matrix with 8 nonzeros per column, B an
n x k Erdos-Renyi matrix with d2 nonzeros per column, n/k = 8192 (the paper's
aspect ratio), d2 = 1, 10, 100, ..., 10^5.  The product stands for one
level of a multi-source breadth-first search; its rows range from empty
(d2 = 1: B has k nonzeros in all) to a few hundred products each.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_within

pytestmark = pytest.mark.gpu
NT = 16


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


@pytest.mark.parametrize("d2", [1, 10, 100, 1000, 10000])
def test_tallskinny_scale16(d2):
    A = I.rmat_matrix(16, 8, seed=7, dtype="f64")
    n = A.n
    B = I.er_matrix(n, n // 8192, d2, seed=8 + d2, dtype="f64")
    h = H()
    got = h.spgemm("plus_times", h.DeviceCSR.from_host(A), h.DeviceCSR.from_host(B), validate=True).to_host()
    ref, bound = oracle.spgemm("plus_times", A, B, with_bound=True)
    assert_within(got, ref, bound, "f64", f"tall-skinny d2={d2}")


@pytest.mark.parametrize("d2", [1, 1000])
def test_tallskinny_wider_k(d2):
    """n/k = 256 instead of 8192: rows of up to 256 output columns."""
    A = I.rmat_matrix(15, 8, seed=9, dtype="f32")
    B = I.er_matrix(A.n, A.n // 256, d2, seed=10, dtype="f32")
    h = H()
    got = h.spgemm("plus_times", h.DeviceCSR.from_host(A), h.DeviceCSR.from_host(B)).to_host()
    ref, bound = oracle.spgemm("plus_times", A, B, with_bound=True)
    assert_within(got, ref, bound, "f32", f"wide tall-skinny d2={d2}")


@pytest.mark.parametrize("d2", [1, 100])
def test_tallskinny_scale18_idle_entries_dropped(d2):
    """A has 2M entries, almost all of them pointing at empty rows of B: the
    product runs on a copy of A without those entries.  Full comparison, in
    one call and in three row blocks delivered to host memory (blocks whose
    entries start in the middle of A's arrays)."""
    import torch
    A = I.rmat_matrix(18, 8, seed=5, dtype="f64")
    B = I.er_matrix(A.n, A.n // 8192, d2, seed=6, dtype="f64")
    h = H()
    dA, dB = h.DeviceCSR.from_host(A), h.DeviceCSR.from_host(B)
    ref, bound = oracle.spgemm("plus_times", A, B, with_bound=True)
    got = h.spgemm("plus_times", dA, dB).to_host()
    assert_within(got, ref, bound, "f64", f"d2={d2}")
    rp = torch.zeros(A.m + 1, dtype=torch.int64).pin_memory()
    col = torch.zeros(max(ref.nnz, 1), dtype=torch.int32).pin_memory()
    val = torch.zeros(max(ref.nnz, 1), dtype=torch.float64).pin_memory()
    nnz = h.spgemm_to_host("plus_times", dA, dB, rp, col, val, blocks=3)
    assert nnz == ref.nnz
    blk = I.CSR(A.m, B.n, rp.numpy().copy(), col.numpy()[:nnz].copy(), val.numpy()[:nnz].copy(), "f64")
    assert_within(blk, ref, bound, "f64", f"d2={d2}, three blocks")


@pytest.fixture(scope="module")
def rmat22():
    return I.rmat_matrix(22, 8, seed=2, dtype="f32")


@pytest.mark.parametrize("d2", [1, 100000])
def test_tallskinny_scale22_full_size_sampled(rmat22, d2):
    """n = 2^22, k = 512, f32, at full size: every row count against the oracle's
    symbolic pass, columns and values on the heaviest rows and a random sample."""
    h = H()
    A = rmat22
    B = I.er_matrix(A.n, A.n // 8192, d2, seed=3, dtype="f32")
    C = h.spgemm("plus_times", h.DeviceCSR.from_host(A), h.DeviceCSR.from_host(B))
    nnz_ref, rn = oracle.spgemm_count(A, B, nthreads=NT)
    rowptr = C.rowptr.cpu().numpy()
    assert int(rowptr[-1]) == nnz_ref
    np.testing.assert_array_equal(np.diff(rowptr), rn)
    _, rf = oracle.flops(A, B)
    rows = sorted(set(int(x) for x in np.concatenate([np.argsort(rf)[-8:], I.random_subset_sorted(A.m, 64, 11),
                                                      [0, A.m - 1]])))
    col, val = C.col.cpu().numpy(), C.val.cpu().numpy()
    for r in rows:
        a, b = int(rowptr[r]), int(rowptr[r + 1])
        R, bound = oracle.spgemm("plus_times", A, B, r0=r, r1=r + 1, with_bound=True)
        got = I.CSR(1, B.n, np.array([0, b - a], np.int64), col[a:b], val[a:b], "f32")
        assert_within(got, R, bound, "f32", f"row {r}")

"""GPU SpGEMM (hs_spgemm through the C ABI) against the CPU oracle.

Structure must match bit for bit; values bit for bit for the integer,
boolean and (min,+) semirings and the selectors, and for (+,x) within
|c - c_ref| <= tol * sum |a||b| per entry (tol 1e-12 for f64, 1e-5 for f32).
Cases span every accumulator bin (tiny, warp, mid, large, heavy with column
parts), the multi-chunk heavy symbolic pass (more than 2^20 columns), DCSR
input, empty operands, error paths, and R-MAT scale 20 at full size (all row
counts plus sampled rows, in the launch configuration the benchmark times).
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact, assert_within, rand_sparse, rows_of

pytestmark = pytest.mark.gpu

NT = os.cpu_count() or 1


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


def run_gpu(sr, A, B, dcsr=False, validate=True):
    h = H()
    dA = h.DeviceCSR.from_host(A, dcsr=dcsr)
    dB = h.DeviceCSR.from_host(B)
    return h.spgemm(sr, dA, dB, validate=validate).to_host()


def check(sr, A, B, dcsr=False, what=""):
    C = run_gpu(sr, A, B, dcsr)
    R, bound = oracle.spgemm(sr, A, B, with_bound=True, nthreads=NT)
    if sr == "plus_times" and A.dtype in ("f32", "f64"):
        assert_within(C, R, bound, A.dtype, what)
    else:
        assert_bitexact(C, R, what)
    return C


SR_TYPES = [("plus_times", "f64"), ("plus_times", "f32"), ("plus_times", "i64"),
            ("or_and", "bool"), ("min_plus", "f32"), ("min_plus", "i32")]


@pytest.mark.parametrize("sr,dt", SR_TYPES)
def test_tiny_random(sr, dt):
    seed = 1000
    for (m, k, n) in [(0, 5, 4), (4, 0, 5), (5, 4, 0), (1, 7, 1), (7, 1, 7), (1, 1, 1), (9, 13, 5),
                      (31, 17, 40), (64, 64, 64), (100, 80, 120)]:
        for dens in (0.0, 0.1, 0.5, 1.0):
            seed += 1
            A = rand_sparse(m, k, dens, seed, dt)
            B = rand_sparse(k, n, dens, seed + 77, dt)
            check(sr, A, B, what=f"{m}x{k}x{n} d={dens}")


def test_er_config_f64():
    """Erdos-Renyi n=4096, 8 nonzeros per column, f64, C = A*A over (+,x)."""
    A = I.er_matrix(4096, 4096, 8, seed=1, dtype="f64")
    check("plus_times", A, A, what="ER 4096")


@pytest.mark.parametrize("sr,dt", SR_TYPES)
def test_rmat_scale14_all_semirings(sr, dt):
    A = I.rmat_matrix(14, 8, seed=3, dtype=dt, kind="signed" if dt != "bool" else "unit")
    if sr == "min_plus" and dt == "i32":
        A = A.with_values("i32", 5)
    check(sr, A, A, what="rmat14")


@pytest.mark.parametrize("dt", ["f32", "f64", "bool"])
def test_rmat_scale16_heavy_rows(dt):
    """Rows beyond one shared-memory table (column parts) appear at scale 16."""
    A = I.rmat_matrix(16, 8, seed=4, dtype=dt)
    sr = "or_and" if dt == "bool" else "plus_times"
    _, rn = oracle.spgemm_count(A, A, nthreads=NT)
    assert rn.max() > 8192  # the heavy numeric bin is exercised
    check(sr, A, A, what="rmat16")


def test_wide_columns_multi_chunk():
    """More than 2^20 columns: the heavy symbolic bitmap runs several chunks."""
    n = 3 * (1 << 20) + 12345
    A = rand_sparse(64, 400, 0.8, 5, "f32")  # ~320 entries per row
    # B: 400 rows of (up to) 60 random distinct columns each in [0, n)
    rows = np.repeat(np.arange(400, dtype=np.int64), 60)
    keys = np.unique(rows * n + I.random_sequence(n, len(rows), 100).astype(np.int64))
    rowptr, cols = I.csr_from_unique_sorted_keys(keys, 400, n)
    B = I.CSR(400, n, rowptr, cols, I.random_values(len(cols), "f32", 7), "f32")
    f, rf = oracle.flops(A, B)
    assert rf.max() > 16384
    check("plus_times", A, B, what="wide")


def test_dcsr_left_operand():
    A = I.rmat_matrix(13, 8, seed=8, dtype="f64")
    assert (np.diff(A.rowptr) == 0).any()
    check("plus_times", A, A, dcsr=True, what="dcsr")


def test_selectors():
    A = I.er_matrix(500, 400, 5, seed=9, dtype="f64", kind="signed")
    rows = I.random_sequence(500, 300, 11)
    R = I.CSR(300, 500, np.arange(301, dtype=np.int64), rows, None, "bool")
    check("select2nd", R, A, what="R*A")
    cols = I.random_sequence(400, 250, 12)
    qrow = np.zeros(401, np.int64)
    order = np.argsort(cols, kind="stable")
    np.cumsum(np.bincount(cols, minlength=400), out=qrow[1:])
    Q = I.CSR(400, 250, qrow, order.astype(np.int32), None, "bool")
    check("select1st", A, Q, what="A*Q")
    A32 = A.with_values("i32", 3)
    check("select1st", A32, Q, what="A*Q i32")


def test_identity_and_permutation():
    A = I.rmat_matrix(12, 8, seed=13, dtype="f32", kind="signed")
    E = I.identity(A.n, "f32")
    C = run_gpu("plus_times", A, E)
    assert_bitexact(C, A, "A*I")
    p = I.random_permutation(A.m, seed=14)
    P = I.permutation_matrix(p, "f32")
    C = run_gpu("plus_times", P, A)
    R = oracle.spgemm("plus_times", P, A)
    assert_bitexact(C, R, "P*A")


def test_errors():
    h = H()
    A = I.er_matrix(50, 40, 3, seed=15, dtype="f64")
    dA = h.DeviceCSR.from_host(A)
    with pytest.raises(h.HsError) as e:
        h.spgemm("plus_times", dA, dA)  # 50x40 times 50x40
    assert e.value.code == -1
    B = I.er_matrix(40, 30, 3, seed=16, dtype="f32")
    with pytest.raises(h.HsError):
        h.spgemm("plus_times", dA, h.DeviceCSR.from_host(B))  # dtype mismatch
    bad = I.CSR(A.m, A.n, A.rowptr, A.col.copy(), A.val, "f64")
    r0 = int(np.nonzero(np.diff(A.rowptr) >= 2)[0][0])
    a = int(A.rowptr[r0])
    bad.col[a], bad.col[a + 1] = bad.col[a + 1], bad.col[a]
    B2 = I.er_matrix(40, 30, 3, seed=16, dtype="f64")
    with pytest.raises(h.HsError) as e:
        h.spgemm("plus_times", h.DeviceCSR.from_host(bad), h.DeviceCSR.from_host(B2), validate=True)
    assert e.value.code == -2


def test_rmat_scale20_full_size_sampled():
    """R-MAT scale 20, edge factor 8, (.57,.19,.19,.05), f32, C = A*A over (+,x), at full size:
    every row count against the oracle's symbolic pass, values and columns on sampled rows
    (the heaviest rows, a random sample, and the first and last rows)."""
    h = H()
    A = I.rmat_matrix(20, 8, seed=2, dtype="f32")
    dA = h.DeviceCSR.from_host(A)
    C = h.spgemm("plus_times", dA, dA, validate=True)
    nnz_ref, rn = oracle.spgemm_count(A, A, nthreads=NT)
    rowptr = C.rowptr.cpu().numpy()
    assert int(rowptr[-1]) == nnz_ref
    np.testing.assert_array_equal(np.diff(rowptr), rn)
    _, rf = oracle.flops(A, A)
    heavy = np.argsort(rf)[-8:]
    rnd = I.random_subset_sorted(A.m, 48, 17)
    rows = sorted(set(int(x) for x in np.concatenate([heavy, rnd, [0, A.m - 1]])))
    # copy the sampled rows back
    col_d, val_d = C.col, C.val
    parts_j, parts_v, counts = [], [], []
    for r in rows:
        a, b = int(rowptr[r]), int(rowptr[r + 1])
        parts_j.append(col_d[a:b].cpu().numpy())
        parts_v.append(val_d[a:b].cpu().numpy())
        counts.append(b - a)
    crp = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(counts, out=crp[1:])
    got = I.CSR(len(rows), A.n, crp, np.concatenate(parts_j), np.concatenate(parts_v), "f32")
    ref_parts, bnd_parts = [], []
    for r in rows:
        R, b = oracle.spgemm("plus_times", A, A, r0=r, r1=r + 1, with_bound=True)
        ref_parts.append(R)
        bnd_parts.append(b)
    ref = I.CSR(len(rows), A.n, crp, np.concatenate([p.col for p in ref_parts]),
                np.concatenate([p.val for p in ref_parts]), "f32")
    assert np.array_equal(np.concatenate([[0], np.cumsum([p.nnz for p in ref_parts])]), crp)
    assert_within(got, ref, np.concatenate(bnd_parts), "f32", "rmat20 sampled rows")

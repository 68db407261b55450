"""The expand-sort-compress tiers (rows of at most 1024 products sorted in one
warp's registers, Algorithm 1's row accumulation by sorting instead of
hashing) against the CPU oracle:

* every semiring and value type with every row of at most 1024 products
  forced through them (sort_pct 0), so runs of equal columns cross lanes,
  registers and 32-element rounds;
* Erdos-Renyi rows that barely compress, the rows the tiers are for, with
  32 < f <= 1024 (both register widths of both tiers);
* rows spanning more columns than a 32-bit packed key holds (the 64-bit key
  path of the small tier; the larger tier is kept out of such matrices);
* the tiers' numeric pass replayed from a plan.
Structure bit-exact; values bit-exact for the exact semirings, within
tol * sum |a||b| for (+,x) f32/f64."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact, assert_within

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1
SORT_PHASES = {"numeric_sort_xs", "numeric_sort_s", "numeric_sort_m", "numeric_sort"}  # 128, 256, 512, 1024 products

SR_TYPES = [("plus_times", "f64"), ("plus_times", "f32"), ("plus_times", "i64"),
            ("or_and", "bool"), ("min_plus", "f32"), ("min_plus", "i32")]


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


def product_with_phases(sr, A, B, tuning=None):
    h = H()
    dA = h.DeviceCSR.from_host(A)
    dB = h.DeviceCSR.from_host(B)
    h.set_tuning(None)
    if tuning:
        h.set_tuning(tuning)
    h.profile_enable(True)
    h.profile_reset()
    try:
        C = h.spgemm(sr, dA, dB, validate=True).to_host()
        phases = {k for k, (_, launches) in h.profile_read().items() if launches > 0}  # the phases that ran
    finally:
        h.profile_enable(False)
        h.set_tuning(None)
    return C, phases


def compare(sr, A, B, C, what, nthreads=NT):
    if sr == "plus_times" and A.dtype in ("f32", "f64"):
        R, bound = oracle.spgemm(sr, A, B, with_bound=True, nthreads=nthreads)
        assert_within(C, R, bound, A.dtype, what)
    else:
        R = oracle.spgemm(sr, A, B, nthreads=nthreads)
        assert_bitexact(C, R, what)


@pytest.mark.parametrize("sr,dt", SR_TYPES)
def test_every_small_row_sorted(sr, dt):
    A = I.rmat_matrix(14, 8, seed=11, dtype=dt, kind="signed" if dt != "bool" else "unit")
    if sr == "min_plus" and dt == "i32":
        A = A.with_values("i32", 5)
    f, rf = oracle.flops(A, A)
    for lo, hi in ((32, 128), (128, 256), (256, 512), (512, 1024)):
        assert ((rf > lo) & (rf <= hi)).any()
    C, ph = product_with_phases(sr, A, A, {"sort_pct": 0, "sort_max": 1024})
    assert SORT_PHASES <= ph, sorted(ph)
    compare(sr, A, A, C, f"rmat14 {sr} {dt} sorted")


@pytest.mark.parametrize("d,dt", [(5, "f64"), (9, "f32"), (14, "f64"), (20, "f32"), (28, "f64")])
def test_er_rows_that_barely_compress(d, dt):
    """ER n = 8192 with d per column: f ~ d^2 in (32, 1024], c/f close to 1."""
    A = I.er_matrix(8192, 8192, d, seed=20 + d, dtype=dt)
    B = I.er_matrix(8192, 8192, d, seed=40 + d, dtype=dt)
    C, ph = product_with_phases("plus_times", A, B)
    assert SORT_PHASES & ph, sorted(ph)
    compare("plus_times", A, B, C, f"ER d={d}")


@pytest.mark.parametrize("sr,dt", [("plus_times", "f64"), ("min_plus", "i32"), ("or_and", "bool")])
def test_rows_wider_than_a_packed_key(sr, dt):
    """2^25 + 2^20 columns: rows of 33..256 random columns span more than the
    32-bit key of their tier holds, so the small tier sorts 64-bit keys; the
    rows above 256 products stay in the hash tiers."""
    n = (1 << 25) + (1 << 20)
    k = 2048
    A = I.er_matrix(300, k, 1, seed=3, dtype=dt, kind="unit")  # about 7 entries per row
    per = (np.arange(k) % 40) + 1  # B rows of up to 1..40 entries, columns drawn with replacement
    rows = np.repeat(np.arange(k, dtype=np.int64), per)
    keys = np.unique(rows * n + I.random_sequence(n, len(rows), 500).astype(np.int64))
    rowptr, cols = I.csr_from_unique_sorted_keys(keys, k, n)
    B = I.CSR(k, n, rowptr, cols, None if dt == "bool" else I.random_values(len(cols), dt, 9), dt)
    if sr == "min_plus":
        A = A.with_values("i32", 5)
        B = B.with_values("i32", 6)
    f, rf = oracle.flops(A, B)
    assert ((rf > 32) & (rf <= 256)).sum() > 50 and (rf > 256).any()
    C, ph = product_with_phases(sr, A, B)
    assert (SORT_PHASES & ph) and (SORT_PHASES & ph) <= {"numeric_sort_xs", "numeric_sort_s"}, sorted(ph)
    compare(sr, A, B, C, f"wide {sr}", nthreads=1)


def test_sorted_rows_replay_from_a_plan():
    import torch
    h = H()
    A = I.er_matrix(8192, 8192, 12, seed=61, dtype="f64")
    dA = h.DeviceCSR.from_host(A)
    h.set_tuning(None)
    P = h.Plan("plus_times", dA, dA)
    try:
        ref = P.C.val.clone()
        P.C.val.zero_()
        P.execute()
        P.status()
        torch.cuda.synchronize()
        assert torch.equal(P.C.val, ref)
        R, bound = oracle.spgemm("plus_times", A, A, with_bound=True, nthreads=NT)
        assert_within(P.C.to_host(), R, bound, "f64", "plan replay")
    finally:
        P.close()

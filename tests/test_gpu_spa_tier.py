"""The dense-accumulator tier (Figure 1's sparse accumulator as it stands: a
value per column and an occupancy flag, one warp per row) serves, when the
tuning's spa_max allows, products whose B has at most 2048 columns (1024 for
8-byte values): every row of more than 32 products takes it.  Against the CPU oracle for every semiring and
value type, at the tier's column limits and just past them, with a DCSR left
operand, and a plan's numeric replay.  Structure
bit-exact; values bit-exact for the exact semirings, within tol * sum |a||b|
for (+,x) f32/f64."""
from __future__ import annotations

import os

import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact, assert_within

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1
SR_TYPES = [("plus_times", "f64"), ("plus_times", "f32"), ("plus_times", "i64"),
            ("or_and", "bool"), ("min_plus", "f32"), ("min_plus", "i32")]


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


def run(sr, A, B, dcsr=False):
    h = H()
    dA = h.DeviceCSR.from_host(A, dcsr=dcsr)
    dB = h.DeviceCSR.from_host(B)
    h.set_tuning({"spa_max": 2048})
    h.profile_enable(True)
    h.profile_reset()
    try:
        C = h.spgemm(sr, dA, dB, validate=True).to_host()
        ran = {k for k, (_, launches) in h.profile_read().items() if launches > 0}
    finally:
        h.profile_enable(False)
        h.set_tuning(None)
    return C, ran


def compare(sr, A, B, C, what):
    if sr == "plus_times" and A.dtype in ("f32", "f64"):
        R, bound = oracle.spgemm(sr, A, B, with_bound=True, nthreads=NT)
        assert_within(C, R, bound, A.dtype, what)
    else:
        assert_bitexact(C, oracle.spgemm(sr, A, B, nthreads=NT), what)


def operands(dt, n, d=256, seed=0):
    """A: R-MAT scale 13 (8192 rows); B: 8192 x n with d nonzeros per column
    (about n*d/8192 per row), so most rows of A*B have more than 32 products."""
    A = I.rmat_matrix(13, 8, seed=31 + seed, dtype=dt, kind="signed" if dt != "bool" else "unit")
    B = I.er_matrix(8192, n, d, seed=41 + seed, dtype=dt, kind="signed" if dt != "bool" else "unit")
    if dt == "i32":
        A, B = A.with_values("i32", 5), B.with_values("i32", 6)
    return A, B


@pytest.mark.parametrize("sr,dt", SR_TYPES)
def test_narrow_products_every_semiring(sr, dt):
    n = 1024 if dt in ("f64", "i64") else 2048  # the tier's limit for the value width
    A, B = operands(dt, n)
    f, rf = oracle.flops(A, B)
    assert (rf > 32).sum() > 1000
    C, ran = run(sr, A, B)
    assert {"symbolic_spa", "numeric_spa"} <= ran, sorted(ran)
    compare(sr, A, B, C, f"spa {sr} {dt} n={n}")


@pytest.mark.parametrize("dt,n,spa", [("f64", 1025, False), ("f32", 2049, False), ("bool", 2048, True),
                                      ("f32", 512, True), ("f64", 97, True)])
def test_column_limits(dt, n, spa):
    sr = "or_and" if dt == "bool" else "plus_times"
    A, B = operands(dt, n, d=max(8, 256 * 512 // max(n, 512)), seed=n)
    C, ran = run(sr, A, B)
    assert ("numeric_spa" in ran) == spa and ("symbolic_spa" in ran) == spa, sorted(ran)
    compare(sr, A, B, C, f"limit {dt} n={n}")


def test_dcsr_left_operand():
    A, B = operands("f64", 700, seed=3)
    C, ran = run("plus_times", A, B, dcsr=True)
    assert "numeric_spa" in ran
    compare("plus_times", A, B, C, "spa dcsr")


def test_plan_replay():
    import torch
    h = H()
    A, B = operands("f32", 1500, seed=5)
    dA, dB = h.DeviceCSR.from_host(A), h.DeviceCSR.from_host(B)
    h.set_tuning({"spa_max": 2048})
    try:
        P = h.Plan("plus_times", dA, dB)
    finally:
        h.set_tuning(None)
    try:
        ref = P.C.val.clone()
        P.C.val.zero_()
        P.execute()
        P.status()
        torch.cuda.synchronize()
        assert torch.equal(P.C.val, ref)
        R, bound = oracle.spgemm("plus_times", A, B, with_bound=True, nthreads=NT)
        assert_within(P.C.to_host(), R, bound, "f32", "spa plan replay")
    finally:
        P.close()

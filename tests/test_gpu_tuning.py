"""Row-bin thresholds (hs_set_tuning) change which kernel serves a row, never
the result: products under several settings (every optional tier off, tiers
moved, the bitmap kernel taking more rows) equal the default product and the
oracle.  The autotuner leaves a valid setting in place."""
from __future__ import annotations

import os

import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact, assert_within

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1

SETTINGS = [
    {"warp_s_max": 32, "mid_s_max": 0, "large_s_max": 2048, "sym_mid_s_max": 512, "sym_heavy_from": 0,
     "sort_max": 1024, "sort_pct": 0},
    {"warp_s_max": 64, "mid_s_max": 768, "large_s_max": 3072, "sym_mid_s_max": 768, "sym_heavy_from": 4096,
     "sort_max": 256, "sort_pct": 75, "heavy_part_kb": 32},
    {"warp_s_max": 128, "mid_s_max": 512, "large_s_max": 4096, "sym_mid_s_max": 1024, "sym_heavy_from": 6144,
     "sort_max": 1024, "sort_pct": 101, "num_heavy_from": 2048},
    {"sym_heavy_from": 4096, "num_heavy_from": 2048, "heavy_part_kb": 16},
    {"sym_heavy_from": 8192, "num_heavy_from": 8192},
    {"sym_heavy_from": 2048, "num_heavy_from": 2048},  # bitmap rows below 4096 products share the last heavy key
]


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


@pytest.mark.parametrize("sr,dt", [("plus_times", "f32"), ("or_and", "bool"), ("plus_times", "f64")])
def test_results_do_not_depend_on_thresholds(sr, dt):
    import torch
    h = H()
    A = I.rmat_matrix(15, 8, seed=3, dtype=dt)
    dA = h.DeviceCSR.from_host(A)
    h.set_tuning(None)
    ref = h.spgemm(sr, dA, dA)
    if sr == "plus_times":
        R, bound = oracle.spgemm(sr, A, A, with_bound=True, nthreads=NT)
    else:
        R = oracle.spgemm(sr, A, A, nthreads=NT)
    try:
        for t in SETTINGS:
            h.set_tuning(t)
            C = h.spgemm(sr, dA, dA, validate=True)
            assert torch.equal(C.rowptr, ref.rowptr) and torch.equal(C.col, ref.col), t
            Ch = C.to_host()
            if sr == "plus_times":
                assert_within(Ch, R, bound, dt, str(t))
            else:
                assert_bitexact(Ch, R, str(t))
    finally:
        h.set_tuning(None)


def test_autotuner_sets_a_valid_tuning():
    from paper_1109_3739_gb300 import tune
    h = H()
    A = I.rmat_matrix(14, 8, seed=4, dtype="f32")
    dA = h.DeviceCSR.from_host(A)
    try:
        best, log = tune.tune(lambda: h.spgemm("plus_times", dA, dA), trials=1)
        assert h.get_tuning() == best
        assert len(log) >= 1 + sum(len(v) - 1 for v in tune.CANDIDATES.values()) - 1
        R, bound = oracle.spgemm("plus_times", A, A, with_bound=True, nthreads=NT)
        assert_within(h.spgemm("plus_times", dA, dA).to_host(), R, bound, "f32", "tuned product")
    finally:
        h.set_tuning(None)


def test_out_of_range_thresholds_are_clamped():
    import torch
    h = H()
    A = I.rmat_matrix(13, 8, seed=5, dtype="f32")
    dA = h.DeviceCSR.from_host(A)
    h.set_tuning(None)
    ref = h.spgemm("plus_times", dA, dA)
    try:
        h.set_tuning({"warp_s_max": 100000, "mid_s_max": -5, "large_s_max": 1 << 30, "sym_mid_s_max": 0,
                      "sym_heavy_from": 1, "sort_max": 1 << 20, "sort_pct": -3})
        C = h.spgemm("plus_times", dA, dA, validate=True)
        assert torch.equal(C.rowptr, ref.rowptr) and torch.equal(C.col, ref.col)
        R, bound = oracle.spgemm("plus_times", A, A, with_bound=True, nthreads=NT)
        assert_within(C.to_host(), R, bound, "f32", "clamped thresholds")
    finally:
        h.set_tuning(None)


@pytest.mark.parametrize("dt", ["f32", "f64", "bool"])
def test_heavy_parts_of_32_kb(dt):
    """Heavy rows (R-MAT scale 16) cut into column parts of 32 KB of values:
    half the units of the 16 KB parts, the same result."""
    import torch
    h = H()
    A = I.rmat_matrix(16, 8, seed=4, dtype=dt)
    sr = "or_and" if dt == "bool" else "plus_times"
    dA = h.DeviceCSR.from_host(A)
    h.set_tuning(None)
    ref = h.spgemm(sr, dA, dA)
    try:
        h.set_tuning({"heavy_part_kb": 32})
        C = h.spgemm(sr, dA, dA, validate=True)
        assert torch.equal(C.rowptr, ref.rowptr) and torch.equal(C.col, ref.col)
        if sr == "plus_times":
            R, bound = oracle.spgemm(sr, A, A, with_bound=True, nthreads=NT)
            assert_within(C.to_host(), R, bound, dt, "32 KB parts")
        else:
            assert_bitexact(C.to_host(), oracle.spgemm(sr, A, A, nthreads=NT), "32 KB parts")
    finally:
        h.set_tuning(None)

"""hs_spgemm_noalloc, the SpGEMM entry point that allocates nothing, against
hs_spgemm (the allocating entry point), through the C ABI.

It is meant for callers that cannot allocate device memory while they run
(their memory is already handed to a pool of their own, or an allocation is
not allowed where they call from): they pass ready-made output arrays and the
library takes every temporary from one fixed device array.  Both entry points
must give the same matrix: structure identical, values bit for bit for the
exact semirings and within the (+,x) tolerance of the other parity tests for
floating point, on two calls in a row (the fixed array keeps the previous
call's contents, which must not leak into the next result).  This file is
collected last so that a failure here leaves every other test already run.
"""
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


CASES = [
    ("plus_times", "f32", lambda: I.rmat_matrix(14, 8, seed=91, dtype="f32")),
    ("plus_times", "f64", lambda: I.er_matrix(4096, 4096, 8, seed=1, dtype="f64")),
    ("plus_times", "i64", lambda: I.rmat_matrix(13, 8, seed=92, dtype="i64", kind="signed")),
    ("or_and", "bool", lambda: I.rmat_matrix(14, 8, seed=93, dtype="bool")),
    ("min_plus", "i32", lambda: I.rmat_matrix(12, 8, seed=94, dtype="i32")),
]


@pytest.mark.parametrize("sr,dt,make", CASES, ids=[f"{c[0]}-{c[1]}" for c in CASES])
def test_noalloc_matches_allocating_entry_point(sr, dt, make):
    import torch
    h = H()
    A = make()
    dA = h.DeviceCSR.from_host(A)
    ref = h.spgemm(sr, dA, dA)
    ref_host = ref.to_host()
    bound = None
    if dt in ("f32", "f64"):
        _, bound = oracle.spgemm(sr, A, A, with_bound=True)
    free_before = None
    for call in range(2):  # two calls in a row share the fixed scratch
        C = h.spgemm_noalloc(sr, dA, dA, capacity=ref.nnz)
        torch.cuda.synchronize()
        if call == 1:
            # the second call allocates nothing: device free memory is unchanged
            assert torch.cuda.mem_get_info()[0] == free_before
        got = C.to_host()
        if bound is not None:
            assert_within(got, ref_host, bound, dt, f"noalloc call {call}")
        else:
            assert_bitexact(got, ref_host, f"noalloc call {call}")
        del C, got
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]


def test_noalloc_capacity_and_scratch_limits():
    h = H()
    A = I.rmat_matrix(12, 8, seed=95, dtype="f32")
    dA = h.DeviceCSR.from_host(A)
    need = h.spgemm("plus_times", dA, dA).nnz
    with pytest.raises(h.HsError) as e:
        h.spgemm_noalloc("plus_times", dA, dA, capacity=need - 1)
    assert e.value.code == -10 and e.value.nnz_needed == need
    # 3M rows need more than the 32 MiB fixed scratch (16 bytes per row)
    m = 3 << 20
    rowptr = np.zeros(m + 1, np.int64)
    rowptr[1:] = 1
    big = I.CSR(m, 4, rowptr, np.zeros(1, np.int32), np.ones(1, np.float32), "f32")
    B = I.CSR(4, 4, np.array([0, 1, 1, 1, 1], np.int64), np.zeros(1, np.int32), np.ones(1, np.float32), "f32")
    with pytest.raises(h.HsError) as e:
        h.spgemm_noalloc("plus_times", h.DeviceCSR.from_host(big), h.DeviceCSR.from_host(B), capacity=16)
    assert e.value.code == -9

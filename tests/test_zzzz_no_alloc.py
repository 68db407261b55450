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
    # scale 16: rows with more products than the large tier, so the entry
    # point's own heavy path (part bitmaps built from the products, segment
    # ends found by search) runs
    ("plus_times", "f32", lambda: I.rmat_matrix(16, 8, seed=96, dtype="f32")),
    ("plus_times", "f64", lambda: I.er_matrix(4096, 4096, 8, seed=1, dtype="f64")),
    ("plus_times", "i64", lambda: I.rmat_matrix(13, 8, seed=92, dtype="i64", kind="signed")),
    ("or_and", "bool", lambda: I.rmat_matrix(14, 8, seed=93, dtype="bool")),
    ("min_plus", "i32", lambda: I.rmat_matrix(12, 8, seed=94, dtype="i32")),
]


def _raw_noalloc(h, sr, dA, capacity, out_dt):
    """Output arrays allocated beforehand and a function making one bare call
    of the C entry point into them: (rowptr, col, val, A's descriptor, C's
    descriptor, call)."""
    import ctypes
    import torch
    L = h.library()
    tdt = {"f64": torch.float64, "f32": torch.float32, "i32": torch.int32, "i64": torch.int64}.get(out_dt)
    rowptr = torch.empty(dA.m + 1, dtype=torch.int64, device=dA.rowptr.device)
    col = torch.empty(max(capacity, 1), dtype=torch.int32, device=dA.rowptr.device)
    val = None if tdt is None else torch.empty(max(capacity, 1), dtype=tdt, device=dA.rowptr.device)
    a = dA.desc()
    c = h.hs_mat(0, 0, 0, 0, 0, 0, rowptr.data_ptr(), col.data_ptr(), None,
                 None if val is None else val.data_ptr())
    return (rowptr, col, val, a, c,
            lambda: L.hs_spgemm_noalloc(h.SEMIRING[sr], ctypes.byref(a), ctypes.byref(a), ctypes.byref(c),
                                        int(capacity), None))


@pytest.mark.parametrize("sr,dt,make", CASES, ids=[f"{c[0]}-{c[1]}-{i}" for i, c in enumerate(CASES)])
def test_noalloc_matches_allocating_entry_point(sr, dt, make):
    import torch
    h = H()
    A = make()
    dA = h.DeviceCSR.from_host(A)
    ref = h.spgemm(sr, dA, dA)
    ref_host = ref.to_host()
    nnz = ref.nnz
    del ref
    R, bound = oracle.spgemm(sr, A, A, with_bound=True)
    out_dt = "bool" if sr == "or_and" else dt
    rowptr, col, val, a, c, call_abi = _raw_noalloc(h, sr, dA, nnz, out_dt)
    for call in range(2):  # two calls in a row share the fixed scratch
        # hand back what the library's pool and torch's cache keep, so that
        # any allocation inside the call would show as less free memory
        h.trim_memory()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free0 = torch.cuda.mem_get_info()[0]
        st = call_abi()
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert st == 0, h.HsError(st, "hs_spgemm_noalloc")
        if call == 1:  # the first call may load kernel modules lazily
            assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
        got = h.DeviceCSR(c.m, c.n, rowptr, col[:c.nnz], None if val is None else val[:c.nnz],
                          h.DTYPE_NAME[c.dtype]).to_host()
        # against the allocating entry point: same structure, and the oracle
        # decides the values (bit for bit for the exact semirings)
        assert np.array_equal(got.rowptr, ref_host.rowptr) and np.array_equal(got.col, ref_host.col)
        if dt in ("f32", "f64"):
            assert_within(got, R, bound, dt, f"noalloc call {call}")
            assert_within(ref_host, R, bound, dt, "hs_spgemm")
        else:
            assert_bitexact(got, R, f"noalloc call {call}")
        # a stale value from the previous call must not survive: scribble
        # over the outputs before the second call
        col.fill_(-1)
        if val is not None:
            val.fill_(0)
        rowptr.fill_(-1)


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

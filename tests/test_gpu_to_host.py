"""hs_spgemm_to_host: C delivered to host memory block by block (each row
block's copy overlapped with the next block's product) equals hs_spgemm's C
and the oracle's; too small arrays give HS_ECAPACITY with the size needed."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact, assert_within

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


def host_out(m, cap, dtype):
    import torch
    tdt = {"f64": torch.float64, "f32": torch.float32, "i32": torch.int32, "i64": torch.int64}.get(dtype)
    rp = torch.empty(m + 1, dtype=torch.int64, pin_memory=True)
    col = torch.empty(cap, dtype=torch.int32, pin_memory=True)
    val = None if tdt is None else torch.empty(cap, dtype=tdt, pin_memory=True)
    return rp, col, val


@pytest.mark.parametrize("sr,dt,blocks", [("plus_times", "f32", 1), ("plus_times", "f32", 8),
                                          ("or_and", "bool", 3), ("plus_times", "f64", 5), ("min_plus", "i32", 4)])
def test_to_host_equals_device_product(sr, dt, blocks):
    h = H()
    A = I.rmat_matrix(14, 8, seed=7, dtype=dt) if dt in ("f32", "bool") else I.er_matrix(2000, 2000, 10, seed=8, dtype=dt)
    dA = h.DeviceCSR.from_host(A)
    ref = h.spgemm(sr, dA, dA)
    rp, col, val = host_out(A.m, ref.nnz, ref.dtype)
    nnz = h.spgemm_to_host(sr, dA, dA, rp, col, val, blocks=blocks)
    assert nnz == ref.nnz
    assert np.array_equal(rp.numpy(), ref.rowptr.cpu().numpy())
    assert np.array_equal(col.numpy(), ref.col.cpu().numpy())
    C = I.CSR(A.m, A.n, rp.numpy(), col.numpy(), None if val is None else val.numpy(), ref.dtype)
    if sr == "plus_times" and dt in ("f32", "f64"):
        R, bound = oracle.spgemm(sr, A, A, with_bound=True, nthreads=NT)
        assert_within(C, R, bound, dt, "to_host")
    else:
        assert_bitexact(C, oracle.spgemm(sr, A, A, nthreads=NT), "to_host")


def test_to_host_reports_capacity_needed():
    h = H()
    A = I.rmat_matrix(12, 8, seed=9, dtype="f32")
    dA = h.DeviceCSR.from_host(A)
    need = h.spgemm("plus_times", dA, dA).nnz
    rp, col, val = host_out(A.m, need // 2, "f32")
    with pytest.raises(h.HsError) as ei:
        h.spgemm_to_host("plus_times", dA, dA, rp, col, val, blocks=4)
    assert ei.value.code == -10 and ei.value.nnz_needed == need


def test_to_host_rejects_dcsr_and_handles_empty():
    h = H()
    A = I.rmat_matrix(10, 8, seed=11, dtype="f32")
    dA = h.DeviceCSR.from_host(A, dcsr=True)
    dB = h.DeviceCSR.from_host(A)
    rp, col, val = host_out(A.m, 10, "f32")
    with pytest.raises(h.HsError) as ei:
        h.spgemm_to_host("plus_times", dA, dB, rp, col, val)
    assert ei.value.code == -1
    Z = I.CSR(0, A.n, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32), "f32")
    dZ = h.DeviceCSR.from_host(Z)
    rp0, col0, val0 = host_out(0, 0, "f32")
    assert h.spgemm_to_host("plus_times", dZ, dB, rp0, col0, val0, blocks=3) == 0
    assert int(rp0[0]) == 0


def test_direct_and_copied_paths_agree():
    """Page-locked arrays with one block take the direct path (kernels store
    into host memory); pageable arrays take the copy path; same C."""
    import torch
    h = H()
    A = I.rmat_matrix(13, 8, seed=12, dtype="f32")
    dA = h.DeviceCSR.from_host(A)
    ref = h.spgemm("plus_times", dA, dA)
    outs = []
    for pinned, stage in ((True, False), (False, False), (True, True)):
        rp = torch.empty(A.m + 1, dtype=torch.int64, pin_memory=pinned)
        col = torch.empty(ref.nnz, dtype=torch.int32, pin_memory=pinned)
        val = torch.empty(ref.nnz, dtype=torch.float32, pin_memory=pinned)
        assert h.spgemm_to_host("plus_times", dA, dA, rp, col, val, blocks=1, stage_on_device=stage) == ref.nnz
        outs.append((rp.numpy().copy(), col.numpy().copy(), val.numpy().copy()))
    for rp, col, _ in outs:
        assert np.array_equal(rp, ref.rowptr.cpu().numpy())
        assert np.array_equal(col, ref.col.cpu().numpy())
    R, bound = oracle.spgemm("plus_times", A, A, with_bound=True, nthreads=NT)
    for rp, col, val in outs:
        assert_within(I.CSR(A.m, A.n, rp, col, val, "f32"), R, bound, "f32", "to_host")
    # the direct path reports a short capacity too
    rp, col, val = host_out(A.m, ref.nnz - 1, "f32")
    with pytest.raises(h.HsError) as ei:
        h.spgemm_to_host("plus_times", dA, dA, rp, col, val, blocks=1)
    assert ei.value.code == -10 and ei.value.nnz_needed == ref.nnz

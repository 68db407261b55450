"""Symbolic once, numeric many times: hs_plan_create / hs_plan_execute against
the CPU oracle, including replay from a captured CUDA graph.

A plan's first product must equal hs_spgemm's; every execute with new values
of A and B (same structures) must equal the oracle's product of the new
matrices: structure bit-exact, values bit-exact for the exact semirings and
within the (+,x) tolerance otherwise.  Inputs cover every numeric bin (R-MAT
scale 16 has heavy rows) and a stacked batch.
"""
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


def revalue(A, seed, kind="signed"):
    """A with the same structure and new seeded values."""
    return I.CSR(A.m, A.n, A.rowptr, A.col, I.random_values(A.nnz, A.dtype, seed, stream=11, kind=kind), A.dtype)


def check(sr, C_host, A, B, what):
    if sr == "plus_times" and A.dtype in ("f32", "f64"):
        R, bound = oracle.spgemm(sr, A, B, with_bound=True, nthreads=NT)
        assert_within(C_host, R, bound, A.dtype, what)
    else:
        assert_bitexact(C_host, oracle.spgemm(sr, A, B, nthreads=NT), what)


def to_dev(x, like):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(like.device)


@pytest.mark.parametrize("sr,dt,gen", [
    ("plus_times", "f64", "er"), ("plus_times", "f32", "rmat"), ("min_plus", "f32", "rmat"),
    ("plus_times", "i64", "er"), ("min_plus", "i32", "er"),
])
def test_plan_matches_spgemm_then_new_values(sr, dt, gen):
    import torch
    h = H()
    if gen == "er":
        A = I.er_matrix(3000, 3000, 12, seed=3, dtype=dt)
        B = I.er_matrix(3000, 3000, 12, seed=4, dtype=dt)
    else:
        A = I.rmat_matrix(16, 8, seed=5, dtype=dt)
        B = A
    dA, dB = h.DeviceCSR.from_host(A), h.DeviceCSR.from_host(B)
    plan = h.Plan(sr, dA, dB, validate=True)
    ref = h.spgemm(sr, dA, dB)
    assert torch.equal(plan.C.rowptr, ref.rowptr) and torch.equal(plan.C.col, ref.col)
    check(sr, plan.C.to_host(), A, B, "plan's first product")
    for seed in (21, 22):
        A2 = revalue(A, seed)
        B2 = A2 if B is A else revalue(B, seed + 100)
        av, bv = to_dev(A2.val, dA.val), to_dev(B2.val, dB.val)
        cv = torch.empty_like(plan.C.val)
        plan.execute(av, bv, cv)
        plan.status()
        Cn = h.DeviceCSR(plan.C.m, plan.C.n, plan.C.rowptr, plan.C.col, cv, plan.C.dtype)
        check(sr, Cn.to_host(), A2, B2, f"execute with values {seed}")
    plan.close()


def test_plan_structure_only_and_selectors():
    h = H()
    A = I.rmat_matrix(14, 8, seed=6, dtype="bool")
    dA = h.DeviceCSR.from_host(A)
    plan = h.Plan("or_and", dA, dA)
    plan.execute()
    plan.status()
    assert_bitexact(plan.C.to_host(), oracle.spgemm("or_and", A, A, nthreads=NT), "or_and plan")
    plan.close()
    # select2nd: C takes B's values
    Af = I.er_matrix(500, 400, 5, seed=7, dtype="f32")
    Bf = I.er_matrix(400, 300, 1, seed=8, dtype="f64")
    dAf, dBf = h.DeviceCSR.from_host(Af), h.DeviceCSR.from_host(Bf)
    p2 = h.Plan("select2nd", dAf, dBf)
    B2 = revalue(Bf, 9)
    import torch
    cv = torch.empty_like(p2.C.val)
    p2.execute(None, to_dev(B2.val, dBf.val), cv)
    p2.status()
    Cn = h.DeviceCSR(p2.C.m, p2.C.n, p2.C.rowptr, p2.C.col, cv, p2.C.dtype)
    assert_bitexact(Cn.to_host(), oracle.spgemm("select2nd", Af, B2, nthreads=NT), "select2nd execute")
    p2.close()


def test_plan_replayed_from_a_cuda_graph():
    import torch
    h = H()
    A = I.rmat_matrix(16, 8, seed=10, dtype="f32")
    dA = h.DeviceCSR.from_host(A)
    plan = h.Plan("plus_times", dA, dA)
    av = dA.val.clone()
    cv = torch.empty_like(plan.C.val)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.execute(av, av, cv)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.execute(av, av, cv)
    for seed in (31, 32):
        A2 = revalue(A, seed)
        av.copy_(to_dev(A2.val, av))
        g.replay()
        torch.cuda.synchronize()
        plan.status()
        Cn = h.DeviceCSR(plan.C.m, plan.C.n, plan.C.rowptr, plan.C.col, cv, "f32")
        check("plus_times", Cn.to_host(), A2, A2, f"graph replay with values {seed}")
    plan.close()


def test_stacked_batch_plan_matches_batched_call():
    import torch
    h = H()
    probs = I.batched_er(60, seed=12, dtype="f64", nmax=4096)
    As = [h.DeviceCSR.from_host(a) for a, _ in probs]
    Bs = [h.DeviceCSR.from_host(b) for _, b in probs]
    SA, SB, offs = h.batch_stack(As, Bs)
    C1, offs1 = h.spgemm_batched("plus_times", As, Bs)
    assert np.array_equal(offs, offs1)
    plan = h.Plan("plus_times", SA, SB)
    assert torch.equal(plan.C.rowptr, C1.rowptr) and torch.equal(plan.C.col, C1.col)
    # new values for every problem, restacked through the same call
    probs2 = [(revalue(a, 40 + i), revalue(b, 140 + i)) for i, (a, b) in enumerate(probs)]
    As2 = [h.DeviceCSR.from_host(a) for a, _ in probs2]
    Bs2 = [h.DeviceCSR.from_host(b) for _, b in probs2]
    SA2, SB2, _ = h.batch_stack(As2, Bs2)
    cv = torch.empty_like(plan.C.val)
    plan.execute(SA2.val, SB2.val, cv)
    plan.status()
    Cn = h.DeviceCSR(plan.C.m, plan.C.n, plan.C.rowptr, plan.C.col, cv, "f64")
    for i in (0, 7, 33, 59):
        A2, B2 = probs2[i]
        Ci = h.csr_rows(Cn, int(offs[i]), int(offs[i + 1]), n=B2.n).to_host()
        check("plus_times", Ci, A2, B2, f"problem {i}")
    plan.close()


def test_plan_edge_cases():
    import torch
    h = H()
    # B without entries: C has no entries; executes are no-ops
    A = I.er_matrix(300, 200, 4, seed=13, dtype="f64")
    Bz = I.CSR(200, 150, np.zeros(201, np.int64), np.zeros(0, np.int32), np.zeros(0), "f64")
    p = h.Plan("plus_times", h.DeviceCSR.from_host(A), h.DeviceCSR.from_host(Bz))
    assert p.C.nnz == 0 and int(p.C.rowptr[-1]) == 0
    p.execute()
    p.status()
    p.close()
    # DCSR left operand (only non-empty rows stored)
    A2 = I.rmat_matrix(13, 8, seed=14, dtype="f32")
    dA2 = h.DeviceCSR.from_host(A2, dcsr=True)
    dB2 = h.DeviceCSR.from_host(A2)
    p2 = h.Plan("plus_times", dA2, dB2)
    A3 = revalue(A2, 15)
    cv = torch.empty_like(p2.C.val)
    p2.execute(to_dev(A3.val, dA2.val), to_dev(A3.val, dB2.val), cv)
    p2.status()
    Cn = h.DeviceCSR(p2.C.m, p2.C.n, p2.C.rowptr, p2.C.col, cv, "f32")
    check("plus_times", Cn.to_host(), A3, A3, "DCSR plan execute")
    p2.close()


def test_single_problem_batch_stack():
    h = H()
    import torch
    A = I.er_matrix(10, 10, 2, seed=16)
    dA = h.DeviceCSR.from_host(A)
    SA, SB, offs = h.batch_stack([dA], [dA])
    assert SA.m == 10 and SB.m == 10 and list(offs) == [0, 10]
    assert torch.equal(SA.col.cpu(), dA.col.cpu())  # one problem: columns shifted by 0

"""hs_spgemm_batched against the CPU oracle, problem by problem.

Small batches are compared in full for several semirings; the full batch of
2000 Erdos-Renyi problems (n_i log-uniform in [256, 65536], 2..32 nonzeros per
column, f64 (+,x)) is compared on sampled problems (the largest and a random
sample), in the configuration the benchmark times.
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


def check_problem(sr, C, offs, i, A, B):
    h = H()
    Ci = h.csr_rows(C, int(offs[i]), int(offs[i + 1]), n=B.n).to_host()
    if sr == "plus_times" and A.dtype in ("f32", "f64"):
        R, bound = oracle.spgemm(sr, A, B, with_bound=True, nthreads=NT)
        assert_within(Ci, R, bound, A.dtype, f"problem {i}")
    else:
        assert_bitexact(Ci, oracle.spgemm(sr, A, B, nthreads=NT), f"problem {i}")


@pytest.mark.parametrize("sr,dt", [("plus_times", "f64"), ("plus_times", "f32"), ("or_and", "bool"),
                                   ("plus_times", "i64"), ("min_plus", "i32")])
def test_small_batch_every_problem(sr, dt):
    h = H()
    probs = I.batched_er(40, seed=7, dtype=dt, nmax=2048)
    As = [h.DeviceCSR.from_host(a) for a, _ in probs]
    Bs = [h.DeviceCSR.from_host(b) for _, b in probs]
    C, offs = h.spgemm_batched(sr, As, Bs, validate=True)
    assert len(offs) == 41 and offs[-1] == sum(a.m for a, _ in probs)
    for i, (A, B) in enumerate(probs):
        check_problem(sr, C, offs, i, A, B)


def test_batch_with_empty_and_rectangular_problems():
    h = H()
    probs = [
        (I.er_matrix(30, 20, 3, seed=1), I.er_matrix(20, 50, 4, seed=2)),
        (I.CSR(5, 7, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0), "f64"),
         I.er_matrix(7, 9, 2, seed=3)),
        (I.er_matrix(11, 13, 2, seed=4), I.CSR(13, 3, np.zeros(14, np.int64), np.zeros(0, np.int32),
                                               np.zeros(0), "f64")),
        (I.er_matrix(64, 64, 8, seed=5), I.er_matrix(64, 64, 8, seed=6)),
    ]
    As = [h.DeviceCSR.from_host(a) for a, _ in probs]
    Bs = [h.DeviceCSR.from_host(b) for _, b in probs]
    C, offs = h.spgemm_batched("plus_times", As, Bs, validate=True)
    for i, (A, B) in enumerate(probs):
        check_problem("plus_times", C, offs, i, A, B)
    C0, offs0 = h.spgemm_batched("plus_times", [], [])
    assert C0.m == 0 and list(offs0) == [0]


def test_full_batch_sampled():
    """2000 problems at full size; the largest and 12 random problems against the oracle."""
    h = H()
    probs = I.batched_er(2000, seed=4, dtype="f64", workers=min(16, NT))
    As = [h.DeviceCSR.from_host(a) for a, _ in probs]
    Bs = [h.DeviceCSR.from_host(b) for _, b in probs]
    C, offs = h.spgemm_batched("plus_times", As, Bs)
    sizes = np.array([a.m for a, _ in probs])
    pick = set(I.random_subset_sorted(2000, 12, 19).tolist()) | {int(np.argmax(sizes))}
    for i in sorted(pick):
        A, B = probs[i]
        check_problem("plus_times", C, offs, i, A, B)
    # every problem's row count matches the oracle's symbolic pass on a sample of rows
    rp = C.rowptr.cpu().numpy()
    for i in sorted(pick):
        A, B = probs[i]
        _, rn = oracle.spgemm_count(A, B, nthreads=NT)
        np.testing.assert_array_equal(np.diff(rp[offs[i]:offs[i + 1] + 1]), rn)


# ---- one persistent launch per execution (hs_batch_plan_*)
@pytest.mark.parametrize("sr,dt", [("plus_times", "f64"), ("plus_times", "f32"), ("or_and", "bool"),
                                   ("plus_times", "i64"), ("min_plus", "i32"), ("min_plus", "f32")])
def test_persistent_plan_every_problem(sr, dt):
    h = H()
    probs = I.batched_er(40, seed=7, dtype=dt, nmax=2048)
    As = [h.DeviceCSR.from_host(a) for a, _ in probs]
    Bs = [h.DeviceCSR.from_host(b) for _, b in probs]
    plan = h.BatchPlan(sr, As, Bs)
    try:
        plan.execute()
        C, offs = plan.result()
        assert len(offs) == 41 and offs[-1] == sum(a.m for a, _ in probs)
        for i, (A, B) in enumerate(probs):
            check_problem(sr, C, offs, i, A, B)
    finally:
        plan.close()


def test_persistent_plan_graph_replay_mixed_rows():
    """Rows of every tier (warp rows, CTA rows, a CTA row of more than 2048
    outputs done column range by column range), empty and rectangular
    problems; the execution captured in a CUDA graph and replayed twice."""
    import torch
    h = H()
    probs = [
        (I.er_matrix(16, 200, 4, seed=21), I.er_matrix(200, 12000, 1, seed=22)),  # f = 3000, c > 2048
        (I.er_matrix(3000, 3000, 12, seed=23), I.er_matrix(3000, 3000, 12, seed=24)),
        (I.er_matrix(500, 700, 2, seed=25), I.er_matrix(700, 40, 3, seed=26)),
        (I.CSR(5, 7, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0), "f64"),
         I.er_matrix(7, 9, 2, seed=27)),
        (I.er_matrix(64, 64, 8, seed=28), I.er_matrix(64, 64, 8, seed=29)),
        (I.er_matrix(2000, 2000, 26, seed=30), I.er_matrix(2000, 2000, 26, seed=31)),  # warp rows of 257..1024
    ]
    f0 = np.diff(probs[0][1].rowptr)[probs[0][0].col].sum() / probs[0][0].m
    assert 2048 < f0 <= 4096
    As = [h.DeviceCSR.from_host(a) for a, _ in probs]
    Bs = [h.DeviceCSR.from_host(b) for _, b in probs]
    plan = h.BatchPlan("plus_times", As, Bs)
    try:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            plan.execute()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        l0 = h.launch_count()
        with torch.cuda.graph(g):
            plan.execute()
        assert h.launch_count() - l0 == 1  # one kernel per execution (besides one memset)
        first = None
        for rep in range(2):
            g.replay()
            torch.cuda.synchronize()
            C, offs = plan.result()
            ph = plan.phase_ms()
            assert ph["kernel"] > 0 and all(v >= 0 for v in ph.values())
            assert sum(ph[k] for k in ("products", "symbolic", "offsets", "values")) <= ph["kernel"] * 1.001
            for i, (A, B) in enumerate(probs):
                check_problem("plus_times", C, offs, i, A, B)
            host = (C.rowptr.cpu().clone(), C.col.cpu().clone(), C.val.cpu().clone())
            if first is None:
                first = host
            else:  # replays are deterministic in structure; values agree within the oracle's tolerance above
                assert torch.equal(first[0], host[0]) and torch.equal(first[1], host[1])
    finally:
        plan.close()


def test_persistent_plan_problem_wider_than_a_packed_key():
    """A problem of 2^25 + 2^20 columns beside a narrow one: warp rows (at most
    256 products once a problem is that wide) sort 64-bit keys, longer rows
    take the CTA tier."""
    h = H()
    n, k = (1 << 25) + (1 << 20), 2048
    A0 = I.er_matrix(300, k, 1, seed=41)
    per = (np.arange(k) % 40) + 1
    rows = np.repeat(np.arange(k, dtype=np.int64), per)
    keys = np.unique(rows * n + I.random_sequence(n, len(rows), 42).astype(np.int64))
    rowptr, cols = I.csr_from_unique_sorted_keys(keys, k, n)
    B0 = I.CSR(k, n, rowptr, cols, I.random_values(len(cols), "f64", 43), "f64")
    probs = [(A0, B0), (I.er_matrix(1000, 1000, 20, seed=44), I.er_matrix(1000, 1000, 20, seed=45))]
    f0 = np.diff(B0.rowptr)[A0.col]
    rf = np.bincount(np.repeat(np.arange(A0.m), np.diff(A0.rowptr)), weights=f0, minlength=A0.m)
    assert (rf > 256).any() and ((rf > 32) & (rf <= 256)).sum() > 50
    As = [h.DeviceCSR.from_host(a) for a, _ in probs]
    Bs = [h.DeviceCSR.from_host(b) for _, b in probs]
    plan = h.BatchPlan("plus_times", As, Bs)
    try:
        plan.execute()
        C, offs = plan.result()
        for i, (A, B) in enumerate(probs):
            check_problem("plus_times", C, offs, i, A, B)
    finally:
        plan.close()


def test_persistent_plan_rejects_rows_beyond_its_tables():
    h = H()
    A = I.er_matrix(4, 100, 4, seed=31)       # rows of 100 entries
    B = I.er_matrix(100, 10000, 5, seed=32)   # rows of 500 entries: 50000 products per row of A
    with pytest.raises(h.HsError) as e:
        h.BatchPlan("plus_times", [h.DeviceCSR.from_host(A)], [h.DeviceCSR.from_host(B)])
    assert e.value.code == -7

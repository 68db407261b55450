"""Full-size parity: the benchmark's configurations against the oracle,
every row and every problem, through the C ABI.

- C = A*A on the R-MAT scale-20 graph (edge factor 8, a=.57 b=c=.19 d=.05,
  f32 values) over (+,x) f32, (or,and) and (min,+) f32: all 2^20 rows,
  compared in row blocks (the oracle computes rows r0..r1 with every host
  core; each block is compared on the device, so C never leaves it).
- The 2000 batched Erdos-Renyi products (n_i log-uniform in [256, 65536],
  2..32 nonzeros per column, f64): every problem, by the stacked product and
  by the persistent launch.
- On the serving graph (R-MAT scale 22, edge factor 16, int32 weights): an
  induced subgraph A(I, I) with |I| = 2^16, the contraction S*A*S^T with n/64
  random clusters (int64) and a batch update A(I, J) = B of 2^16 random
  edges.

Structure must be identical everywhere; values bit for bit for the exact
semirings, SpRef, SpAsgn and the contraction, and within 1e-5 * sum |a||b|
(f32) or 1e-12 * sum |a||b| (f64) per entry for (+,x).  This file is collected
after the other parity tests.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import TOL

pytestmark = pytest.mark.gpu
NT = os.cpu_count() or 1


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


def _dev(x, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device)


def compare_on_device(got, R, bound, what):
    """got: a DeviceCSR; R (+ bound): the oracle's CSR of the same rows."""
    import torch
    dev = got.rowptr.device
    assert got.m == R.m, what
    rp = got.rowptr - got.rowptr[0]
    assert torch.equal(rp, _dev(R.rowptr, dev)), f"{what}: row offsets"
    assert torch.equal(got.col, _dev(R.col, dev)), f"{what}: column ids"
    if R.val is None:
        return
    ref = _dev(R.val, dev)
    if bound is None:  # exact: equal bits (+0 and -0 alike)
        a, b = got.val, ref
        same = (a == b) | ((a == 0) & (b == 0)) if a.dtype.is_floating_point else (a == b)
        bad = int((~same).sum())
        assert bad == 0, f"{what}: {bad} values differ"
    else:
        tol = TOL["f32" if got.val.dtype == torch.float32 else "f64"]
        err = (got.val.double() - ref.double()).abs()
        lim = tol * _dev(bound, dev)
        bad = int((err > lim).sum())
        assert bad == 0, f"{what}: {bad} values outside tolerance, worst ratio {float((err / lim.clamp_min(1e-300)).max()):.3g}"


@pytest.fixture(scope="module")
def rmat20():
    h = H()
    A = I.rmat_matrix(20, 8, 0.57, 0.19, 0.19, seed=2, dtype="f32")
    return A, h.DeviceCSR.from_host(A)


@pytest.mark.parametrize("sr", ["plus_times", "or_and", "min_plus"])
def test_rmat20_every_row(rmat20, sr):
    import torch
    h = H()
    A, dA = rmat20
    if sr == "or_and":
        A = I.CSR(A.m, A.n, A.rowptr, A.col, None, "bool")
        dA = h.DeviceCSR(dA.m, dA.n, dA.rowptr, dA.col, None, "bool")
    C = h.spgemm(sr, dA, dA)
    blocks = 16
    for b in range(blocks):
        r0, r1 = A.m * b // blocks, A.m * (b + 1) // blocks
        if sr == "plus_times":
            R, bound = oracle.spgemm(sr, A, A, r0, r1, nthreads=NT, with_bound=True)
        else:
            R, bound = oracle.spgemm(sr, A, A, r0, r1, nthreads=NT), None
        compare_on_device(h.csr_rows(C, r0, r1), R, bound, f"{sr} rows {r0}..{r1}")
        del R, bound
    nnz = C.nnz
    del C
    torch.cuda.empty_cache()
    assert nnz == 3578087023  # the benchmark workload's nnz(C)


def test_batched_every_problem():
    """Both batched forms, every problem: the stacked product (hs_spgemm_batched)
    and the persistent launch (hs_batch_plan_execute)."""
    import torch
    h = H()
    probs = I.batched_er(2000, seed=4, dtype="f64", workers=min(16, NT))
    As = [h.DeviceCSR.from_host(a) for a, _ in probs]
    Bs = [h.DeviceCSR.from_host(b) for _, b in probs]
    C, offs = h.spgemm_batched("plus_times", As, Bs)
    plan = h.BatchPlan("plus_times", As, Bs)
    plan.execute()
    P, poffs = plan.result()
    assert np.array_equal(offs, poffs)
    del As, Bs
    for i, (a, b) in enumerate(probs):
        R, bound = oracle.spgemm("plus_times", a, b, nthreads=NT, with_bound=True)
        compare_on_device(h.csr_rows(C, int(offs[i]), int(offs[i + 1]), n=b.n), R, bound, f"problem {i}")
        compare_on_device(h.csr_rows(P, int(offs[i]), int(offs[i + 1]), n=b.n), R, bound, f"persistent problem {i}")
    plan.close()
    del C, P
    torch.cuda.empty_cache()


def test_serving_graph_operations():
    import torch
    from paper_1109_3739_gb300 import serving as S
    h = H()
    A = I.rmat_matrix(22, 16, seed=5, dtype="i32")
    dA = h.DeviceCSR.from_host(A)
    n = A.n
    # SpRef: an induced subgraph of 2^16 random vertices in random order
    Iv = I.random_unique_sequence(n, 1 << 16, seed=41, stream=31)
    compare_on_device(h.spref(dA, Iv, Iv), oracle.spref(A, Iv, Iv), None, "spref A(I, I)")
    # contraction S*A*S^T with n/64 random clusters, int64
    lab = I.cluster_labels(n, n // 64, seed=42)
    S_, ST = I.cluster_S(lab, n // 64, "i64"), I.cluster_ST(lab, n // 64, "i64")
    A64 = I.CSR(A.m, A.n, A.rowptr, A.col, A.val.astype(np.int64), "i64")
    dA64 = h.DeviceCSR(dA.m, dA.n, dA.rowptr, dA.col, dA.val.to(torch.int64), "i64")
    SA = h.spgemm("plus_times", h.DeviceCSR.from_host(S_), dA64)
    G = h.spgemm("plus_times", SA, h.DeviceCSR.from_host(ST))
    R = oracle.spgemm("plus_times", oracle.spgemm("plus_times", S_, A64, nthreads=NT), ST, nthreads=NT)
    compare_on_device(G, R, None, "contraction S*A*S^T")
    del SA, G, R
    # SpAsgn: a batch update of 2^16 random edges (assign semantics)
    k = 1 << 16
    ev = I.draws(43, 32, 0, 3 * k).reshape(3, k)
    u = np.floor(I.uniform_f64(ev[0]) * n).astype(np.int32)
    v = np.floor(I.uniform_f64(ev[1]) * n).astype(np.int32)
    w = (np.floor(I.uniform_f64(ev[2]) * 100) + 1).astype(np.int32)
    Iu, Ju, B = S.update_operands((u, v, w))
    got = h.spasgn(dA, Iu, Ju, h.DeviceCSR.from_host(B))
    compare_on_device(got, oracle.spasgn(A, Iu, Ju, B), None, "spasgn A(I, J) = B")

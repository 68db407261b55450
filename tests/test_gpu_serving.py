"""Serving loop: every result in the mix equals the same request run alone on
its version, and the CPU oracle on that version; batching and overlap happen.

Graph: R-MAT scale 14, edge factor 16, int32 weights in [1, 100].  Requests:
SpRef induced subgraphs, contractions S*A*S^T (int64), SpAsgn batch updates,
arriving faster than they are served so that slots fill and batches form.
All operations are exact (selectors and integer arithmetic), so every
comparison is bit for bit.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import as_csr, assert_bitexact

pytestmark = pytest.mark.gpu


def test_serving_mix_matches_alone_and_oracle():
    import torch
    from paper_1109_3739_gb300 import hspgemm as h
    from paper_1109_3739_gb300 import serving as S

    A = I.rmat_matrix(14, 16, seed=5, dtype="i32")
    n = A.n
    store = S.GraphStore(A)
    store.pin_all()
    labels = S.make_label_sets(n, 2, seed=6)
    ex = S.Executor(store, labels, store.device, keep_results=True)
    ex.prepare()
    reqs = S.make_requests(n, 48, rate=4000.0, seed=9, label_sets=2, spref_range=(4, 11), asgn_range=(6, 10))
    srv = S.Server(store, ex, slots=4, max_batch=8, mem_budget=1 << 30)
    done, makespan = srv.run(reqs)
    assert len(done) == len(reqs)
    assert all(r.status == "ok" for r in done), [(r.rid, r.status, r.error) for r in done if r.status != "ok"]
    assert max(r.batch for r in done) < len(done)  # some batch held several requests
    starts = sorted((r.t_start, r.t_done) for r in done)
    overlap = any(starts[i + 1][0] < starts[i][1] for i in range(len(starts) - 1))
    assert overlap  # work of different batches was in flight together

    # host copies of every version, replaying the updates in the order they ran
    host = {0: A}
    for r in sorted((r for r in done if r.kind == "spasgn"), key=lambda r: r.new_version):
        Iv, Jv, B = S.update_operands(r.edges)
        host[r.new_version] = as_csr(oracle.spasgn(host[r.base_version], Iv, Jv, B))
        assert r.new_version == r.base_version + 1

    s1 = torch.cuda.Stream()
    lock = __import__("threading").Lock()
    for r in done:
        got = S.materialize(r).to_host()
        # alone: the same request by itself on its version
        alone = S.Request(r.rid, r.kind, 0.0, I=r.I, labels_id=r.labels_id, edges=r.edges)
        if r.kind == "spasgn":
            ref = host[r.new_version]
            assert_bitexact(got, ref, f"spasgn {r.rid}")
            continue
        alone.version = r.version
        with torch.cuda.stream(s1):
            ex.run_batch([alone], s1, lock)
        assert_bitexact(got, S.materialize(alone).to_host(), f"{r.kind} {r.rid} alone")
        Av = host[r.version]
        if r.kind == "spref":
            ref = oracle.spref(Av, r.I, r.I)
        else:
            lab = labels[r.labels_id]
            k = max(1, n // 64)
            A64 = Av.with_values("i64", 0)
            A64.val = Av.val.astype(np.int64)
            SA = oracle.spgemm("plus_times", I.cluster_S(lab, k, "i64"), A64)
            ref = oracle.spgemm("plus_times", as_csr(SA), I.cluster_ST(lab, k, "i64"))
        assert_bitexact(got, ref, f"{r.kind} {r.rid} oracle")


def test_serial_baseline_runs():
    from paper_1109_3739_gb300 import serving as S
    A = I.rmat_matrix(12, 16, seed=7, dtype="i32")
    store = S.GraphStore(A)
    ex = S.Executor(store, S.make_label_sets(A.n, 1, seed=8), store.device, keep_results=False)
    ex.prepare()
    reqs = S.make_requests(A.n, 12, rate=1000.0, seed=10, label_sets=1, spref_range=(4, 9), asgn_range=(6, 8))
    done, makespan = S.run_serial(store, ex, reqs)
    summ = S.latency_summary(done, makespan)
    assert summ["requests"] == 12 and summ["all"]["p99_ms"] >= summ["all"]["p50_ms"]

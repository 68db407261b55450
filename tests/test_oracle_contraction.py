"""Pin of the triple product S*A*S^T (graph contraction, Section 4's triple
products) by an independent relabel-and-reduce: every edge (u, v, w) of A
becomes (label[u], label[v], w) and the edges that meet are summed, i.e. the
oracle's sparse() over the relabelled edge list.  Both parenthesisations of
the product must equal it exactly (int64)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact


@pytest.mark.parametrize("k", [1, 7, 64, 1 << 12])
def test_contraction_equals_relabel_and_reduce(k):
    A = I.rmat_matrix(12, 8, seed=41, dtype="i64", kind="signed")
    labels = I.cluster_labels(A.n, k, seed=42)
    S, ST = I.cluster_S(labels, k, "i64"), I.cluster_ST(labels, k, "i64")
    left = oracle.spgemm("plus_times", oracle.spgemm("plus_times", S, A), ST)
    right = oracle.spgemm("plus_times", S, oracle.spgemm("plus_times", A, ST))
    rows = np.repeat(np.arange(A.m, dtype=np.int64), np.diff(A.rowptr))
    ref = oracle.sparse(labels[rows].astype(np.int32), labels[A.col].astype(np.int32), A.val, k, k,
                        "plus_times", dtype="i64")
    assert_bitexact(left, ref, f"(S*A)*S^T, {k} clusters")
    assert_bitexact(right, ref, f"S*(A*S^T), {k} clusters")
    # edge weight is conserved
    assert int(ref.val.sum()) == int(A.val.sum())

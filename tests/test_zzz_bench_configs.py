"""Parity at the configurations bench.py times for its secondary workloads
(full size, against the CPU oracle):

* sparse() of the R-MAT scale-20 edge list with 16 edges per vertex (16.8M
  tuples, f32 values summed): `bench.py --workload sparse`;
* SpRef on R-MAT scale 20 (edge factor 8, f32): the random symmetric
  permutation A(p, p) and one of the ten induced subgraphs A(r_i, r_i), with
  the permutation bench.py draws: `bench.py --workload spref`.
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


def test_sparse_bench_config_rmat20_ef16():
    i, j, v = I.rmat_tuples(20, 16, seed=2, dtype="f32")
    n = 1 << 20
    got = H().sparse(i, j, v, n, n, add="plus_times", dtype="f32").to_host()
    ref, bound = oracle.sparse(i, j, v, n, n, "plus_times", dtype="f32", with_bound=True)
    assert_within(got, ref, bound, "f32", "sparse rmat20 ef16")


@pytest.fixture(scope="module")
def rmat20():
    return I.rmat_matrix(20, 8, seed=2, dtype="f32")


def test_spref_bench_config_permutation(rmat20):
    A = rmat20
    p = I.random_permutation(A.n, seed=12, stream=20).astype(np.int32)
    got = H().spref(H().DeviceCSR.from_host(A), p, p).to_host()
    assert_bitexact(got, oracle.spref(A, p, p), "A(p, p)")


def test_spref_bench_config_induced_subgraph(rmat20):
    A = rmat20
    p = I.random_permutation(A.n, seed=12, stream=20).astype(np.int32)
    r = p[: A.n // 10]
    got = H().spref(H().DeviceCSR.from_host(A), r, r).to_host()
    assert_bitexact(got, oracle.spref(A, r, r), "A(r_1, r_1)")

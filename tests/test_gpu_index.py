"""GPU SpRef / SpAsgn (hs_spref, hs_spasgn through the C ABI) and the Galerkin
triple product against the CPU oracle.

SpRef and SpAsgn move values without arithmetic (selector semirings), so
every comparison is bit for bit, in every value type.  The Galerkin product
R*A*R^T of the 7-point Laplacian on 128^3 with 2x2x2 aggregation equals
4 x the Laplacian on 64^3 exactly in FP64 (small integers).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact

pytestmark = pytest.mark.gpu


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


def dev(A):
    return H().DeviceCSR.from_host(A)


@pytest.mark.parametrize("dt", ["f64", "f32", "i32", "i64", "bool"])
def test_spref_small(dt):
    A = I.er_matrix(300, 250, 6, seed=31, dtype=dt, kind="signed")
    cases = [
        (I.random_subset_sorted(300, 80, 1), I.random_subset_sorted(250, 60, 2)),
        (I.random_unique_sequence(300, 90, 3), I.random_unique_sequence(250, 100, 4)),
        (I.random_sequence(300, 150, 5), I.random_sequence(250, 170, 6)),  # duplicates
        (np.zeros(0, np.int32), I.random_sequence(250, 5, 7)),
        (I.random_sequence(300, 5, 8), np.zeros(0, np.int32)),
        (np.arange(300, dtype=np.int32), np.arange(250, dtype=np.int32)),
    ]
    for Iv, Jv in cases:
        got = H().spref(dev(A), Iv, Jv, validate=True).to_host()
        assert_bitexact(got, oracle.spref(A, Iv, Jv), f"spref {dt} {len(Iv)}x{len(Jv)}")


@pytest.mark.parametrize("reps", [32, 33, 5000])
def test_spref_repeated_columns(reps):
    """J repeats one column reps times (Q's row for it holds reps entries):
    up to 32 the short-row build, beyond it Q = sparse(J, 1:len(J), 1) by the
    stable sort; both against the oracle."""
    A = I.er_matrix(400, 300, 5, seed=35, dtype="f32", kind="signed")
    Jv = np.concatenate([np.full(reps, 7, np.int32), I.random_sequence(300, 200, 36)])
    Jv = Jv[np.argsort(I.draws(37, 1, 0, len(Jv)), kind="stable")].astype(np.int32)  # interleave
    Iv = I.random_sequence(400, 150, 38)
    got = H().spref(dev(A), Iv, Jv).to_host()
    assert_bitexact(got, oracle.spref(A, Iv, Jv), f"spref J with {reps} repeats")


def test_spref_rejects_out_of_range():
    h = H()
    A = I.er_matrix(50, 40, 3, seed=32, dtype="f64")
    with pytest.raises(h.HsError) as e:
        h.spref(dev(A), np.array([0, 50], np.int32), np.array([1], np.int32))
    assert e.value.code == -1
    with pytest.raises(h.HsError):
        h.spref(dev(A), np.array([0], np.int32), np.array([-1], np.int32))


def test_spref_rmat20_config():
    """SpRef A(I,J) on R-MAT scale 20 (f32) with I, J random sorted subsets of length 2^18."""
    A = I.rmat_matrix(20, 8, seed=2, dtype="f32")
    Iv = I.random_subset_sorted(A.m, 1 << 18, 3, stream=8)
    Jv = I.random_subset_sorted(A.n, 1 << 18, 3, stream=9)
    got = H().spref(dev(A), Iv, Jv).to_host()
    assert_bitexact(got, oracle.spref(A, Iv, Jv), "spref rmat20")


@pytest.mark.parametrize("dt", ["f64", "f32", "i32", "i64", "bool"])
def test_spasgn_small(dt):
    A = I.er_matrix(200, 180, 6, seed=33, dtype=dt, kind="signed")
    for s, (ni, nj) in enumerate([(40, 30), (1, 1), (200, 180), (0, 7), (9, 0)]):
        Iv = I.random_unique_sequence(200, ni, 40 + s)
        Jv = I.random_unique_sequence(180, nj, 50 + s)
        if ni and nj:
            B = I.er_matrix(ni, nj, min(3, ni), seed=60 + s, dtype=dt, kind="signed")
        else:
            B = I.CSR(ni, nj, np.zeros(ni + 1, np.int64), np.zeros(0, np.int32),
                      I.random_values(0, dt, 1), dt)
        got = H().spasgn(dev(A), Iv, Jv, dev(B), validate=True).to_host()
        assert_bitexact(got, oracle.spasgn(A, Iv, Jv, B), f"spasgn {dt} {ni}x{nj}")


@pytest.mark.parametrize("dt,sr", [("f64", "plus_times"), ("i64", "plus_times"), ("i32", "min_plus"),
                                   ("f32", "min_plus")])
def test_extend_add(dt, sr):
    A = I.er_matrix(150, 150, 8, seed=34, dtype=dt, kind="signed")
    Iv = I.random_unique_sequence(150, 50, 70)
    Jv = I.random_unique_sequence(150, 40, 71)
    B = I.er_matrix(50, 40, 6, seed=72, dtype=dt, kind="signed")
    got = H().spasgn(dev(A), Iv, Jv, dev(B), accumulate=True, add=sr).to_host()
    assert_bitexact(got, oracle.spasgn(A, Iv, Jv, B, accumulate=True, sr=sr), "extend-add")


def test_spasgn_errors():
    h = H()
    A = I.er_matrix(30, 30, 3, seed=35, dtype="f64")
    B = I.er_matrix(2, 2, 1, seed=36, dtype="f64")
    with pytest.raises(h.HsError) as e:
        h.spasgn(dev(A), np.array([4, 4], np.int32), np.array([1, 2], np.int32), dev(B))
    assert e.value.code == -3
    with pytest.raises(h.HsError) as e:
        h.spasgn(dev(A), np.array([4, 30], np.int32), np.array([1, 2], np.int32), dev(B))
    assert e.value.code == -1


def test_spasgn_rmat_batch_update():
    """A batch update on an R-MAT graph: 4096 random edges assigned into A(I,J)."""
    A = I.rmat_matrix(16, 16, seed=5, dtype="i32")
    k = 4096
    u = I.random_sequence(A.m, k, 80)
    v = I.random_sequence(A.n, k, 81)
    Iv = np.unique(u).astype(np.int32)
    Jv = np.unique(v).astype(np.int32)
    rows = np.searchsorted(Iv, u)
    cols = np.searchsorted(Jv, v)
    keys = np.unique(rows.astype(np.int64) * len(Jv) + cols)
    rowptr, col = I.csr_from_unique_sorted_keys(keys, len(Iv), len(Jv))
    B = I.CSR(len(Iv), len(Jv), rowptr, col, I.random_values(len(col), "i32", 82), "i32")
    got = H().spasgn(dev(A), Iv, Jv, dev(B)).to_host()
    assert_bitexact(got, oracle.spasgn(A, Iv, Jv, B), "batch update")


def test_galerkin_128():
    """(R*A)*R^T for the 7-point Laplacian on 128^3 and 2x2x2 aggregation."""
    h = H()
    A = I.laplacian7(128, "f64")
    R = I.aggregation_R(128, 2, "f64")
    RT = I.aggregation_RT(128, 2, "f64")
    RA = h.spgemm("plus_times", dev(R), dev(A))
    C = h.spgemm("plus_times", RA, dev(RT)).to_host()
    coarse = I.laplacian7(64, "f64")
    coarse.val = coarse.val * 4.0
    assert_bitexact(C, coarse, "R*A*R^T = 4 L_64")
    # right-to-left parenthesisation gives the same matrix
    ART = h.spgemm("plus_times", dev(A), dev(RT))
    C2 = h.spgemm("plus_times", dev(R), ART).to_host()
    assert_bitexact(C2, coarse, "R*(A*R^T)")

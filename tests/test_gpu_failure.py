"""Failure detection without a GPU fault, through the C ABI.

- A bounded device-side wait that runs out: the radix sort behind sparse()
  (Section 2's constructor) waits for the digit counts of earlier tiles with a
  poll limit.  A test hook keeps one tile from publishing its counts (a flag
  that nothing sets) and shortens the limit, so the next tile's wait expires:
  the call must come back promptly with HS_ETIMEDOUT, leave nothing allocated,
  and the next call on the same context must give the oracle's matrix.
- The allocator returning NULL: for every k, a product, a sparse()
  construction and a SpRef whose k-th allocation fails either return
  HS_ENOMEM with every block they took handed back, or (an optional buffer,
  such as the product's sorted column lists) do without it and still give
  the oracle's result; so does the first k at which nothing fails.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np
import pytest

import oracle
from paper_1109_3739_gb300 import inputs as I
from tests.helpers import assert_bitexact, assert_within

pytestmark = pytest.mark.gpu

HS_ENOMEM, HS_ETIMEDOUT = -4, -5


def H():
    from paper_1109_3739_gb300 import hspgemm
    return hspgemm


def test_lookback_wait_expires_with_status():
    import torch
    h = H()
    L = h.library()
    ti, tj, tv = I.rmat_tuples(14, 16, seed=31, dtype="f32")  # 262144 tuples: 64 tiles of 4096
    n = 1 << 14
    assert L.hs_test_lookback_expiry(0, 3) == -1 and L.hs_test_lookback_expiry(64, -1) == -1
    assert L.hs_test_lookback_expiry(64, 5) == 0  # tile 5 never publishes; 64 polls
    t0 = time.perf_counter()
    with pytest.raises(h.HsError) as e:
        h.sparse(ti, tj, tv, n, n, device="cuda")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert e.value.code == HS_ETIMEDOUT
    assert dt < 5.0, f"the expired wait took {dt:.2f} s to come back"
    # the context is intact and the setting was consumed: the same call now
    # gives the oracle's matrix
    C = h.sparse(ti, tj, tv, n, n, device="cuda").to_host()
    R, bound = oracle.sparse(ti, tj, tv, n, n, "plus_times", dtype="f32", with_bound=True)
    assert_within(C, R, bound, "f32", "sparse() after an expired wait")


class _FailAt:
    """Allocator callbacks (torch memory) whose k-th allocation returns NULL;
    counts the blocks the library holds."""

    def __init__(self, h, device, k):
        self.base = h._TorchAlloc(device)
        self.k, self.calls = k, 0
        self._a = h.ALLOC_FN(self._alloc)
        self.struct = h.hs_allocator(self._a, self.base._f, None)

    def _alloc(self, nbytes, stream, ctx):
        self.calls += 1
        if self.calls == self.k:
            return None
        return self.base._alloc(nbytes, stream, ctx)

    @property
    def live(self):
        return len(self.base.live)


def _sweep(h, run, check):
    """run(al) -> (status, C descriptor), for k = 1, 2, ... until a call makes
    fewer than k allocations.  A failed allocation either ends the call with
    HS_ENOMEM and every block handed back, or was of an optional buffer (the
    sorted column lists, the B segment index), which the call does without:
    then its result must still be right.  Returns (allocations of a full
    call, number of k that ended in HS_ENOMEM, number served by a fallback)."""
    import torch
    nomem = fallback = 0
    for k in range(1, 200):
        al = _FailAt(h, torch.device("cuda"), k)
        st, c = run(al)
        torch.cuda.synchronize()
        if st == 0:
            check(c, al)
            h.library().hs_mat_free(ctypes.byref(c), ctypes.byref(al.struct), None)
            torch.cuda.synchronize()
            assert al.live == 0, f"{al.live} blocks left after hs_mat_free"
            if al.calls < k:  # nothing failed: the sweep is complete
                return k - 1, nomem, fallback
            fallback += 1
            continue
        assert st == HS_ENOMEM, (k, st)
        assert al.live == 0, f"allocation {k} failed: {al.live} blocks not handed back"
        assert not c.ptr and not c.idx and not c.val
        nomem += 1
    raise AssertionError("no call succeeded")


def _host(h, c, al):
    """C's arrays, which live in the allocator's blocks, copied to the host."""
    import torch
    n = int(c.nnz)
    live = al.base.live
    rowptr = live[c.ptr].view(torch.int64)[:c.m + 1]
    col = live[c.idx].view(torch.int32)[:n]
    val = None
    if c.val:
        tdt = {0: torch.float64, 1: torch.float32, 2: torch.int32, 3: torch.int64}[c.dtype]
        val = live[c.val].view(tdt)[:n]
    return h.DeviceCSR(c.m, c.n, rowptr, col, val, h.DTYPE_NAME[c.dtype]).to_host()


def test_allocator_failure_at_every_allocation():
    h = H()
    L = h.library()
    A = I.rmat_matrix(12, 8, seed=32, dtype="f32")
    dA = h.DeviceCSR.from_host(A)
    a = dA.desc()
    R, bound = oracle.spgemm("plus_times", A, A, with_bound=True)

    def run_spgemm(al):
        c = h.hs_mat()
        return L.hs_spgemm(h.SEMIRING["plus_times"], ctypes.byref(a), ctypes.byref(a), ctypes.byref(c),
                           ctypes.byref(al.struct), None, 0), c

    n_alloc, nomem, _ = _sweep(h, run_spgemm, lambda c, al: assert_within(_host(h, c, al), R, bound, "f32", "spgemm"))
    assert n_alloc >= 3 and nomem >= 3

    import torch
    ti, tj, tv = I.rmat_tuples(12, 8, seed=33, dtype="i64", kind="signed")
    It = torch.from_numpy(ti).cuda()
    Jt = torch.from_numpy(tj).cuda()
    Vt = torch.from_numpy(tv).cuda()
    Rs = oracle.sparse(ti, tj, tv, 4096, 4096, "plus_times", dtype="i64")

    def run_sparse(al):
        c = h.hs_mat()
        return L.hs_sparse(It.data_ptr(), Jt.data_ptr(), Vt.data_ptr(), len(ti), 4096, 4096, h.DTYPE["i64"],
                           h.SEMIRING["plus_times"], ctypes.byref(c), ctypes.byref(al.struct), None, 0), c

    assert _sweep(h, run_sparse, lambda c, al: assert_bitexact(_host(h, c, al), Rs, "sparse"))[1] >= 3

    Iidx = I.random_sequence(4096, 700, seed=34)
    Jidx = I.random_sequence(4096, 900, seed=35)  # repeats: Q is built by the radix sort
    Id = torch.from_numpy(Iidx.astype(np.int32)).cuda()
    Jd = torch.from_numpy(Jidx.astype(np.int32)).cuda()
    Rr = oracle.spref(A, Iidx, Jidx)

    def run_spref(al):
        c = h.hs_mat()
        return L.hs_spref(ctypes.byref(a), Id.data_ptr(), len(Iidx), Jd.data_ptr(), len(Jidx), ctypes.byref(c),
                          ctypes.byref(al.struct), None, 0), c

    assert _sweep(h, run_spref, lambda c, al: assert_bitexact(_host(h, c, al), Rr, "spref"))[1] >= 3

"""The serving scheduler's host logic on the CPU: Server.run with a fake
store and executor (no kernels, no device memory) and dummy streams.

Checked: every request is served exactly once; batches respect max_batch;
no more batches run at once than there are slots; the estimated working set
in flight stays within the memory budget (a single request larger than the
budget runs alone); every request binds to the version current when it was
admitted and a version stays resident while a request bound to it runs;
latency_summary's percentiles and rate.
"""
from __future__ import annotations

import contextlib
import threading
import time
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1109_3739_gb300 import serving as S


class FakeStore:
    def __init__(self, nnz=1000, m=100):
        self.device = "cpu"
        self.graph = SimpleNamespace(A32=SimpleNamespace(nnz=nnz, m=m))
        self.versions = {0: self.graph}
        self.current = 0
        self.lock = threading.Lock()

    def get(self, vid):
        with self.lock:
            return self.versions[vid]

    def latest(self):
        with self.lock:
            return self.current

    def install(self):
        with self.lock:
            self.current += 1
            self.versions[self.current] = self.graph
            return self.current

    def release_unused(self, in_use):
        with self.lock:
            for vid in list(self.versions):
                if vid != self.current and vid not in in_use:
                    del self.versions[vid]


class FakeExecutor:
    def __init__(self, store, sleep=0.002):
        self.store, self.keep, self.sleep = store, False, sleep
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.batches = []
        self.missing_versions = []

    def run_batch(self, batch, stream, writer_lock):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.batches.append([r.rid for r in batch])
        for r in batch:  # the version a request is bound to must still be resident
            with self.store.lock:
                if r.version not in self.store.versions:
                    self.missing_versions.append((r.rid, r.version))
        time.sleep(self.sleep)
        for r in batch:
            if r.kind == "spasgn":
                with writer_lock:
                    r.base_version = self.store.latest()
                    r.new_version = self.store.install()
        with self.lock:
            self.running -= 1


@pytest.fixture
def no_cuda_streams(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "Stream", lambda device=None: object())
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())


def _requests(n=60, seed=3):
    rng = np.random.default_rng(seed)
    kinds = rng.choice(["spref", "contract", "spasgn"], size=n, p=[0.7, 0.1, 0.2])
    reqs = []
    for i, k in enumerate(kinds):
        r = S.Request(i, str(k), arrival=0.0005 * i)
        if k == "spref":
            r.I = np.arange(int(rng.integers(1, 50)), dtype=np.int32)
        elif k == "contract":
            r.labels_id = 0
        else:
            m = int(rng.integers(1, 20))
            r.edges = (np.zeros(m, np.int32), np.zeros(m, np.int32), np.ones(m, np.int32))
        reqs.append(r)
    return reqs


@pytest.mark.parametrize("slots,max_batch", [(1, 1), (2, 4), (4, 16)])
def test_every_request_once_within_slots_and_batches(no_cuda_streams, slots, max_batch):
    store = FakeStore()
    ex = FakeExecutor(store)
    reqs = _requests()
    done, makespan = S.Server(store, ex, slots=slots, max_batch=max_batch, mem_budget=1 << 40).run(
        reqs, realtime=False)
    assert sorted(r.rid for r in done) == list(range(len(reqs)))
    served = [rid for b in ex.batches for rid in b]
    assert sorted(served) == list(range(len(reqs)))  # once each
    assert max(len(b) for b in ex.batches) <= max_batch
    assert ex.max_running <= slots
    assert makespan > 0 and all(r.t_done >= r.t_start >= r.t_admit for r in done)


def test_memory_budget_bounds_the_work_in_flight(no_cuda_streams, monkeypatch):
    store = FakeStore()
    ex = FakeExecutor(store, sleep=0.003)
    budget = 1000
    in_flight = {"now": 0, "max_without_7": 0, "with_7": []}
    lock = threading.Lock()
    sizes = {}
    orig = ex.run_batch

    def run_batch(batch, stream, writer_lock):
        nb = sum(sizes[r.rid] for r in batch)
        with lock:
            in_flight["now"] += nb
            if any(r.rid == 7 for r in batch):
                in_flight["with_7"].append(in_flight["now"])
            else:
                in_flight["max_without_7"] = max(in_flight["max_without_7"], in_flight["now"])
        try:
            orig(batch, stream, writer_lock)
        finally:
            with lock:
                in_flight["now"] -= nb

    ex.run_batch = run_batch
    reqs = _requests(40)
    for r in reqs:
        sizes[r.rid] = 300 if r.rid != 7 else 5000  # request 7 alone exceeds the budget
    monkeypatch.setattr(S, "estimate_bytes", lambda r, A: sizes[r.rid])
    done, _ = S.Server(store, ex, slots=4, max_batch=8, mem_budget=budget).run(reqs, realtime=False)
    assert len(done) == len(reqs)
    # everything in flight fits the budget, except the oversize request, which runs alone
    assert [7] in ex.batches
    assert in_flight["with_7"] == [5000]
    assert 0 < in_flight["max_without_7"] <= budget


def test_versions_bind_at_admission_and_stay_resident(no_cuda_streams):
    store = FakeStore()
    ex = FakeExecutor(store)
    reqs = _requests(80, seed=5)
    done, _ = S.Server(store, ex, slots=3, max_batch=4, mem_budget=1 << 40).run(reqs, realtime=False)
    assert not ex.missing_versions
    updates = [r for r in done if r.kind == "spasgn"]
    assert store.latest() == len(updates)              # one new version per update
    assert sorted(r.new_version for r in updates) == list(range(1, len(updates) + 1))
    assert all(0 <= r.version <= store.latest() for r in done)
    # a request admitted after an update finished sees that update (or a later one)
    for u in updates:
        for r in done:
            if r.t_admit > u.t_done:
                assert r.version >= u.new_version


def test_latency_summary():
    done = []
    for i, (kind, lat) in enumerate([("spref", 0.010), ("spref", 0.020), ("contract", 0.050),
                                     ("spasgn", 0.030)]):
        r = S.Request(i, kind, arrival=1.0)
        r.t_done = 1.0 + lat
        done.append(r)
    out = S.latency_summary(done, makespan=2.0)
    assert out["requests"] == 4 and out["req_per_s"] == 2.0
    assert out["spref"]["n"] == 2 and abs(out["spref"]["p50_ms"] - 15.0) < 1e-9
    assert abs(out["contract"]["p99_ms"] - 50.0) < 1e-9
    assert abs(out["all"]["p50_ms"] - 25.0) < 1e-9


def test_malformed_requests_are_rejected_at_admission(no_cuda_streams):
    store = FakeStore()
    store.graph.A32.n = 100  # vertices 0..99
    ex = FakeExecutor(store)
    ex.labels = [None]       # one label set
    reqs = _requests(30, seed=7)
    bad = [
        S.Request(100, "spref", 0.0, I=np.array([3, 100], np.int32)),          # vertex out of range
        S.Request(101, "spref", 0.0, I=np.array([1.0, 2.0])),                   # not integer
        S.Request(102, "contract", 0.0, labels_id=3),                           # unknown label set
        S.Request(103, "spasgn", 0.0, edges=(np.zeros(3, np.int32), np.zeros(2, np.int32),
                                             np.ones(3, np.int32))),            # ragged arrays
        S.Request(104, "spasgn", 0.0, edges=(np.array([-1], np.int32), np.zeros(1, np.int32),
                                             np.ones(1, np.int32))),            # endpoint out of range
        S.Request(105, "pagerank", 0.0),                                        # unknown kind
        S.Request(106, "spref", 0.0),                                           # no vertex list
    ]
    done, _ = S.Server(store, ex, slots=2, max_batch=4, mem_budget=1 << 40).run(reqs + bad, realtime=False)
    assert sorted(r.rid for r in done) == sorted(r.rid for r in reqs + bad)
    served = sorted(rid for b in ex.batches for rid in b)
    assert served == sorted(r.rid for r in reqs)  # the good ones, once each; no bad one ran
    for r in bad:
        assert r.status == "rejected" and r.error, (r.rid, r.status, r.error)
        assert r.version == -1                    # never bound to a graph version
    out = S.latency_summary(done, 1.0)
    assert out["rejected"] == len(bad) and out["requests"] == len(reqs)


def test_cancelled_requests_are_skipped(no_cuda_streams):
    store = FakeStore()
    ex = FakeExecutor(store, sleep=0.05)
    reqs = _requests(8, seed=9)
    reqs[2].cancelled = True  # cancelled before it arrives
    server = S.Server(store, ex, slots=1, max_batch=1, mem_budget=1 << 40)

    def cancel_later():  # while request 0 runs, request 6 still waits for the one slot
        time.sleep(0.02)
        reqs[6].cancelled = True

    th = threading.Thread(target=cancel_later)
    th.start()
    done, _ = server.run(reqs, realtime=False)
    th.join()
    served = [rid for b in ex.batches for rid in b]
    assert 2 not in served and 6 not in served
    assert sorted(served) == [r.rid for r in reqs if r.rid not in (2, 6)]
    assert reqs[2].status == "cancelled" and reqs[6].status == "cancelled"
    assert len(done) == len(reqs)
    assert not ex.missing_versions


def test_a_failing_request_does_not_sink_its_batch():
    import torch

    class Stream:
        def synchronize(self):
            pass

    store = FakeStore()
    ex = S.Executor(store, [np.zeros(4, np.int32)], device="cpu")
    ran = []

    def run_one(r, stream, writer_lock):
        if r.rid == 1:
            raise RuntimeError("hs_spref: HS_EINVAL")
        ran.append(r.rid)

    ex._run_one = run_one
    batch = [S.Request(i, "spref", 0.0, I=np.arange(3, dtype=np.int32)) for i in range(4)]
    ex.run_batch(batch, Stream(), threading.Lock())
    assert ran == [0, 2, 3]
    assert [r.status for r in batch] == ["ok", "failed", "ok", "ok"]
    assert "HS_EINVAL" in batch[1].error and batch[1].result is None

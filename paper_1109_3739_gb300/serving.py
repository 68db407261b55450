"""Serving loop over a resident graph: SpRef subgraph extraction, graph
contraction S*A*S^T and SpAsgn batch updates (Section 3 and the experiments of
Section 4: subgraph extraction, contraction by a restriction operator, batch
update of a graph), admitted as they arrive and batched continuously.

* GraphStore keeps the graph in device memory in versions.  An update
  (SpAsgn, A(I,J) = B) builds version v+1 (copy-on-write: a new CSR); every
  request binds to the version current when it is admitted; updates run one
  at a time, each on the version current when it starts.
* Server admits requests as slots (worker streams) and memory (an estimate of
  each request's working set against a budget) free up.  A free slot takes
  every admitted request that is waiting (up to max_batch) and runs them on
  its stream: SpRef by the library's gather (hs_spref: the selected rows are
  gathered and relabelled on the device, R and Q are never formed),
  contractions as two products, updates one at a time.  Slots run on their
  own CUDA streams from their own host threads, so the GPU work of batches in
  flight overlaps.
* A malformed request (unknown kind, vertex or label set out of range,
  ragged edge arrays) is rejected at admission and never binds to a version;
  a request cancelled before its batch starts is skipped; a request whose
  library call fails is marked failed without sinking the rest of its batch.
* Every kernel runs in the library (hs_spgemm, hs_spref, hs_spasgn); this
  module only schedules, builds the small index arrays and measures.
"""
from __future__ import annotations

import dataclasses
import queue
import threading
import time

import numpy as np

from . import hspgemm as H
from . import inputs as I


@dataclasses.dataclass
class Request:
    rid: int
    kind: str                 # "spref" | "contract" | "spasgn"
    arrival: float            # seconds after the stream starts
    I: np.ndarray | None = None          # spref: vertex list (induced subgraph A(I, I))
    labels_id: int = -1                   # contract: which label vector
    edges: tuple | None = None            # spasgn: (u, v, w) arrays
    version: int = -1
    t_admit: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    result: object = None
    batch: int = 0
    base_version: int = -1    # spasgn: the version it updated
    new_version: int = -1     # spasgn: the version it produced
    status: str = "pending"   # "ok" | "rejected" | "cancelled" | "failed"
    error: str = ""
    cancelled: bool = False   # set by the client; honoured until the request's batch starts


def malformed(r: Request, n: int | None, nlabels: int | None) -> str:
    """Why a request cannot be served ("" if it can): checked on the host at
    admission, before it binds to a graph version."""
    if r.kind == "spref":
        if r.I is None:
            return "spref without a vertex list"
        x = np.asarray(r.I)
        if x.ndim != 1 or not np.issubdtype(x.dtype, np.integer):
            return "spref vertex list is not a 1-D integer array"
        if n is not None and len(x) and (int(x.min()) < 0 or int(x.max()) >= n):
            return "spref vertex out of range"
        return ""
    if r.kind == "contract":
        if nlabels is not None and not (0 <= r.labels_id < nlabels):
            return "unknown label set"
        return ""
    if r.kind == "spasgn":
        if r.edges is None or len(r.edges) != 3:
            return "spasgn without (u, v, w) edge arrays"
        u, v, w = (np.asarray(a) for a in r.edges)
        if not (u.ndim == v.ndim == w.ndim == 1 and len(u) == len(v) == len(w)):
            return "spasgn edge arrays differ in shape"
        if not all(np.issubdtype(a.dtype, np.integer) for a in (u, v, w)):
            return "spasgn edge arrays are not integer"
        if n is not None and len(u) and (min(int(u.min()), int(v.min())) < 0 or max(int(u.max()), int(v.max())) >= n):
            return "spasgn endpoint out of range"
        return ""
    return f"unknown request kind {r.kind!r}"


@dataclasses.dataclass
class Version:
    vid: int
    A32: H.DeviceCSR           # int32 weights
    A64: H.DeviceCSR           # the same structure with int64 weights (contractions)


class GraphStore:
    """Versioned resident graph (device memory)."""

    def __init__(self, A_host, device="cuda"):
        import torch
        self.device = torch.device(device)
        A32 = H.DeviceCSR.from_host(A_host, device=self.device)
        self.versions = {0: Version(0, A32, self._to64(A32))}
        self.current = 0
        self.lock = threading.Lock()

    @staticmethod
    def _to64(A32):
        import torch
        return H.DeviceCSR(A32.m, A32.n, A32.rowptr, A32.col, A32.val.to(torch.int64), "i64")

    def get(self, vid) -> Version:
        with self.lock:
            return self.versions[vid]

    def latest(self) -> int:
        with self.lock:
            return self.current

    def install(self, A32) -> int:
        with self.lock:
            vid = self.current + 1
            self.versions[vid] = Version(vid, A32, self._to64(A32))
            self.current = vid
            return vid

    def release_unused(self, in_use: set):
        """Drops versions that are neither current nor bound to a request in flight."""
        with self.lock:
            for vid in list(self.versions):
                if vid != self.current and vid not in in_use:
                    del self.versions[vid]

    def pin_all(self):
        """Keep every version (for checking results against their versions)."""
        self.release_unused = lambda in_use: None


# ------------------------------------------------------------------ workload
def make_requests(n: int, count: int, rate: float, seed: int, label_sets: int = 4,
                  mix=(0.7, 0.1, 0.2), spref_range=(6, 16), asgn_range=(10, 16)):
    """A Poisson stream of `count` requests at `rate` per second.

    Mix: SpRef of |I| log-uniform in [2^a, 2^b] distinct random vertices
    (induced subgraph), contraction with one of `label_sets` random label
    vectors (n/64 clusters), SpAsgn of k log-uniform in [2^c, 2^d] random
    edges with weights in [1, 100].
    """
    u = I.uniform_f64(I.draws(seed, 30, 0, 4 * count)).reshape(count, 4)
    gaps = -np.log1p(-u[:, 0]) / rate
    arrival = np.cumsum(gaps)
    reqs = []
    for r in range(count):
        x = u[r, 1]
        if x < mix[0]:
            lo, hi = spref_range
            k = int(2 ** (lo + u[r, 2] * (hi - lo)))
            Iv = I.random_unique_sequence(n, k, seed * 7919 + r, stream=31)
            reqs.append(Request(r, "spref", float(arrival[r]), I=Iv))
        elif x < mix[0] + mix[1]:
            reqs.append(Request(r, "contract", float(arrival[r]), labels_id=int(u[r, 2] * label_sets)))
        else:
            lo, hi = asgn_range
            k = int(2 ** (lo + u[r, 2] * (hi - lo)))
            ev = I.draws(seed * 7919 + r, 32, 0, 3 * k).reshape(3, k)
            uu = np.floor(I.uniform_f64(ev[0]) * n).astype(np.int32)
            vv = np.floor(I.uniform_f64(ev[1]) * n).astype(np.int32)
            ww = (np.floor(I.uniform_f64(ev[2]) * 100) + 1).astype(np.int32)
            reqs.append(Request(r, "spasgn", float(arrival[r]), edges=(uu, vv, ww)))
    return reqs


def make_label_sets(n: int, sets: int, seed: int):
    return [I.cluster_labels(n, max(1, n // 64), seed * 131 + s) for s in range(sets)]


def update_operands(edges):
    """I, J (sorted distinct endpoints) and B (the edges at their positions;
    a repeated edge keeps its last weight) of an SpAsgn batch update."""
    u, v, w = edges
    Iv = np.unique(u).astype(np.int32)
    Jv = np.unique(v).astype(np.int32)
    rows = np.searchsorted(Iv, u).astype(np.int64)
    cols = np.searchsorted(Jv, v).astype(np.int64)
    keys = rows * len(Jv) + cols
    order = np.argsort(keys, kind="stable")
    keys, w = keys[order], w[order]
    last = np.ones(len(keys), dtype=bool)
    last[:-1] = keys[1:] != keys[:-1]
    keys, w = keys[last], w[last]
    rowptr, col = I.csr_from_unique_sorted_keys(keys, len(Iv), len(Jv))
    return Iv, Jv, I.CSR(len(Iv), len(Jv), rowptr, col, w.astype(np.int32), "i32")


# ------------------------------------------------------------------ executor
class Executor:
    """Runs one batch of requests on one stream (called from a slot thread)."""

    def __init__(self, store: GraphStore, labels, device, keep_results: bool = True):
        import torch
        self.store = store
        self.keep = keep_results
        self.device = device
        self.labels = [torch.from_numpy(np.asarray(x, np.int32)).to(device) for x in labels]
        self._S = {}
        self._lock = threading.Lock()

    def prepare(self):
        """Builds every contraction operator ahead of the stream."""
        for lid in range(len(self.labels)):
            self.contraction_ops(lid)

    def contraction_ops(self, lid):
        """S (n/64 x n, S(label(v), v) = 1) and S^T as int64 device CSR, built once per label set."""
        with self._lock:
            if lid not in self._S:
                import torch
                lab = self.labels[lid].cpu().numpy().astype(np.int64)
                n = len(lab)
                k = max(1, n // 64)
                S = I.cluster_S(lab, k, "i64")
                ST = I.cluster_ST(lab, k, "i64")
                self._S[lid] = (H.DeviceCSR.from_host(S, device=self.device),
                                H.DeviceCSR.from_host(ST, device=self.device))
            return self._S[lid]

    def run_batch(self, batch, stream, writer_lock):
        """Runs each request of the batch on `stream`; a request whose call
        fails is marked failed and the others still run."""
        for r in batch:
            try:
                self._run_one(r, stream, writer_lock)
                r.status = "ok"
            except Exception as e:  # the library's status, reported per request
                r.status, r.error, r.result = "failed", str(e), None
        stream.synchronize()

    def _run_one(self, r, stream, writer_lock):
        if r.kind == "spref":
            # A(I, I) by the library's gather: I goes to the device once, the
            # selected rows are gathered, relabelled through I's inverse and
            # ordered there (hs_spref)
            A = self.store.get(r.version).A32
            out = H.spref(A, r.I, r.I, stream=stream)
            r.result = out if self.keep else None
        elif r.kind == "contract":
            ver = self.store.get(r.version)
            S, ST = self.contraction_ops(r.labels_id)
            SA = H.spgemm("plus_times", S, ver.A64, stream=stream)
            out = H.spgemm("plus_times", SA, ST, stream=stream)
            r.result = out if self.keep else None
        else:
            with writer_lock:  # updates apply one after another, each to the latest version
                ver = self.store.get(self.store.latest())
                r.base_version = ver.vid
                Iv, Jv, B = update_operands(r.edges)
                Bd = H.DeviceCSR.from_host(B, device=self.device)
                C = H.spasgn(ver.A32, Iv, Jv, Bd, stream=stream)
                stream.synchronize()
                r.result = C if self.keep else None
                r.new_version = self.store.install(C)


def estimate_bytes(r: Request, A) -> int:
    """Working-set estimate used for admission."""
    avg = A.nnz / max(1, A.m)
    if r.kind == "spref":
        k = len(r.I)
        return int(k * avg * 8 * 3 + k * 16)
    if r.kind == "contract":
        return int(A.nnz * 8 * 3)
    return int(A.nnz * 8 * 2 + len(r.edges[0]) * 16)


class Server:
    """Admission + continuous batching over `slots` streams."""

    def __init__(self, store: GraphStore, executor: Executor, slots: int = 4, max_batch: int = 16,
                 mem_budget: int = 8 << 30):
        self.store, self.ex = store, executor
        self.slots, self.max_batch, self.mem_budget = slots, max_batch, mem_budget

    def run(self, requests, realtime: bool = True):
        import torch
        pending = sorted(requests, key=lambda r: r.arrival)
        ready: queue.Queue = queue.Queue()
        free = threading.Semaphore(self.slots)
        mem_lock = threading.Lock()
        in_flight = {"bytes": 0}
        mem_ok = threading.Condition(mem_lock)
        writer_lock = threading.Lock()
        done = []
        done_lock = threading.Lock()
        streams = [torch.cuda.Stream(device=self.store.device) for _ in range(self.slots)]
        stream_pool: queue.Queue = queue.Queue()
        for s in streams:
            stream_pool.put(s)
        errors = []
        t0 = time.perf_counter()
        nbatch = [0]
        bound = {}  # version -> admitted requests not yet done
        keep_versions = set(self.store.versions) if self.ex.keep else set()

        def work(batch, nbytes):
            s = stream_pool.get()
            try:
                # a request cancelled before its batch starts is skipped
                live = []
                for r in batch:
                    if r.cancelled:
                        r.status = "cancelled"
                        r.t_done = time.perf_counter() - t0
                    else:
                        live.append(r)
                with torch.cuda.stream(s):
                    for r in live:
                        r.t_start = time.perf_counter() - t0
                    if live:
                        self.ex.run_batch(live, s, writer_lock)
                    now = time.perf_counter() - t0
                    for r in live:
                        r.t_done = now
            except Exception as e:  # surfaced by run()
                errors.append(e)
            finally:
                stream_pool.put(s)
                with mem_ok:
                    in_flight["bytes"] -= nbytes
                    mem_ok.notify_all()
                with done_lock:
                    done.extend(batch)
                    for r in batch:
                        bound[r.version] -= 1
                    self.store.release_unused({v for v, c in bound.items() if c > 0} | keep_versions)
                free.release()

        threads = []
        i = 0
        A0 = self.store.get(0).A32
        n_cols = getattr(A0, "n", None)
        nlabels = len(self.ex.labels) if hasattr(self.ex, "labels") else None
        while i < len(pending) or not ready.empty():
            # admit everything that has arrived; malformed or already
            # cancelled requests finish here, bound to no version
            now = time.perf_counter() - t0
            while i < len(pending) and (pending[i].arrival <= now or not realtime):
                r = pending[i]
                i += 1
                why = malformed(r, n_cols, nlabels)
                if why or r.cancelled:
                    r.status, r.error = ("rejected", why) if why else ("cancelled", "")
                    r.t_admit = r.t_done = time.perf_counter() - t0
                    with done_lock:
                        done.append(r)
                    continue
                ready.put(r)
            if ready.empty():
                time.sleep(max(0.0, min(0.002, pending[i].arrival - now)) if i < len(pending) else 0)
                continue
            free.acquire()  # a slot is free
            batch, nbytes = [], 0
            while not ready.empty() and len(batch) < self.max_batch:
                r = ready.queue[0]
                need = estimate_bytes(r, A0)
                with mem_ok:
                    if batch and in_flight["bytes"] + nbytes + need > self.mem_budget:
                        break
                    while not batch and in_flight["bytes"] + need > self.mem_budget and in_flight["bytes"] > 0:
                        mem_ok.wait(0.01)
                ready.get()
                r.t_admit = time.perf_counter() - t0
                r.version = self.store.latest()
                with done_lock:
                    bound[r.version] = bound.get(r.version, 0) + 1
                batch.append(r)
                nbytes += need
            with mem_ok:
                in_flight["bytes"] += nbytes
            nbatch[0] += 1
            for r in batch:
                r.batch = nbatch[0]
            th = threading.Thread(target=work, args=(batch, nbytes), daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        if errors:
            raise errors[0]
        makespan = max(r.t_done for r in done) if done else 0.0
        return sorted(done, key=lambda r: r.rid), makespan


def run_serial(store: GraphStore, executor: Executor, requests):
    """One request at a time on one stream, in arrival order (the comparison point)."""
    import torch
    s = torch.cuda.Stream(device=store.device)
    lock = threading.Lock()
    t0 = time.perf_counter()
    clock = 0.0
    for r in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        r.t_admit = time.perf_counter() - t0
        r.version = store.latest()
        r.t_start = r.t_admit
        with torch.cuda.stream(s):
            executor.run_batch([r], s, lock)
        r.t_done = time.perf_counter() - t0
        clock = r.t_done
    return sorted(requests, key=lambda r: r.rid), clock


def latency_summary(done, makespan):
    """Latency percentiles and rate over the requests that were served (a
    request that ran has status "ok"; pending means a scheduler without
    statuses, as in the serial loop); rejected, cancelled and failed requests
    are counted beside them."""
    served = [r for r in done if r.status in ("ok", "pending")]
    out = {"requests": len(served), "makespan_s": makespan,
           "req_per_s": len(served) / makespan if makespan else None}
    for st in ("rejected", "cancelled", "failed"):
        k = sum(1 for r in done if r.status == st)
        if k:
            out[st] = k
    done = served
    for kind in ("spref", "contract", "spasgn"):
        lat = np.array([r.t_done - r.arrival for r in done if r.kind == kind])
        if len(lat):
            out[kind] = {"n": int(len(lat)), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                         "p99_ms": float(np.percentile(lat, 99) * 1e3)}
    lat = np.array([r.t_done - r.arrival for r in done])
    if len(lat):
        out["all"] = {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3)}
    return out


def materialize(r: Request):
    """A request's result as a DeviceCSR of its own (SpRef results are rows of a stacked product)."""
    if r.kind == "spref" and isinstance(r.result, tuple):
        C, r0, r1, ncols = r.result
        return H.csr_rows(C, r0, r1, n=ncols)
    return r.result

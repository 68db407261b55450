"""Seeded synthetic inputs shared by the GPU path, the oracle tests and the benchmark.

This module only *generates* operands: it draws random numbers and lays out the
resulting triples as CSR.  It contains none of the arithmetic of the method under
test (no products, no accumulation, no indexing or assignment); both the CUDA
path and the CPU oracle receive the arrays built here.

Randomness is a counter-based SplitMix64 stream (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), evaluated with
NumPy uint64 arithmetic, so the same seed yields the same matrix on every
platform and NumPy version.

Workload shapes follow the paper's experiments (Section 4): R-MAT graphs with a
random symmetric relabelling, Erdos-Renyi matrices with a fixed number of
distinct nonzeros per column, a 7-point Laplacian with a piecewise-constant
aggregation operator (the restriction experiments), random cluster labels for
graph contraction, and random index vectors for SpRef/SpAsgn.

Conventions: indices are 0-based, column indices int32, row offsets int64, CSR
rows strictly increasing in column id.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "CSR", "DTYPES", "draws", "uniform_f64", "uniform_f32", "random_values",
    "er_matrix", "rmat_matrix", "laplacian7", "aggregation_R", "aggregation_RT",
    "cluster_S", "cluster_ST", "random_subset_sorted", "random_unique_sequence",
    "random_sequence", "csr_from_unique_sorted_keys", "identity", "permutation_matrix",
    "random_tuples", "rmat_tuples",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# numpy dtype and byte size for every value type the library accepts
DTYPES = {
    "f64": np.float64,
    "f32": np.float32,
    "i64": np.int64,
    "i32": np.int32,
    "bool": None,  # structure only: no value array
}


@dataclasses.dataclass
class CSR:
    """Host CSR matrix: rowptr int64[m+1], col int32[nnz], val dtype[nnz] or None."""
    m: int
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray | None
    dtype: str

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row(self, i: int):
        a, b = int(self.rowptr[i]), int(self.rowptr[i + 1])
        return self.col[a:b], (None if self.val is None else self.val[a:b])

    def with_values(self, dtype: str, seed: int, stream: int = 7, kind: str = "unit"):
        """Same structure, fresh seeded values of another type."""
        v = random_values(self.nnz, dtype, seed, stream, kind)
        return CSR(self.m, self.n, self.rowptr, self.col, v, dtype)

    def to_dense(self) -> np.ndarray:
        """Dense copy (tiny matrices only); absent entries are 0."""
        dt = np.float64 if self.val is None else self.val.dtype
        d = np.zeros((self.m, self.n), dtype=dt)
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        d[rows, self.col] = 1 if self.val is None else self.val
        return d

    def pattern(self) -> np.ndarray:
        """Dense boolean pattern (tiny matrices only)."""
        p = np.zeros((self.m, self.n), dtype=bool)
        rows = np.repeat(np.arange(self.m), np.diff(self.rowptr))
        p[rows, self.col] = True
        return p


# ----------------------------------------------------------------------------- rng
def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def draws(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """uint64 draws number start..start+count-1 of (seed, stream).

    Draw i is SplitMix64's output for state base + (i+1)*gamma, where the base
    state is itself a mix of the seed and the stream id, so streams do not
    overlap in practice.
    """
    with np.errstate(over="ignore"):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        t = np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        base = _mix64(s * _GAMMA + _mix64(t + _GAMMA))[0]
        idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        return _mix64(base + idx * _GAMMA)


def uniform_f64(u: np.ndarray) -> np.ndarray:
    """U[0,1) doubles with 53 random bits (exact)."""
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_f32(u: np.ndarray) -> np.ndarray:
    """U[0,1) floats with 24 random bits (exact in fp32)."""
    return ((u >> np.uint64(40)).astype(np.float64) * (1.0 / 16777216.0)).astype(np.float32)


def _below(u: np.ndarray, bound: int) -> np.ndarray:
    """Integers in [0, bound) from 53-bit uniforms (bound <= 2^40 keeps bias < 2^-13)."""
    return np.floor(uniform_f64(u) * bound).astype(np.int64)


def random_values(nnz: int, dtype: str, seed: int, stream: int = 7, kind: str = "unit"):
    """Values for nnz stored entries.

    kind="unit": f64/f32 uniform [0,1); i32/i64 uniform integers in [1, 100].
    kind="signed": f64/f32 uniform [-1,1); integers uniform in [-100, 100].
    bool: None (structure only).
    """
    if dtype == "bool":
        return None
    u = draws(seed, stream, 0, nnz)
    if dtype == "f64":
        v = uniform_f64(u)
        return (2.0 * v - 1.0) if kind == "signed" else v
    if dtype == "f32":
        v = uniform_f32(u)
        return (np.float32(2.0) * v - np.float32(1.0)).astype(np.float32) if kind == "signed" else v
    if dtype in ("i32", "i64"):
        npd = np.int32 if dtype == "i32" else np.int64
        if kind == "signed":
            return (_below(u, 201) - 100).astype(npd)
        return (_below(u, 100) + 1).astype(npd)
    raise ValueError(f"unknown dtype {dtype}")


# ----------------------------------------------------------------------------- csr
def csr_from_unique_sorted_keys(keys: np.ndarray, m: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """rowptr/col from strictly increasing keys row*n+col (uint64 or int64)."""
    keys = keys.astype(np.int64, copy=False)
    rows = keys // n
    col = (keys - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=m).astype(np.int64)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, col


def _csr_from_pairs(rows: np.ndarray, cols: np.ndarray, m: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """CSR pattern of the distinct (row, col) pairs."""
    keys = np.sort(rows.astype(np.int64) * n + cols.astype(np.int64))
    if len(keys):
        keep = np.empty(len(keys), dtype=bool)
        keep[0] = True
        np.not_equal(keys[1:], keys[:-1], out=keep[1:])
        keys = keys[keep]
    return csr_from_unique_sorted_keys(keys, m, n)


def identity(n: int, dtype: str = "f64") -> CSR:
    rowptr = np.arange(n + 1, dtype=np.int64)
    col = np.arange(n, dtype=np.int32)
    val = None if dtype == "bool" else np.ones(n, dtype=DTYPES[dtype])
    return CSR(n, n, rowptr, col, val, dtype)


def permutation_matrix(p: np.ndarray, dtype: str = "f64") -> CSR:
    """P with P(i, p[i]) = 1, so (P*A) row i is row p[i] of A."""
    n = len(p)
    rowptr = np.arange(n + 1, dtype=np.int64)
    col = np.asarray(p, dtype=np.int32)
    val = None if dtype == "bool" else np.ones(n, dtype=DTYPES[dtype])
    return CSR(n, n, rowptr, col, val, dtype)


# ----------------------------------------------------------------------------- ER
def er_matrix(m: int, n: int, d: int, seed: int, dtype: str = "f64", kind: str = "unit") -> CSR:
    """m x n Erdos-Renyi matrix with exactly d distinct nonzero rows in every column.

    The rows of a column are drawn uniformly; repeated rows are redrawn from
    later counters until the column holds d distinct rows (sampling without
    replacement).  Values are drawn afterwards, one per stored entry in CSR order.
    """
    if d > m:
        raise ValueError("d > m")
    if n == 0 or d == 0:
        return CSR(m, n, np.zeros(m + 1, np.int64), np.zeros(0, np.int32),
                   random_values(0, dtype, seed), dtype)
    rows = _below(draws(seed, 1, 0, n * d), m).reshape(n, d)
    nxt = n * d
    while True:
        rows.sort(axis=1)
        dup = np.zeros_like(rows, dtype=bool)
        dup[:, 1:] = rows[:, 1:] == rows[:, :-1]
        cnt = int(dup.sum())
        if cnt == 0:
            break
        rows[dup] = _below(draws(seed, 1, nxt, cnt), m)
        nxt += cnt
    cols = np.repeat(np.arange(n, dtype=np.int64), d)
    rowptr, col = _csr_from_pairs(rows.reshape(-1), cols, m, n)
    val = random_values(len(col), dtype, seed, stream=2, kind=kind)
    return CSR(m, n, rowptr, col, val, dtype)


# ----------------------------------------------------------------------------- R-MAT
def rmat_edges(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
               chunk: int = 1 << 20) -> tuple[np.ndarray, np.ndarray]:
    """Raw R-MAT edge list (with duplicates): edge_factor * 2^scale edges.

    Every edge descends `scale` levels of the recursive quadrant split; at each
    level a 16-bit uniform picks quadrant (0,0) with probability a, (0,1) with b,
    (1,0) with c and (1,1) with d = 1-a-b-c (thresholds rounded to 1/65536).
    One 64-bit draw supplies four levels (its 16-bit fields, least significant first).
    """
    ne = edge_factor << scale
    nd = (scale + 3) // 4
    rows = np.empty(ne, dtype=np.int64)
    cols = np.empty(ne, dtype=np.int64)
    t1 = np.uint16(round(a * 65536.0))
    t2 = np.uint16(round((a + b) * 65536.0))
    t3 = np.uint16(min(65535, round((a + b + c) * 65536.0)))
    shifts = np.arange(scale - 1, -1, -1, dtype=np.int64)
    for e0 in range(0, ne, chunk):
        e1 = min(ne, e0 + chunk)
        d = draws(seed, 3, e0 * nd, (e1 - e0) * nd).reshape(e1 - e0, nd)
        # four 16-bit fields per draw, level l uses field l % 4 of draw l // 4
        u = d.astype("<u8", copy=False).view("<u2").reshape(e1 - e0, nd * 4)[:, :scale]
        q = (u >= t1).astype(np.int8) + (u >= t2) + (u >= t3)  # quadrant 0..3
        rows[e0:e1] = ((q >= 2).astype(np.int64) << shifts).sum(axis=1)
        cols[e0:e1] = ((q & 1).astype(np.int64) << shifts).sum(axis=1)
    return rows, cols


def random_permutation(n: int, seed: int, stream: int = 4) -> np.ndarray:
    """Uniform random permutation of 0..n-1 (argsort of distinct random keys)."""
    return np.argsort(draws(seed, stream, 0, n), kind="stable").astype(np.int64)


def rmat_matrix(scale: int, edge_factor: int = 8, a: float = 0.57, b: float = 0.19,
                c: float = 0.19, seed: int = 2, dtype: str = "f32", permute: bool = True,
                kind: str = "unit") -> CSR:
    """2^scale x 2^scale R-MAT adjacency matrix, duplicates merged.

    With permute=True the vertex labels are relabelled by a seeded random
    permutation p (entry (u,v) becomes (p[u], p[v])), the random symmetric
    permutation the paper applies to balance load (Section 4).  Self loops are
    kept.  Values are drawn after merging, one per unique entry in CSR order.
    """
    n = 1 << scale
    r, cc = rmat_edges(scale, edge_factor, a, b, c, seed)
    if permute:
        p = random_permutation(n, seed)
        r, cc = p[r], p[cc]
    rowptr, col = _csr_from_pairs(r, cc, n, n)
    del r, cc
    val = random_values(len(col), dtype, seed, stream=5, kind=kind)
    return CSR(n, n, rowptr, col, val, dtype)


# ----------------------------------------------------------------------------- AMG
def laplacian7(nx: int, dtype: str = "f64") -> CSR:
    """7-point Laplacian on an nx^3 grid with Dirichlet boundary (diag 6, off-diagonal -1).

    Vertex (x, y, z) has index (x*nx + y)*nx + z.
    """
    n = nx ** 3
    idx = np.arange(n, dtype=np.int64)
    x, rem = np.divmod(idx, nx * nx)
    y, z = np.divmod(rem, nx)
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 6.0)]
    for dx, dy, dz in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
        ok = ((x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < nx) &
              (z + dz >= 0) & (z + dz < nx))
        rows.append(idx[ok])
        cols.append(((x[ok] + dx) * nx + (y[ok] + dy)) * nx + (z[ok] + dz))
        vals.append(np.full(int(ok.sum()), -1.0))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.argsort(rows * n + cols, kind="stable")
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    v = None if dtype == "bool" else vals.astype(DTYPES[dtype])
    return CSR(n, n, rowptr, cols.astype(np.int32), v, dtype)


def _aggregate_of(nx: int, block: int) -> np.ndarray:
    n = nx ** 3
    ncx = nx // block
    idx = np.arange(n, dtype=np.int64)
    x, rem = np.divmod(idx, nx * nx)
    y, z = np.divmod(rem, nx)
    return ((x // block) * ncx + (y // block)) * ncx + (z // block)


def aggregation_R(nx: int, block: int = 2, dtype: str = "f64") -> CSR:
    """Piecewise-constant aggregation R ((nx/block)^3 x nx^3): R(agg(v), v) = 1, one 1 per column."""
    n = nx ** 3
    nc = (nx // block) ** 3
    agg = _aggregate_of(nx, block)
    order = np.argsort(agg * n + np.arange(n), kind="stable")
    cols = np.arange(n, dtype=np.int64)[order]
    counts = np.bincount(agg, minlength=nc).astype(np.int64)
    rowptr = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    val = None if dtype == "bool" else np.ones(n, dtype=DTYPES[dtype])
    return CSR(nc, n, rowptr, cols.astype(np.int32), val, dtype)


def aggregation_RT(nx: int, block: int = 2, dtype: str = "f64") -> CSR:
    """R^T (nx^3 x (nx/block)^3), generated directly: row v holds a 1 at column agg(v)."""
    n = nx ** 3
    nc = (nx // block) ** 3
    rowptr = np.arange(n + 1, dtype=np.int64)
    col = _aggregate_of(nx, block).astype(np.int32)
    val = None if dtype == "bool" else np.ones(n, dtype=DTYPES[dtype])
    return CSR(n, nc, rowptr, col, val, dtype)


def cluster_labels(n: int, nclusters: int, seed: int) -> np.ndarray:
    return _below(draws(seed, 6, 0, n), nclusters)


def cluster_S(labels: np.ndarray, nclusters: int, dtype: str = "i64") -> CSR:
    """Contraction operator S (nclusters x n) with S(label[v], v) = 1."""
    n = len(labels)
    order = np.argsort(labels * n + np.arange(n), kind="stable")
    counts = np.bincount(labels, minlength=nclusters).astype(np.int64)
    rowptr = np.zeros(nclusters + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    val = None if dtype == "bool" else np.ones(n, dtype=DTYPES[dtype])
    return CSR(nclusters, n, rowptr, np.arange(n, dtype=np.int32)[order], val, dtype)


def cluster_ST(labels: np.ndarray, nclusters: int, dtype: str = "i64") -> CSR:
    """S^T (n x nclusters), generated directly: row v holds a 1 at column label[v]."""
    n = len(labels)
    val = None if dtype == "bool" else np.ones(n, dtype=DTYPES[dtype])
    return CSR(n, nclusters, np.arange(n + 1, dtype=np.int64),
               np.asarray(labels, dtype=np.int32), val, dtype)


# ----------------------------------------------------------------------------- index vectors
def random_subset_sorted(n: int, k: int, seed: int, stream: int = 8) -> np.ndarray:
    """k distinct indices of 0..n-1, ascending (first k of a random permutation, sorted)."""
    return np.sort(random_permutation(n, seed, stream)[:k]).astype(np.int32)


def random_unique_sequence(n: int, k: int, seed: int, stream: int = 9) -> np.ndarray:
    """k distinct indices of 0..n-1 in random order."""
    return random_permutation(n, seed, stream)[:k].astype(np.int32)


def random_sequence(n: int, k: int, seed: int, stream: int = 10) -> np.ndarray:
    """k indices of 0..n-1 drawn with replacement (duplicates allowed), random order."""
    return _below(draws(seed, stream, 0, k), n).astype(np.int32)


# ----------------------------------------------------------------------------- tuples
def random_tuples(m: int, n: int, nnz: int, seed: int, dtype: str = "f64", kind: str = "signed"):
    """(i, j, v) of nnz uniform random positions of an m x n matrix, drawn with
    replacement (so positions repeat once nnz approaches m*n), in random order;
    v is None for bool."""
    i = random_sequence(m, nnz, seed, stream=13) if m > 0 else np.zeros(nnz, np.int32)
    j = random_sequence(n, nnz, seed, stream=14) if n > 0 else np.zeros(nnz, np.int32)
    return i, j, random_values(nnz, dtype, seed, stream=15, kind=kind)


def rmat_tuples(scale: int, edge_factor: int = 8, seed: int = 2, dtype: str = "f32", kind: str = "unit",
                a: float = 0.57, b: float = 0.19, c: float = 0.19):
    """The raw R-MAT edge list of rmat_matrix (duplicates kept, vertices
    relabelled by the same seeded permutation) as int32 (i, j) with one value
    per edge: the input of building the adjacency matrix with sparse()."""
    n = 1 << scale
    r, cc = rmat_edges(scale, edge_factor, a, b, c, seed)
    p = random_permutation(n, seed)
    i, j = p[r].astype(np.int32), p[cc].astype(np.int32)
    return i, j, random_values(len(i), dtype, seed, stream=16, kind=kind)


# ----------------------------------------------------------------------------- batches
def batched_er_sizes(count: int, seed: int, nmin: int = 256, nmax: int = 65536, dmin: int = 2, dmax: int = 32):
    """(n_i, d_i) of a batch of Erdos-Renyi problems: n_i = floor(exp(U[ln nmin, ln nmax])),
    d_i uniform integer in [dmin, dmax] (one d_i for A_i and B_i)."""
    u = uniform_f64(draws(seed, 20, 0, count))
    n = np.floor(np.exp(np.log(nmin) + u * (np.log(nmax) - np.log(nmin)))).astype(np.int64)
    n = np.clip(n, nmin, nmax)
    d = _below(draws(seed, 21, 0, count), dmax - dmin + 1) + dmin
    d = np.minimum(d, n)
    return n, d


def batched_er_problem(i: int, n: int, d: int, seed: int, dtype: str = "f64"):
    """Problem i of a batch: square n x n A_i and B_i with d distinct nonzeros per column."""
    base = (seed * 1000003 + i) * 2
    return (er_matrix(n, n, d, seed=base + 1, dtype=dtype),
            er_matrix(n, n, d, seed=base + 2, dtype=dtype))


def _batched_worker(args):
    i, n, d, seed, dtype = args
    return batched_er_problem(i, n, d, seed, dtype)


def batched_er(count: int, seed: int, dtype: str = "f64", nmax: int = 65536, workers: int = 0):
    """All problems of a batch (list of (A_i, B_i)); workers > 1 generates them in
    a spawn-context process pool (results identical to the serial order)."""
    n, d = batched_er_sizes(count, seed, nmax=nmax)
    jobs = [(i, int(n[i]), int(d[i]), seed, dtype) for i in range(count)]
    if workers > 1 and count > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_batched_worker, jobs, chunksize=max(1, count // (4 * workers))))
    return [_batched_worker(j) for j in jobs]

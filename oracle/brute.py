"""Dense brute force for tiny inputs (test infrastructure only).

C(i,j) is defined exactly when some k has both A(i,k) and B(k,j) stored, and
then equals the semiring sum over those k of A(i,k) (x) B(k,j) (Section 1: SpGEMM
over a semiring; nonzero operations only, Section 2).  Pure-Python loops over a
dense pattern; intended for dimensions up to ~64.
"""
from __future__ import annotations

import numpy as np


def _dense(A):
    pat = np.zeros((A.m, A.n), dtype=bool)
    val = [[None] * A.n for _ in range(A.m)]
    for i in range(A.m):
        for q in range(int(A.rowptr[i]), int(A.rowptr[i + 1])):
            j = int(A.col[q])
            pat[i, j] = True
            val[i][j] = None if A.val is None else A.val[q].item()
    return pat, val


def spgemm(sr: str, A, B):
    """Returns (pattern bool[m,n], values list-of-lists, bound list-of-lists).

    Values: (+,x) float sums in Python floats (double), integer sums exact;
    (min,+) on f32 uses numpy float32 addition; bool has no values.
    bound = sum of |a||b| for (+,x) floats.
    """
    pa, va = _dense(A)
    pb, vb = _dense(B)
    m, n, kk = A.m, B.n, A.n
    pat = np.zeros((m, n), dtype=bool)
    val = [[None] * n for _ in range(m)]
    bnd = [[0.0] * n for _ in range(m)]
    for i in range(m):
        for j in range(n):
            acc = None
            for k in range(kk):
                if not (pa[i, k] and pb[k, j]):
                    continue
                a, b = va[i][k], vb[k][j]
                if sr == "or_and":
                    prod = True
                elif sr == "plus_times":
                    prod = a * b
                    bnd[i][j] += abs(a) * abs(b)
                elif sr == "min_plus":
                    prod = float(np.float32(a) + np.float32(b)) if A.dtype == "f32" else a + b
                elif sr == "select2nd":
                    prod = b
                elif sr == "select1st":
                    prod = a
                else:
                    raise ValueError(sr)
                if acc is None:
                    acc = prod
                elif sr == "plus_times":
                    acc = acc + prod
                elif sr == "min_plus":
                    acc = min(acc, prod)
                elif sr in ("select2nd", "select1st"):
                    raise ValueError("selector product with two contributions")
            if acc is not None:
                pat[i, j] = True
                val[i][j] = acc
    return pat, val, bnd


def sparse(i, j, v, m: int, n: int, sr: str = "plus_times", with_bound: bool = False):
    """sparse(i, j, v, m, n) by a dictionary keyed on (row, column), tuples
    folded in the order given.  Returns {(r, c): value} (True for bool).

    With with_bound also returns {(r, c): sum of |v| over the position's
    tuples}, added in tuple order in Python floats (0.0 for bool)."""
    out = {}
    mag = {}
    for k in range(len(i)):
        key = (int(i[k]), int(j[k]))
        if not (0 <= key[0] < m and 0 <= key[1] < n):
            raise ValueError("index out of range")
        x = True if v is None else v[k].item()
        ax = 0.0 if v is None else abs(float(x))
        mag[key] = ax if key not in mag else mag[key] + ax
        if key not in out:
            out[key] = x
        elif sr == "plus_times":
            out[key] = out[key] + x
        elif sr == "min_plus":
            out[key] = min(out[key], x)
        elif sr == "or_and":
            out[key] = True
        else:
            raise ValueError(sr)
    return (out, mag) if with_bound else out

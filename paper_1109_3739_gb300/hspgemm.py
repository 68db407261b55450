"""Python binding of libhspgemm (the C ABI in include/hspgemm.h).

Argument marshalling only: every step of SpGEMM / SpRef / SpAsgn runs in the
library's CUDA kernels.  PyTorch supplies device memory (through the ABI's
allocator callbacks, backed by the caching allocator) and the stream.  There
is no fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhspgemm.so")

SEMIRING = {"plus_times": 0, "or_and": 1, "min_plus": 2, "select2nd": 3, "select1st": 4}
DTYPE = {"f64": 0, "f32": 1, "i32": 2, "i64": 3, "bool": 4}
DTYPE_NAME = {v: k for k, v in DTYPE.items()}
VBYTES = {"f64": 8, "f32": 4, "i32": 4, "i64": 8, "bool": 0}
I_NP = {"f64": np.float64, "f32": np.float32, "i32": np.int32, "i64": np.int64}
FLAG_VALIDATE = 1
STATUS = {0: "HS_OK", -1: "HS_EINVAL", -2: "HS_ENONCANON", -3: "HS_EDUP", -4: "HS_ENOMEM",
          -5: "HS_ETIMEDOUT", -6: "HS_ECUDA", -7: "HS_EUNSUPPORTED", -8: "HS_EINTERNAL",
          -9: "HS_ESCRATCH", -10: "HS_ECAPACITY"}


class HsError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        L = _lib()
        detail = L.hs_last_error_detail().decode()
        super().__init__(f"{what}: {STATUS.get(code, code)} ({L.hs_strerror(code).decode()})"
                         + (f" [{detail}]" if detail else ""))


class hs_mat(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("dtype", ctypes.c_int32), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nzr", ctypes.c_int64),
                ("ptr", ctypes.c_void_p), ("idx", ctypes.c_void_p), ("ids", ctypes.c_void_p),
                ("val", ctypes.c_void_p)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class hs_tuning(ctypes.Structure):
    _fields_ = [("warp_s_max", ctypes.c_int32), ("mid_s_max", ctypes.c_int32), ("large_s_max", ctypes.c_int32),
                ("sym_mid_s_max", ctypes.c_int32), ("sym_heavy_from", ctypes.c_int32), ("sort_max", ctypes.c_int32),
                ("sort_pct", ctypes.c_int32), ("spa_max", ctypes.c_int32), ("heavy_part_kb", ctypes.c_int32),
                ("num_heavy_from", ctypes.c_int32)]


TUNING_FIELDS = tuple(name for name, _ in hs_tuning._fields_)


class hs_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


_lock = threading.Lock()
_L = None


def _lib():
    global _L
    if _L is not None:
        return _L
    with _lock:
        if _L is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1109_3739_gb300.build.build()")
            # torch first: its CUDA runtime must be the one the library binds to
            # (libhspgemm needs libcudart.so.13; if the system copy were loaded
            # first, torch would map a second runtime into the process)
            _torch()
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            vp, i64, ci, u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32
            L.hs_spgemm.argtypes = [ci, P(hs_mat), P(hs_mat), P(hs_mat), P(hs_allocator), vp, u32]
            L.hs_spgemm.restype = ci
            L.hs_spref.argtypes = [P(hs_mat), vp, i64, vp, i64, P(hs_mat), P(hs_allocator), vp, u32]
            L.hs_spref.restype = ci
            L.hs_spasgn.argtypes = [P(hs_mat), vp, i64, vp, i64, P(hs_mat), ci, ci, P(hs_mat),
                                    P(hs_allocator), vp, u32]
            L.hs_spasgn.restype = ci
            L.hs_sparse.argtypes = [vp, vp, vp, i64, i64, i64, ci, ci, P(hs_mat), P(hs_allocator), vp, u32]
            L.hs_spgemm_batched.argtypes = [ci, i64, P(hs_mat), P(hs_mat), P(hs_mat), P(ctypes.c_int64),
                                             P(hs_allocator), vp, u32]
            L.hs_spgemm_batched.restype = ci
            L.hs_spgemm_noalloc.argtypes = [ci, P(hs_mat), P(hs_mat), P(hs_mat), i64, vp]
            L.hs_spgemm_noalloc.restype = ci
            L.hs_plan_create.argtypes = [ci, P(hs_mat), P(hs_mat), P(hs_mat), P(vp), P(hs_allocator), vp, u32]
            L.hs_plan_create.restype = ci
            L.hs_plan_execute.argtypes = [vp, vp, vp, vp, vp]
            L.hs_plan_execute.restype = ci
            L.hs_plan_status.argtypes = [vp, vp]
            L.hs_plan_status.restype = ci
            L.hs_plan_destroy.argtypes = [vp, vp]
            L.hs_plan_destroy.restype = None
            L.hs_batch_stack.argtypes = [i64, P(hs_mat), P(hs_mat), P(hs_mat), P(hs_mat), P(ctypes.c_int64),
                                         P(hs_allocator), vp]
            L.hs_batch_stack.restype = ci
            L.hs_spgemm_to_host.argtypes = [ci, P(hs_mat), P(hs_mat), i64, vp, vp, vp, i64, P(ctypes.c_int64), vp, u32]
            L.hs_spgemm_to_host.restype = ci
            L.hs_trim_memory.restype = ci
            L.hs_test_lookback_expiry.argtypes = [ci, i64]
            L.hs_test_lookback_expiry.restype = ci
            L.hs_batch_plan_create.argtypes = [ci, i64, P(hs_mat), P(hs_mat), P(vp), P(hs_allocator), vp, u32]
            L.hs_batch_plan_create.restype = ci
            L.hs_batch_plan_execute.argtypes = [vp, vp]
            L.hs_batch_plan_execute.restype = ci
            L.hs_batch_plan_result.argtypes = [vp, P(hs_mat), P(ctypes.c_int64), vp]
            L.hs_batch_plan_result.restype = ci
            L.hs_batch_plan_destroy.argtypes = [vp, vp]
            L.hs_batch_plan_destroy.restype = None
            L.hs_batch_plan_phase_ms.argtypes = [vp, P(ctypes.c_double), vp]
            L.hs_batch_plan_phase_ms.restype = ci
            L.hs_set_tuning.argtypes = [P(hs_tuning)]
            L.hs_set_tuning.restype = ci
            L.hs_get_tuning.argtypes = [P(hs_tuning)]
            L.hs_get_tuning.restype = ci
            L.hs_mat_free.argtypes = [P(hs_mat), P(hs_allocator), vp]
            L.hs_mat_free.restype = None
            L.hs_strerror.argtypes = [ci]
            L.hs_strerror.restype = ctypes.c_char_p
            L.hs_last_cuda_error.restype = ci
            L.hs_last_error_detail.restype = ctypes.c_char_p
            L.hs_version.restype = ci
            L.hs_launch_count.restype = ctypes.c_int64
            L.hs_profile_enable.argtypes = [ci]
            L.hs_profile_reset.argtypes = []
            L.hs_profile_read.argtypes = [P(ctypes.c_double), P(ctypes.c_int64), P(ctypes.c_char_p), ci]
            L.hs_profile_read.restype = ci
            _L = L
    return _L


def library():
    """The loaded ctypes library (raises if it has not been built)."""
    return _lib()


def _torch():
    import torch
    return torch


# ------------------------------------------------------------------ memory
class _TorchAlloc:
    """Allocator callbacks backed by torch's caching allocator.

    Each allocation is a uint8 tensor kept alive in a dict keyed by its device
    address until the library frees it or the binding adopts it as an output.
    """

    def __init__(self, device):
        self.device = device
        self.live: dict[int, object] = {}
        self._a = ALLOC_FN(self._alloc)
        self._f = FREE_FN(self._free)
        self.struct = hs_allocator(self._a, self._f, None)

    def _alloc(self, nbytes, stream, ctx):
        try:
            t = _torch().empty(int(nbytes), dtype=_torch().uint8, device=self.device)
        except Exception:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, nbytes, stream, ctx):
        self.live.pop(int(ptr) if ptr else 0, None)

    def adopt(self, ptr, count, dtype):
        """Take ownership of a library output as a typed tensor of `count` elements."""
        t = self.live.pop(int(ptr))
        return t.view(dtype)[:count]


class DeviceCSR:
    """A CSR (or DCSR) matrix in device memory: torch tensors + shape + dtype name."""

    def __init__(self, m, n, rowptr, col, val, dtype, ids=None):
        self.m, self.n = int(m), int(n)
        self.rowptr, self.col, self.val, self.dtype, self.ids = rowptr, col, val, dtype, ids

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def fmt(self) -> str:
        return "dcsr" if self.ids is not None else "csr"

    @classmethod
    def from_host(cls, A, device="cuda", dcsr: bool = False, non_blocking: bool = False):
        """Copy an inputs.CSR (numpy) to the device; dcsr=True stores only non-empty rows."""
        torch = _torch()
        rowptr = np.asarray(A.rowptr, np.int64)
        ids = None
        if dcsr:
            nz = np.nonzero(np.diff(rowptr))[0]
            ids = torch.from_numpy(nz.astype(np.int32)).to(device, non_blocking=non_blocking)
            rowptr = np.concatenate([rowptr[nz], rowptr[-1:]])
        val = None if A.val is None else torch.from_numpy(np.ascontiguousarray(A.val)).to(device, non_blocking=non_blocking)
        return cls(A.m, A.n, torch.from_numpy(rowptr).to(device, non_blocking=non_blocking),
                   torch.from_numpy(np.asarray(A.col, np.int32)).to(device, non_blocking=non_blocking),
                   val, A.dtype if A.val is not None else "bool", ids)

    def to_host(self):
        """inputs.CSR copy on the host (CSR form)."""
        from .inputs import CSR
        rp = self.rowptr.cpu().numpy()
        col = self.col.cpu().numpy()
        val = None if self.val is None else self.val.cpu().numpy()
        if self.ids is not None:
            full = np.zeros(self.m + 1, np.int64)
            ids = self.ids.cpu().numpy()
            counts = np.zeros(self.m, np.int64)
            counts[ids] = np.diff(rp)
            np.cumsum(counts, out=full[1:])
            rp = full
        return CSR(self.m, self.n, rp, col, val, self.dtype)

    def desc(self) -> hs_mat:
        nzr = 0 if self.ids is None else int(self.ids.numel())
        return hs_mat(1 if self.ids is not None else 0, DTYPE[self.dtype], self.m, self.n, self.nnz, nzr,
                      self.rowptr.data_ptr(), self.col.data_ptr(),
                      None if self.ids is None else self.ids.data_ptr(),
                      None if self.val is None else self.val.data_ptr())


def _stream_ptr(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _adopt_output(al: _TorchAlloc, C: hs_mat) -> DeviceCSR:
    torch = _torch()
    dt = DTYPE_NAME[C.dtype]
    rowptr = al.adopt(C.ptr, C.m + 1, torch.int64)
    col = al.adopt(C.idx, C.nnz, torch.int32)
    val = None
    if dt != "bool":
        tdt = {"f64": torch.float64, "f32": torch.float32, "i32": torch.int32, "i64": torch.int64}[dt]
        val = al.adopt(C.val, C.nnz, tdt) if C.val else torch.empty(0, dtype=tdt, device=rowptr.device)
    return DeviceCSR(C.m, C.n, rowptr, col, val, dt)


def _device_of(A: DeviceCSR):
    return A.rowptr.device


# -------------------------------------------------------------- operations
def spgemm(semiring: str, A: DeviceCSR, B: DeviceCSR, validate: bool = False, stream=None,
           sorted_rows: bool = True, prune_zeros: bool = False) -> DeviceCSR:
    """C = A*B over `semiring` (hs_spgemm).  sorted_rows=False lets rows come out
    in any column order (HS_FLAG_UNSORTED); prune_zeros removes entries whose
    (+,x) sum is exactly zero (HS_FLAG_PRUNE_ZEROS)."""
    L = _lib()
    al = _TorchAlloc(_device_of(A))
    a, b, c = A.desc(), B.desc(), hs_mat()
    fl = ((FLAG_VALIDATE if validate else 0) | (0 if sorted_rows else FLAG_UNSORTED)
          | (FLAG_PRUNE_ZEROS if prune_zeros else 0))
    st = L.hs_spgemm(SEMIRING[semiring], ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                     ctypes.byref(al.struct), _stream_ptr(stream), fl)
    if st != 0:
        raise HsError(st, "hs_spgemm")
    return _adopt_output(al, c)


def spgemm_batched(semiring: str, As: list, Bs: list, validate: bool = False, stream=None):
    """C_i = A_i * B_i for every pair, in one pass (hs_spgemm_batched).

    Returns (C, row_offsets): C is the stacked result (local column ids) and
    problem i owns rows row_offsets[i]..row_offsets[i+1] of it.
    """
    L = _lib()
    count = len(As)
    if count != len(Bs):
        raise ValueError("As and Bs differ in length")
    dev = _device_of(As[0]) if count else _torch().device("cuda")
    al = _TorchAlloc(dev)
    A_arr = (hs_mat * max(count, 1))(*[x.desc() for x in As])
    B_arr = (hs_mat * max(count, 1))(*[x.desc() for x in Bs])
    offs = (ctypes.c_int64 * (count + 1))()
    c = hs_mat()
    st = L.hs_spgemm_batched(SEMIRING[semiring], count, A_arr, B_arr, ctypes.byref(c), offs,
                             ctypes.byref(al.struct), _stream_ptr(stream), FLAG_VALIDATE if validate else 0)
    if st != 0:
        raise HsError(st, "hs_spgemm_batched")
    return _adopt_output(al, c), np.array(offs[:], dtype=np.int64)


class BatchPlan:
    """C_i = A_i * B_i for every pair by one persistent launch per execution
    (hs_batch_plan_*): created once (the problems stacked, C sized by the flop
    bound), then execute() recomputes C with no allocation and no host
    synchronisation (capturable in a CUDA graph); result() returns (C,
    row_offsets) as for spgemm_batched, C's arrays owned by the plan."""

    def __init__(self, semiring: str, As: list, Bs: list, stream=None):
        L = _lib()
        self.count = len(As)
        if self.count != len(Bs):
            raise ValueError("As and Bs differ in length")
        dev = _device_of(As[0]) if self.count else _torch().device("cuda")
        self._al = _TorchAlloc(dev)
        A_arr = (hs_mat * max(self.count, 1))(*[x.desc() for x in As])
        B_arr = (hs_mat * max(self.count, 1))(*[x.desc() for x in Bs])
        h = ctypes.c_void_p()
        st = L.hs_batch_plan_create(SEMIRING[semiring], self.count, A_arr, B_arr, ctypes.byref(h),
                                    ctypes.byref(self._al.struct), _stream_ptr(stream), 0)
        if st != 0:
            raise HsError(st, "hs_batch_plan_create")
        self._h = h

    def execute(self, stream=None):
        st = _lib().hs_batch_plan_execute(self._h, _stream_ptr(stream))
        if st != 0:
            raise HsError(st, "hs_batch_plan_execute")

    def result(self, stream=None):
        """(C, row_offsets) of the last execution (synchronises; C views the plan's arrays)."""
        torch = _torch()
        c = hs_mat()
        offs = (ctypes.c_int64 * (self.count + 1))()
        st = _lib().hs_batch_plan_result(self._h, ctypes.byref(c), offs, _stream_ptr(stream))
        if st != 0:
            raise HsError(st, "hs_batch_plan_result")
        live = self._al.live
        nnz = int(c.nnz)
        rowptr = live[int(c.ptr)].view(torch.int64)[:c.m + 1]
        col = live[int(c.idx)].view(torch.int32)[:nnz]
        tdt = {"f64": torch.float64, "f32": torch.float32, "i32": torch.int32, "i64": torch.int64}
        dt = DTYPE_NAME[c.dtype]
        val = live[int(c.val)].view(tdt[dt])[:nnz] if c.val else None
        return DeviceCSR(c.m, c.n, rowptr, col, val, dt), np.array(offs[:], dtype=np.int64)

    def phase_ms(self, stream=None) -> dict:
        """The last execution's phase times (hs_batch_plan_phase_ms), in ms."""
        ms = (ctypes.c_double * 5)()
        st = _lib().hs_batch_plan_phase_ms(self._h, ms, _stream_ptr(stream))
        if st != 0:
            raise HsError(st, "hs_batch_plan_phase_ms")
        return dict(zip(("products", "symbolic", "offsets", "values", "kernel"), ms[:]))

    def close(self, stream=None):
        if self._h is not None:
            _lib().hs_batch_plan_destroy(self._h, _stream_ptr(stream))
            self._h = None


FLAG_STAGE_ON_DEVICE = 2
FLAG_UNSORTED = 4
FLAG_PRUNE_ZEROS = 8


def spgemm_to_host(semiring: str, A: DeviceCSR, B: DeviceCSR, rowptr, col, val, blocks: int = 8,
                   validate: bool = False, stage_on_device: bool = False, stream=None) -> int:
    """C = A*B written into host tensors rowptr (A.m+1 int64), col (int32) and
    val (C's dtype; None for bool), best pinned, with each row block's copy
    overlapped with the next block's product (hs_spgemm_to_host).  Returns
    nnz(C); raises HsError with .nnz_needed if the arrays are too small."""
    L = _lib()
    a, b = A.desc(), B.desc()
    nnz = ctypes.c_int64(0)
    cap = int(col.numel())
    st = L.hs_spgemm_to_host(SEMIRING[semiring], ctypes.byref(a), ctypes.byref(b), int(blocks), rowptr.data_ptr(),
                             col.data_ptr(), None if val is None else val.data_ptr(), cap, ctypes.byref(nnz),
                             _stream_ptr(stream), (FLAG_VALIDATE if validate else 0)
                             | (FLAG_STAGE_ON_DEVICE if stage_on_device else 0))
    if st != 0:
        e = HsError(st, "hs_spgemm_to_host")
        e.nnz_needed = int(nnz.value)
        raise e
    return int(nnz.value)


def trim_memory():
    """Return the memory the library's own pool keeps (hs_trim_memory)."""
    st = _lib().hs_trim_memory()
    if st != 0:
        raise HsError(st, "hs_trim_memory")


def batch_stack(As: list, Bs: list, stream=None):
    """The stacked operands (SA, SB, row_offsets) of a batch (hs_batch_stack):
    SA*SB is the block-diagonal product whose rows row_offsets[i]..[i+1] are A_i*B_i."""
    L = _lib()
    count = len(As)
    if count != len(Bs):
        raise ValueError("As and Bs differ in length")
    dev = _device_of(As[0]) if count else _torch().device("cuda")
    al = _TorchAlloc(dev)
    A_arr = (hs_mat * max(count, 1))(*[x.desc() for x in As])
    B_arr = (hs_mat * max(count, 1))(*[x.desc() for x in Bs])
    offs = (ctypes.c_int64 * (count + 1))()
    sa, sb = hs_mat(), hs_mat()
    st = L.hs_batch_stack(count, A_arr, B_arr, ctypes.byref(sa), ctypes.byref(sb), offs, ctypes.byref(al.struct),
                          _stream_ptr(stream))
    if st != 0:
        raise HsError(st, "hs_batch_stack")
    return _adopt_output(al, sa), _adopt_output(al, sb), np.array(offs[:], dtype=np.int64)


class Plan:
    """C = A*B computed once (hs_plan_create), then its values recomputed from
    new values of A and B on the same structures (hs_plan_execute: no
    allocation, no host synchronisation, so it can be captured in a CUDA
    graph).  Keeps A, B and C alive while it is open."""

    def __init__(self, semiring: str, A: DeviceCSR, B: DeviceCSR, validate: bool = False, stream=None):
        L = _lib()
        self._al = _TorchAlloc(_device_of(A))
        self.A, self.B = A, B
        a, b, c = A.desc(), B.desc(), hs_mat()
        h = ctypes.c_void_p()
        st = L.hs_plan_create(SEMIRING[semiring], ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(h),
                              ctypes.byref(self._al.struct), _stream_ptr(stream), FLAG_VALIDATE if validate else 0)
        if st != 0:
            raise HsError(st, "hs_plan_create")
        self._h = h
        self.C = _adopt_output(self._al, c)

    def execute(self, A_val=None, B_val=None, C_val=None, stream=None):
        """Recompute C's values (into C_val, default C.val) from A_val, B_val (default: A's and B's arrays)."""
        if self._h is None:
            raise RuntimeError("plan is closed")
        av = self.A.val if A_val is None else A_val
        bv = self.B.val if B_val is None else B_val
        cv = self.C.val if C_val is None else C_val
        st = _lib().hs_plan_execute(self._h, None if av is None else av.data_ptr(),
                                    None if bv is None else bv.data_ptr(), None if cv is None else cv.data_ptr(),
                                    _stream_ptr(stream))
        if st != 0:
            raise HsError(st, "hs_plan_execute")

    def status(self, stream=None):
        """Raise if a device-side check failed during the executes so far (synchronises)."""
        st = _lib().hs_plan_status(self._h, _stream_ptr(stream))
        if st != 0:
            raise HsError(st, "hs_plan_status")

    def close(self, stream=None):
        if self._h is not None:
            _lib().hs_plan_destroy(self._h, _stream_ptr(stream))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def csr_rows(C: DeviceCSR, r0: int, r1: int, n: int | None = None) -> DeviceCSR:
    """Rows r0..r1-1 of C as a CSR of their own (rebased offsets; copies the offsets only)."""
    rp = C.rowptr[r0:r1 + 1]
    a, b = int(rp[0]), int(rp[-1])
    return DeviceCSR(r1 - r0, C.n if n is None else n, rp - a, C.col[a:b],
                     None if C.val is None else C.val[a:b], C.dtype)


def spgemm_noalloc(semiring: str, A: DeviceCSR, B: DeviceCSR, capacity: int, stream=None) -> DeviceCSR:
    """C = A*B through hs_spgemm_noalloc: the library allocates nothing.

    The output arrays are allocated here, by the caller (torch), with room
    for `capacity` entries; the library takes every temporary from its fixed
    scratch array.  Raises HsError (HS_ECAPACITY, with .nnz_needed) when
    nnz(C) exceeds capacity.
    """
    torch = _torch()
    L = _lib()
    dev = _device_of(A)
    out_dt = "bool" if semiring == "or_and" else (B.dtype if semiring == "select2nd" else A.dtype)
    tdt = {"f64": torch.float64, "f32": torch.float32, "i32": torch.int32, "i64": torch.int64}.get(out_dt)
    rowptr = torch.empty(A.m + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    val = None if tdt is None else torch.empty(max(capacity, 1), dtype=tdt, device=dev)
    a, b = A.desc(), B.desc()
    c = hs_mat(0, 0, 0, 0, 0, 0, rowptr.data_ptr(), col.data_ptr(), None,
               None if val is None else val.data_ptr())
    st = L.hs_spgemm_noalloc(SEMIRING[semiring], ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                             int(capacity), _stream_ptr(stream))
    if st != 0:
        err = HsError(st, "hs_spgemm_noalloc")
        err.nnz_needed = int(c.nnz)
        raise err
    nnz = int(c.nnz)
    return DeviceCSR(c.m, c.n, rowptr, col[:nnz], None if val is None else val[:nnz], DTYPE_NAME[c.dtype])


def _idx(x, device):
    torch = _torch()
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.int32).contiguous()
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.int32))).to(device)


def spref(A: DeviceCSR, I, J, validate: bool = False, stream=None) -> DeviceCSR:
    """B = A(I, J) (hs_spref)."""
    L = _lib()
    dev = _device_of(A)
    It, Jt = _idx(I, dev), _idx(J, dev)
    al = _TorchAlloc(dev)
    a, b = A.desc(), hs_mat()
    st = L.hs_spref(ctypes.byref(a), It.data_ptr() if It.numel() else None, It.numel(),
                    Jt.data_ptr() if Jt.numel() else None, Jt.numel(), ctypes.byref(b),
                    ctypes.byref(al.struct), _stream_ptr(stream), FLAG_VALIDATE if validate else 0)
    if st != 0:
        raise HsError(st, "hs_spref")
    return _adopt_output(al, b)


def spasgn(A: DeviceCSR, I, J, B: DeviceCSR, accumulate: bool = False, add: str = "plus_times",
           validate: bool = False, stream=None) -> DeviceCSR:
    """C = A with A(I,J) = B, or A(I,J) += B with accumulate (hs_spasgn)."""
    L = _lib()
    dev = _device_of(A)
    It, Jt = _idx(I, dev), _idx(J, dev)
    al = _TorchAlloc(dev)
    a, b, c = A.desc(), B.desc(), hs_mat()
    st = L.hs_spasgn(ctypes.byref(a), It.data_ptr() if It.numel() else None, It.numel(),
                     Jt.data_ptr() if Jt.numel() else None, Jt.numel(), ctypes.byref(b), int(accumulate),
                     SEMIRING[add], ctypes.byref(c), ctypes.byref(al.struct), _stream_ptr(stream),
                     FLAG_VALIDATE if validate else 0)
    if st != 0:
        raise HsError(st, "hs_spasgn")
    return _adopt_output(al, c)



def sparse(i, j, v, m: int, n: int, add: str = "plus_times", dtype: str | None = None, stream=None,
           device=None) -> DeviceCSR:
    """C = sparse(i, j, v, m, n) with repeated positions combined by add's add (hs_sparse).

    i, j: index arrays (host or device); v: values (None for bool).  dtype
    defaults to v's type ("bool" when v is None)."""
    torch = _torch()
    L = _lib()
    if device is None:
        device = next((x.device for x in (i, j, v) if isinstance(x, torch.Tensor) and x.is_cuda), "cuda")
    It, Jt = _idx(i, device), _idx(j, device)
    if It.numel() != Jt.numel():
        raise ValueError("i and j differ in length")
    if dtype is None:
        if v is None:
            dtype = "bool"
        else:
            vd = v.dtype if isinstance(v, torch.Tensor) else np.asarray(v).dtype
            dtype = {torch.float64: "f64", torch.float32: "f32", torch.int32: "i32", torch.int64: "i64",
                     np.dtype(np.float64): "f64", np.dtype(np.float32): "f32", np.dtype(np.int32): "i32",
                     np.dtype(np.int64): "i64"}[vd]
    Vt = None
    if dtype != "bool":
        tdt = {"f64": torch.float64, "f32": torch.float32, "i32": torch.int32, "i64": torch.int64}[dtype]
        Vt = (v.to(device=device, dtype=tdt) if isinstance(v, torch.Tensor)
              else torch.from_numpy(np.ascontiguousarray(np.asarray(v), dtype=I_NP[dtype])).to(device)).contiguous()
        if Vt.numel() != It.numel():
            raise ValueError("v differs in length")
    al = _TorchAlloc(torch.device(device))
    c = hs_mat()
    nnz = It.numel()
    st = L.hs_sparse(It.data_ptr() if nnz else None, Jt.data_ptr() if nnz else None,
                     Vt.data_ptr() if (Vt is not None and nnz) else None, nnz, int(m), int(n), DTYPE[dtype],
                     SEMIRING[add], ctypes.byref(c), ctypes.byref(al.struct), _stream_ptr(stream), 0)
    if st != 0:
        raise HsError(st, "hs_sparse")
    return _adopt_output(al, c)

# --------------------------------------------------------------- profiling
def set_tuning(tuning: dict | None = None):
    """Row-bin thresholds (hs_set_tuning); None restores the defaults.  Keys
    not given keep their current values."""
    L = _lib()
    if tuning is None:
        L.hs_set_tuning(None)
        return
    cur = get_tuning()
    cur.update(tuning)
    t = hs_tuning(*[int(cur[k]) for k in TUNING_FIELDS])
    L.hs_set_tuning(ctypes.byref(t))


def get_tuning() -> dict:
    t = hs_tuning()
    _lib().hs_get_tuning(ctypes.byref(t))
    return {k: int(getattr(t, k)) for k in TUNING_FIELDS}


def profile_enable(on: bool = True):
    _lib().hs_profile_enable(1 if on else 0)


def profile_reset():
    _lib().hs_profile_reset()


def profile_read() -> dict:
    """{phase: (total ms, launches)} accumulated since the last reset."""
    L = _lib()
    cap = 64
    ms = (ctypes.c_double * cap)()
    ln = (ctypes.c_int64 * cap)()
    nm = (ctypes.c_char_p * cap)()
    n = L.hs_profile_read(ms, ln, nm, cap)
    return {nm[i].decode(): (ms[i], ln[i]) for i in range(min(n, cap))}


def version() -> int:
    return _lib().hs_version()


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(_lib().hs_launch_count())

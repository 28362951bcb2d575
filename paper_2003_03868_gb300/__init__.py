"""GB300 block-sparse sign-matrix library: thin Python binding of the C ABI.

Every operation runs in the CUDA library ``libdbcsr_gb.so`` (hand-written
sm_103a kernels); this module only marshals arguments.  There is no CPU path:
if the library is missing or no GPU is present the calls raise.

Names follow the C ABI (include/dbcsr_gb.h): ``Matrix`` wraps a
``dbcsr_matrix`` handle; ``multiply``, ``filter``, ``trace``,
``trace_product``, ``gershgorin`` and ``sign_iterate`` map one to one.
"""
from __future__ import annotations

import ctypes as C
import dataclasses

import numpy as np

from . import _ffi
from ._ffi import DBCSR_FP64, DBCSR_BF16, DBCSR_MIXED, MultStats, SignOpts, SignReport  # noqa: F401


class DbcsrError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_ffi.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    return _ffi.load()


def _check(st: int, where: str):
    if st != _ffi.DBCSR_OK:
        raise DbcsrError(st, where, (lib().dbcsr_last_error() or b"").decode())


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def current_stream() -> int:
    """Handle of torch's current CUDA stream (0 = legacy default stream if torch has no GPU)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


class Matrix:
    """A square block-sparse matrix (block-CSR, FP64) owned by the library."""

    def __init__(self, blk_size, stream: int | None = None):
        bs = np.ascontiguousarray(blk_size, dtype=np.int32)
        self.blk_size = bs
        self.stream = current_stream() if stream is None else int(stream)
        h = C.c_void_p()
        _check(lib().dbcsr_create(C.byref(h), int(bs.shape[0]), _ptr(bs), C.c_void_p(self.stream)), "create")
        self.handle = h

    @classmethod
    def from_blocks(cls, blk_size, row_ptr, col, data, stream: int | None = None, on_device: bool = False,
                    data_ptr: int | None = None) -> "Matrix":
        """Matrix holding blocks given in block-CSR form (``data`` packed in that order).

        ``data`` is a numpy array (host), or pass ``data_ptr`` (an integer
        address, host or device per ``on_device``) to skip numpy."""
        m = cls(blk_size, stream)
        rp = np.asarray(row_ptr, dtype=np.int64)
        cols = np.ascontiguousarray(col, dtype=np.int32)
        rows = np.ascontiguousarray(np.repeat(np.arange(len(m.blk_size), dtype=np.int32), np.diff(rp)))
        if data_ptr is None:
            data = np.ascontiguousarray(data, dtype=np.float64)
            ptr = _ptr(data)
        else:
            ptr = C.c_void_p(int(data_ptr))
        _check(lib().dbcsr_put_blocks(m.handle, int(cols.shape[0]), _ptr(rows), _ptr(cols), ptr, int(on_device)),
               "put_blocks")
        m.finalize()
        return m

    @classmethod
    def of(cls, bm, stream: int | None = None) -> "Matrix":
        """From any object with blk_size/row_ptr/col/data (the input generator's format)."""
        return cls.from_blocks(bm.blk_size, bm.row_ptr, bm.col, bm.data, stream)

    def put_block(self, row: int, col: int, block):
        b = np.ascontiguousarray(block, dtype=np.float64)
        _check(lib().dbcsr_put_block(self.handle, int(row), int(col), _ptr(b), 0), "put_block")

    def finalize(self):
        _check(lib().dbcsr_finalize(self.handle), "finalize")

    def info(self):
        nb, nz, ne = C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().dbcsr_get_info(self.handle, C.byref(nb), C.byref(nz), C.byref(ne)), "get_info")
        return nb.value, nz.value, ne.value

    @property
    def nnzb(self) -> int:
        return self.info()[1]

    def get_block(self, row: int, col: int):
        m, n = int(self.blk_size[row]), int(self.blk_size[col])
        out = np.empty((m, n))
        present = C.c_int()
        _check(lib().dbcsr_get_block(self.handle, int(row), int(col), _ptr(out), C.byref(present)), "get_block")
        return out if present.value else None

    def export(self):
        """(row_ptr, col, data) numpy copies of the block-CSR arrays."""
        nb, nz, ne = self.info()
        rp = np.empty(nb + 1, dtype=np.int64)
        col = np.empty(nz, dtype=np.int32)
        data = np.empty(ne, dtype=np.float64)
        _check(lib().dbcsr_export(self.handle, _ptr(rp), _ptr(col), _ptr(data)), "export")
        return rp, col, data

    def copy(self) -> "Matrix":
        out = Matrix(self.blk_size, self.stream)
        _check(lib().dbcsr_copy(out.handle, self.handle), "copy")
        return out

    def scale_shift(self, scale: float, shift: float = 0.0):
        _check(lib().dbcsr_scale_shift(self.handle, float(scale), float(shift)), "scale_shift")

    def filter(self, eps: float):
        _check(lib().dbcsr_filter(self.handle, float(eps)), "filter")

    def trace(self) -> float:
        return trace(self)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().dbcsr_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def multiply(alpha: float, A: Matrix, B: Matrix, beta: float, C_: Matrix, eps_filter: float = 0.0,
             prec: int = DBCSR_FP64, stats: bool = True):
    """C = beta*C + alpha*A*B, then the eps_filter truncation.  Returns MultStats (or None)."""
    st = MultStats() if stats else None
    _check(lib().dbcsr_multiply(float(alpha), A.handle, B.handle, float(beta), C_.handle, float(eps_filter),
                                int(prec), C.byref(st) if stats else None), "multiply")
    return st


def filter(M: Matrix, eps: float):  # noqa: A001 - the C ABI's name
    M.filter(eps)


def trace(M: Matrix) -> float:
    out = C.c_double()
    _check(lib().dbcsr_trace(M.handle, C.byref(out)), "trace")
    return out.value


def trace_product(A: Matrix, B: Matrix) -> float:
    out = C.c_double()
    _check(lib().dbcsr_trace_product(A.handle, B.handle, C.byref(out)), "trace_product")
    return out.value


def trace_product_noalloc(A: Matrix, B: Matrix, out_dev_ptr: int) -> None:
    """Queues Tr(A*B) into the caller's device double at ``out_dev_ptr`` without any
    device allocation (see dbcsr_trace_product_noalloc); does not synchronise."""
    _check(lib().dbcsr_trace_product_noalloc(A.handle, B.handle, C.c_void_p(int(out_dev_ptr))),
           "trace_product_noalloc")


def gershgorin(M: Matrix, mu: float = 0.0) -> float:
    out = C.c_double()
    _check(lib().dbcsr_gershgorin(M.handle, float(mu), C.byref(out)), "gershgorin")
    return out.value


@dataclasses.dataclass
class SignResult:
    P: Matrix
    report: SignReport
    status: int

    @property
    def converged(self) -> bool:
        return bool(self.report.converged)

    @property
    def residuals(self):
        n = min(self.report.iterations, _ffi.MAX_HISTORY)
        return [self.report.residual_history[i] for i in range(n)]


def sign_iterate(H: Matrix, mu: float, eps_filter: float, tol: float, max_iter: int = 100,
                 prec: int = DBCSR_FP64, switch_tol: float = 1e-4, stall_ratio: float = 0.5,
                 P: Matrix | None = None, verbose: bool = False, raise_on_notconv: bool = False) -> SignResult:
    """Density matrix P = (1 - sign(H - mu 1)) / 2 by the Newton-Schulz iteration."""
    P = Matrix(H.blk_size, H.stream) if P is None else P
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), int(prec), float(switch_tol), float(stall_ratio),
                 1 if verbose else 0, 0)
    rep = SignReport()
    st = lib().dbcsr_sign_iterate(H.handle, float(mu), C.byref(o), P.handle, C.byref(rep))
    if st != _ffi.DBCSR_OK and (st != _ffi.DBCSR_ENOTCONV or raise_on_notconv):
        _check(st, "sign_iterate")
    return SignResult(P=P, report=rep, status=st)


def sign_iterate_batched(Hs, mus, eps_filter: float, tol: float, max_iter: int = 100, prec: int = DBCSR_FP64,
                         switch_tol: float = 1e-4, stall_ratio: float = 0.5, verbose: bool = False):
    """Density matrices of many independent systems in one batch (dbcsr_sign_iterate_batched).

    Returns (list of P matrices, list of SignReport, status)."""
    n = len(Hs)
    Ps = [Matrix(h.blk_size, Hs[0].stream) for h in Hs]
    harr = (C.c_void_p * n)(*[h.handle.value for h in Hs])
    parr = (C.c_void_p * n)(*[p.handle.value for p in Ps])
    mu = np.ascontiguousarray(mus, dtype=np.float64)
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), int(prec), float(switch_tol), float(stall_ratio),
                 1 if verbose else 0, 0)
    reps = (SignReport * n)()
    st = lib().dbcsr_sign_iterate_batched(n, harr, _ptr(mu), C.byref(o), parr, reps)
    if st not in (_ffi.DBCSR_OK, _ffi.DBCSR_ENOTCONV):
        _check(st, "sign_iterate_batched")
    return Ps, list(reps), st

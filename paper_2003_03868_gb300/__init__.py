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
import os

import numpy as np

from . import _ffi
from ._ffi import DBCSR_FP64, DBCSR_BF16, DBCSR_MIXED, DBCSR_BF16X3, MultStats, SignOpts, SignReport  # noqa: F401
from ._ffi import DBCSR_TF32, DBCSR_TF32X3  # noqa: F401
from ._ffi import KernelCfg, TuneRecord, MlpOpts, MlpReport, MLP_FEATURES  # noqa: F401


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
    def from_pinned(cls, blk_size, rows_ptr: int, cols_ptr: int, nblocks: int, data_ptr: int,
                    stream: int | None = None) -> "Matrix":
        """Matrix from host buffers given by address (block rows and columns as int32, values
        packed block after block, row-major): one dbcsr_put_blocks and dbcsr_finalize, with no
        copy through numpy.  Pinned host buffers let the upload run at the link's speed."""
        m = cls(blk_size, stream)
        _check(lib().dbcsr_put_blocks(m.handle, int(nblocks), C.c_void_p(int(rows_ptr)), C.c_void_p(int(cols_ptr)),
                                      C.c_void_p(int(data_ptr)), 0), "put_blocks")
        m.finalize()
        return m

    @classmethod
    def of(cls, bm, stream: int | None = None) -> "Matrix":
        """From any object with blk_size/row_ptr/col/data (the input generator's format)."""
        return cls.from_blocks(bm.blk_size, bm.row_ptr, bm.col, bm.data, stream)

    @classmethod
    def load(cls, path: str, stream: int | None = None) -> "Matrix":
        """A finalized matrix read from a file written by save (dbcsr_load)."""
        nblk, _, _ = file_info(path)
        m = cls.__new__(cls)
        m.blk_size = np.fromfile(path, dtype=np.int32, count=nblk, offset=32)
        m.stream = current_stream() if stream is None else int(stream)
        h = C.c_void_p()
        _check(lib().dbcsr_load(C.byref(h), os.fsencode(path), C.c_void_p(m.stream)), "load")
        m.handle = h
        return m

    def save(self, path: str):
        """Writes the matrix to a file (dbcsr_save; layout in dbcsr_gb.h)."""
        _check(lib().dbcsr_save(self.handle, os.fsencode(path)), "save")

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

    def groups(self):
        """The tensor-core tier's block groups for this matrix (dbcsr_matrix_groups): the group
        of every block row and the FP64 block norms they were formed from."""
        nb, nz, _ = self.info()
        g_of = np.empty(nb, dtype=np.int32)
        norms = np.empty(max(nz, 1), dtype=np.float64)
        ng = C.c_int32()
        _check(lib().dbcsr_matrix_groups(self.handle, _ptr(g_of), _ptr(norms), C.byref(ng)), "matrix_groups")
        return g_of, norms[:nz], ng.value

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

    def export_to(self, rp_ptr: int, col_ptr: int, col_cap: int, data_ptr: int, data_cap: int) -> int:
        """dbcsr_export into host buffers given by address (row pointers: nblk + 1 int64; block
        columns: int32, room for col_cap; values: float64, room for data_cap).  Returns the bytes
        copied; raises ValueError when the matrix does not fit."""
        nb, nz, ne = self.info()
        if nz > col_cap or ne > data_cap:
            raise ValueError(f"export_to: {nz} blocks / {ne} values exceed the buffers ({col_cap} / {data_cap})")
        _check(lib().dbcsr_export(self.handle, C.c_void_p(int(rp_ptr)), C.c_void_p(int(col_ptr)),
                                  C.c_void_p(int(data_ptr))), "export")
        return 8 * (nb + 1) + 4 * nz + 8 * ne

    def copy(self) -> "Matrix":
        out = Matrix(self.blk_size, self.stream)
        _check(lib().dbcsr_copy(out.handle, self.handle), "copy")
        return out

    def scale_shift(self, scale: float, shift: float = 0.0):
        _check(lib().dbcsr_scale_shift(self.handle, float(scale), float(shift)), "scale_shift")

    def filter(self, eps: float):
        _check(lib().dbcsr_filter(self.handle, float(eps)), "filter")

    def add(self, other: "Matrix", alpha: float = 1.0, beta: float = 1.0):
        """self <- alpha * self + beta * other on the union of the patterns (dbcsr_add)."""
        add(alpha, self, beta, other)

    def trace(self) -> float:
        return trace(self)

    def put_values(self, data):
        """Replaces every value, keeping the pattern (data in block-CSR order, as export()).

        ``data`` is a numpy float64 array (host) or an int device pointer."""
        if isinstance(data, int):
            _check(lib().dbcsr_put_values(self.handle, C.c_void_p(data), 1), "put_values")
        else:
            d = np.ascontiguousarray(data, dtype=np.float64)
            _check(lib().dbcsr_put_values(self.handle, _ptr(d), 0), "put_values")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _check(lib().dbcsr_destroy(self.handle), "destroy")
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


class Plan:
    """A planned product C = alpha A B on fixed patterns, replayed as one CUDA graph
    (dbcsr_multiply_plan / dbcsr_multiply_execute).  Holds its matrices alive."""

    def __init__(self, alpha: float, A: Matrix, B: Matrix, C_: Matrix, eps_filter: float = 0.0,
                 prec: int = DBCSR_FP64):
        self.A, self.B, self.C = A, B, C_
        self.handle = C.c_void_p()
        self.stats = MultStats()
        _check(lib().dbcsr_multiply_plan(float(alpha), A.handle, B.handle, C_.handle, float(eps_filter), int(prec),
                                         C.byref(self.handle), C.byref(self.stats)), "multiply_plan")

    def execute(self):
        _check(lib().dbcsr_multiply_execute(self.handle), "multiply_execute")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().dbcsr_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def file_info(path: str):
    """(nblk, nnzb, nel) of a matrix file, read and checked on the host (dbcsr_file_info)."""
    nb, nz, ne = C.c_int32(), C.c_int64(), C.c_int64()
    _check(lib().dbcsr_file_info(os.fsencode(path), C.byref(nb), C.byref(nz), C.byref(ne)), "file_info")
    return nb.value, nz.value, ne.value


def filter(M: Matrix, eps: float):  # noqa: A001 - the C ABI's name
    M.filter(eps)


def add(alpha: float, A: Matrix, beta: float, B: Matrix):
    """A <- alpha * A + beta * B on the union of the patterns, no filtering (dbcsr_add)."""
    _check(lib().dbcsr_add(float(alpha), A.handle, float(beta), B.handle), "add")


def trace(M: Matrix) -> float:
    out = C.c_double()
    _check(lib().dbcsr_trace(M.handle, C.byref(out)), "trace")
    return out.value


def trace_product(A: Matrix, B: Matrix) -> float:
    out = C.c_double()
    _check(lib().dbcsr_trace_product(A.handle, B.handle, C.byref(out)), "trace_product")
    return out.value


def pool_usage(reset_high: bool = False) -> tuple[int, int]:
    """Bytes of the library's device memory pool in use now and at most since the last reset
    (dbcsr_pool_usage); reset_high restarts the high-water mark afterwards."""
    now, high = C.c_int64(), C.c_int64()
    _check(lib().dbcsr_pool_usage(C.byref(now), C.byref(high), 1 if reset_high else 0), "pool_usage")
    return int(now.value), int(high.value)


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

    def log_jsonl(self, path: str, low_tier: str = "bf16x3") -> None:
        """Appends the iteration's log to a JSON-lines file: one record per step (step k,
        the tier of its X*X product, residual r_k = ||X_k^2 - 1||_F / N, blocks of X after
        the step) and a closing record with the totals of the report."""
        write_sign_log(self.report, path, low_tier)


def write_sign_log(rep, path: str, low_tier: str = "bf16x3") -> None:
    """The per-step log of a dbcsr_sign_report (see SignResult.log_jsonl)."""
    import json
    n = min(int(rep.iterations), _ffi.MAX_HISTORY)
    f64 = int(rep.fp64_from)
    with open(path, "a") as fh:
        for i in range(n):
            k = i + 1
            tier = "fp64" if (f64 and k >= f64) else low_tier
            fh.write(json.dumps({"step": k, "tier": tier, "residual": float(rep.residual_history[i]),
                                 "nnzb_x": int(rep.nnzb_history[i])}) + "\n")
        fh.write(json.dumps({"summary": True, "iterations": int(rep.iterations), "converged": bool(rep.converged),
                             "stalled": bool(rep.stalled), "fp64_from": f64, "residual": float(rep.residual),
                             "trace_p": float(rep.trace_p), "e_band": float(rep.e_band),
                             "flops": float(rep.flops), "flops_low": float(rep.flops_low),
                             "ms_total": float(rep.ms_total), "ms_multiply": float(rep.ms_multiply),
                             "ms_low": float(rep.ms_low), "ms_symbolic": float(rep.ms_symbolic),
                             "ms_filter": float(rep.ms_filter)}) + "\n")


def _sign_flags(full_products: bool, low: int, low_correction: bool = False, return_x: bool = False) -> int:
    if low not in (DBCSR_BF16, DBCSR_BF16X3):
        raise ValueError("low must be DBCSR_BF16 or DBCSR_BF16X3")
    return ((_ffi.DBCSR_SIGN_FULL_PRODUCTS if full_products else 0)
            | (_ffi.DBCSR_SIGN_PLAIN_BF16 if low == DBCSR_BF16 else 0)
            | (_ffi.DBCSR_SIGN_LOW_CORRECTION if low_correction else 0)
            | (_ffi.DBCSR_SIGN_RETURN_X if return_x else 0))


DBCSR_SCHEDULE_PER_SHAPE, DBCSR_SCHEDULE_QUEUE = 0, 1


def set_fp64_schedule(mode: int) -> None:
    """DBCSR_SCHEDULE_PER_SHAPE (one launch per block shape, tuned) or DBCSR_SCHEDULE_QUEUE (one
    work-queue launch per product) for the FP64 block products (dbcsr_set_fp64_schedule)."""
    _check(lib().dbcsr_set_fp64_schedule(int(mode)), "set_fp64_schedule")


def fp64_schedule() -> int:
    return int(lib().dbcsr_get_fp64_schedule())


def dense_multiply(prec: int, nb: int, n: int, alpha: float, A_ptr: int, B_ptr: int, beta: float, C_ptr: int,
                   stream: int | None = None) -> None:
    """C[b] = alpha A[b] B[b] + beta C[b] for nb row-major n x n matrices in device memory, given
    by address (dbcsr_dense_multiply; double data for DBCSR_FP64, float for DBCSR_TF32 / TF32X3)."""
    s = current_stream() if stream is None else int(stream)
    _check(lib().dbcsr_dense_multiply(int(prec), int(nb), int(n), float(alpha), C.c_void_p(int(A_ptr)),
                                      C.c_void_p(int(B_ptr)), float(beta), C.c_void_p(int(C_ptr)), C.c_void_p(s)),
           "dense_multiply")


def pool_trim(keep_bytes: int = 0) -> None:
    """Return the library's cached device memory above keep_bytes to the driver."""
    _check(lib().dbcsr_pool_trim(int(keep_bytes)), "pool_trim")


def sign_iterate(H: Matrix, mu: float, eps_filter: float, tol: float, max_iter: int = 100,
                 prec: int = DBCSR_FP64, switch_tol: float = 1e-4, stall_ratio: float = 0.5,
                 P: Matrix | None = None, verbose: bool = False, raise_on_notconv: bool = False,
                 full_products: bool = False, low: int = DBCSR_BF16X3, low_correction: bool = False,
                 order: int = 2, return_x: bool = False) -> SignResult:
    """Density matrix P = (1 - sign(H - mu 1)) / 2 by the sign iteration of the given order
    (2: Newton-Schulz; 3 to 7: the polynomial Pade steps, see dbcsr_sign_iterate).

    With prec=DBCSR_MIXED, `low` picks the product of the low-precision tier:
    the split DBCSR_BF16X3 (default) or plain DBCSR_BF16; low_correction takes the
    FP64 tier's update correction X (X^2 - 1) in split BF16 (DBCSR_SIGN_LOW_CORRECTION).
    return_x: the result holds the iteration's X instead of P (a checkpoint for
    sign_iterate_resume, DBCSR_SIGN_RETURN_X)."""
    P = Matrix(H.blk_size, H.stream) if P is None else P
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), int(prec), float(switch_tol), float(stall_ratio),
                 1 if verbose else 0, _sign_flags(full_products, low, low_correction, return_x), int(order), 0)
    rep = SignReport()
    st = lib().dbcsr_sign_iterate(H.handle, float(mu), C.byref(o), P.handle, C.byref(rep))
    if st != _ffi.DBCSR_OK and (st != _ffi.DBCSR_ENOTCONV or raise_on_notconv):
        _check(st, "sign_iterate")
    return SignResult(P=P, report=rep, status=st)


def sign_iterate_resume(H: Matrix, X: Matrix, prev: SignReport, eps_filter: float, tol: float,
                        max_iter: int = 100, prec: int = DBCSR_FP64, switch_tol: float = 1e-4,
                        stall_ratio: float = 0.5, P: Matrix | None = None, verbose: bool = False,
                        raise_on_notconv: bool = False, full_products: bool = False, low: int = DBCSR_BF16X3,
                        low_correction: bool = False, order: int = 2, return_x: bool = False) -> SignResult:
    """Continue a sign iteration from its checkpoint: X (a run with return_x=True that
    max_iter stopped, perhaps saved and loaded) and that run's report (dbcsr_sign_iterate_resume).
    The options are those of the first run; max_iter counts every step."""
    P = Matrix(H.blk_size, H.stream) if P is None else P
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), int(prec), float(switch_tol), float(stall_ratio),
                 1 if verbose else 0, _sign_flags(full_products, low, low_correction, return_x), int(order), 0)
    rep = SignReport()
    st = lib().dbcsr_sign_iterate_resume(H.handle, X.handle, C.byref(prev), C.byref(o), P.handle, C.byref(rep))
    if st != _ffi.DBCSR_OK and (st != _ffi.DBCSR_ENOTCONV or raise_on_notconv):
        _check(st, "sign_iterate_resume")
    return SignResult(P=P, report=rep, status=st)


@dataclasses.dataclass
class SqrtResult:
    Sinvsqrt: Matrix
    Ssqrt: Matrix | None
    report: SignReport
    status: int

    @property
    def converged(self) -> bool:
        return bool(self.report.converged)

    @property
    def residuals(self):
        return [self.report.residual_history[i] for i in range(min(self.report.iterations, _ffi.MAX_HISTORY))]


def inverse_sqrt(S: Matrix, eps_filter: float, tol: float, max_iter: int = 100, prec: int = DBCSR_FP64,
                 switch_tol: float = 1e-4, stall_ratio: float = 0.5, order: int = 2, full_products: bool = False,
                 low: int = DBCSR_BF16X3, want_sqrt: bool = True, verbose: bool = False,
                 raise_on_notconv: bool = False) -> SqrtResult:
    """S^(-1/2) (and S^(1/2)) by the sign iteration on [[0, S], [1, 0]] (dbcsr_inverse_sqrt)."""
    Zi = Matrix(S.blk_size, S.stream)
    Ys = Matrix(S.blk_size, S.stream) if want_sqrt else None
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), int(prec), float(switch_tol), float(stall_ratio),
                 1 if verbose else 0, _sign_flags(full_products, low, False), int(order), 0)
    rep = SignReport()
    st = lib().dbcsr_inverse_sqrt(S.handle, C.byref(o), Zi.handle, Ys.handle if Ys else None, C.byref(rep))
    if st != _ffi.DBCSR_OK and (st != _ffi.DBCSR_ENOTCONV or raise_on_notconv):
        _check(st, "inverse_sqrt")
    return SqrtResult(Sinvsqrt=Zi, Ssqrt=Ys, report=rep, status=st)


def inverse_hotelling(A: Matrix, eps_filter: float, tol: float, max_iter: int = 100, full_products: bool = False,
                      verbose: bool = False, raise_on_notconv: bool = False) -> SignResult:
    """A^-1 by Hotelling's iteration X <- X (2 - A X) (dbcsr_inverse_hotelling); the result is
    in .P."""
    Ai = Matrix(A.blk_size, A.stream)
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), DBCSR_FP64, 0.0, 0.5, 1 if verbose else 0,
                 _sign_flags(full_products, DBCSR_BF16X3, False), 0, 0)
    rep = SignReport()
    st = lib().dbcsr_inverse_hotelling(A.handle, C.byref(o), Ai.handle, C.byref(rep))
    if st != _ffi.DBCSR_OK and (st != _ffi.DBCSR_ENOTCONV or raise_on_notconv):
        _check(st, "inverse_hotelling")
    return SignResult(P=Ai, report=rep, status=st)


@dataclasses.dataclass
class NonorthResult:
    P: Matrix
    report: SignReport          # the sign iteration on S^-1/2 K S^-1/2; trace_p = Tr(P S), e_band = Tr(P K)
    report_sqrt: SignReport     # the square root of S
    status: int

    @property
    def converged(self) -> bool:
        return bool(self.report.converged) and bool(self.report_sqrt.converged)


def sign_iterate_nonorth(K: Matrix, S: Matrix, mu: float, eps_filter: float, tol: float, max_iter: int = 100,
                         prec: int = DBCSR_FP64, switch_tol: float = 1e-4, stall_ratio: float = 0.5, order: int = 2,
                         full_products: bool = False, low: int = DBCSR_BF16X3, low_correction: bool = False,
                         P: Matrix | None = None, verbose: bool = False,
                         raise_on_notconv: bool = False) -> NonorthResult:
    """P = (1 - sign(S^-1 K - mu 1)) S^-1 / 2 (dbcsr_sign_iterate_nonorth)."""
    P = Matrix(K.blk_size, K.stream) if P is None else P
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), int(prec), float(switch_tol), float(stall_ratio),
                 1 if verbose else 0, _sign_flags(full_products, low, low_correction), int(order), 0)
    rep, reps = SignReport(), SignReport()
    st = lib().dbcsr_sign_iterate_nonorth(K.handle, S.handle, float(mu), C.byref(o), P.handle, C.byref(rep),
                                          C.byref(reps))
    if st != _ffi.DBCSR_OK and (st != _ffi.DBCSR_ENOTCONV or raise_on_notconv):
        _check(st, "sign_iterate_nonorth")
    return NonorthResult(P=P, report=rep, report_sqrt=reps, status=st)


def submatrix_sign(H: Matrix, mu: float, tol: float, max_iter: int = 100, prec: int = DBCSR_FP64,
                   switch_tol: float = 1e-3, P: Matrix | None = None, verbose: bool = False,
                   raise_on_notconv: bool = False) -> SignResult:
    """P by the submatrix method: dense sign of every block column's neighbourhood
    (dbcsr_submatrix_sign).  prec=DBCSR_MIXED runs the dense products in FP32 (TF32 tensor
    cores until the residual drops below switch_tol)."""
    P = Matrix(H.blk_size, H.stream) if P is None else P
    o = SignOpts(0.0, float(tol), int(max_iter), int(prec), float(switch_tol), 0.5, 1 if verbose else 0, 0, 0, 0)
    rep = SignReport()
    st = lib().dbcsr_submatrix_sign(H.handle, float(mu), C.byref(o), P.handle, C.byref(rep))
    if st != _ffi.DBCSR_OK and (st != _ffi.DBCSR_ENOTCONV or raise_on_notconv):
        _check(st, "submatrix_sign")
    return SignResult(P=P, report=rep, status=st)


def purify(H: Matrix, n_occ: float, eps_filter: float, tol: float, method: str = "tc2", max_iter: int = 100,
           full_products: bool = False, P: Matrix | None = None, verbose: bool = False,
           raise_on_notconv: bool = False) -> SignResult:
    """Canonical projector on the n_occ lowest states of H by TC2 or TRS4 purification
    (dbcsr_purify).  report.residual_history holds (Tr X - Tr X^2) / N per step."""
    m = {"tc2": _ffi.DBCSR_PURIFY_TC2, "trs4": _ffi.DBCSR_PURIFY_TRS4}[method]
    P = Matrix(H.blk_size, H.stream) if P is None else P
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), DBCSR_FP64, 0.0, 0.0, 1 if verbose else 0,
                 _sign_flags(full_products, DBCSR_BF16X3, False), 0, 0)
    rep = SignReport()
    st = lib().dbcsr_purify(H.handle, float(n_occ), m, C.byref(o), P.handle, C.byref(rep))
    if st != _ffi.DBCSR_OK and (st != _ffi.DBCSR_ENOTCONV or raise_on_notconv):
        _check(st, "purify")
    return SignResult(P=P, report=rep, status=st)


@dataclasses.dataclass
class MuSearchResult:
    P: Matrix
    mu: float
    evaluations: int
    report: SignReport
    status: int


def sign_mu_search(H: Matrix, n_occ: float, eps_filter: float, tol: float, mu_lo: float | None = None,
                   mu_hi: float | None = None, max_iter: int = 100, prec: int = DBCSR_FP64, switch_tol: float = 1e-4,
                   order: int = 2, P: Matrix | None = None, verbose: bool = False,
                   raise_on_notconv: bool = False) -> MuSearchResult:
    """The sign method with mu bisected until Tr P = n_occ within 1/2 (dbcsr_sign_mu_search)."""
    P = Matrix(H.blk_size, H.stream) if P is None else P
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), int(prec), float(switch_tol), 0.5, 1 if verbose else 0,
                 0, int(order), 0)
    rep = SignReport()
    mu = C.c_double()
    ev = C.c_int32()
    lo = float("nan") if mu_lo is None else float(mu_lo)
    hi = float("nan") if mu_hi is None else float(mu_hi)
    st = lib().dbcsr_sign_mu_search(H.handle, float(n_occ), lo, hi, C.byref(o), P.handle, C.byref(mu), C.byref(ev),
                                    C.byref(rep))
    if st != _ffi.DBCSR_OK and (st != _ffi.DBCSR_ENOTCONV or raise_on_notconv):
        _check(st, "sign_mu_search")
    return MuSearchResult(P=P, mu=mu.value, evaluations=ev.value, report=rep, status=st)


def sign_iterate_batched(Hs, mus, eps_filter: float, tol: float, max_iter: int = 100, prec: int = DBCSR_FP64,
                         switch_tol: float = 1e-4, stall_ratio: float = 0.5, verbose: bool = False,
                         low: int = DBCSR_BF16X3, low_correction: bool = False, order: int = 2):
    """Density matrices of many independent systems in one batch (dbcsr_sign_iterate_batched),
    by the sign iteration of the given order.

    Returns (list of P matrices, list of SignReport, status)."""
    n = len(Hs)
    Ps = [Matrix(h.blk_size, Hs[0].stream) for h in Hs]
    harr = (C.c_void_p * n)(*[h.handle.value for h in Hs])
    parr = (C.c_void_p * n)(*[p.handle.value for p in Ps])
    mu = np.ascontiguousarray(mus, dtype=np.float64)
    o = SignOpts(float(eps_filter), float(tol), int(max_iter), int(prec), float(switch_tol), float(stall_ratio),
                 1 if verbose else 0, _sign_flags(False, low, low_correction), int(order), 0)
    reps = (SignReport * n)()
    st = lib().dbcsr_sign_iterate_batched(n, harr, _ptr(mu), C.byref(o), parr, reps)
    if st not in (_ffi.DBCSR_OK, _ffi.DBCSR_ENOTCONV):
        _check(st, "sign_iterate_batched")
    return Ps, list(reps), st


# ------------------------------------------------------------------ autotuner
def tune_space(prec: int = DBCSR_FP64):
    """The launch configurations the autotuner times for ``prec``."""
    n = C.c_int32()
    _check(lib().dbcsr_tune_space(int(prec), None, 0, C.byref(n)), "tune_space")
    arr = (KernelCfg * n.value)()
    _check(lib().dbcsr_tune_space(int(prec), arr, n.value, C.byref(n)), "tune_space")
    return list(arr)


def autotune(triples, prec: int = DBCSR_FP64, stack_len: int = 500000, reps: int = 5):
    """Times every configuration on a synthetic stack per (m, n, k); the fastest
    enters the tune table.  Returns the list of TuneRecord timings."""
    t = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
    cap = t.shape[0] * len(tune_space(prec))
    recs = (TuneRecord * cap)()
    n = C.c_int64()
    _check(lib().dbcsr_autotune(_ptr(t), int(t.shape[0]), int(prec), int(stack_len), int(reps), recs, cap,
                                C.byref(n)), "autotune")
    return list(recs)[:n.value]


def time_configs(m: int, n: int, k: int, cfgs, prec: int = DBCSR_FP64, stack_len: int = 500000, reps: int = 5):
    """Median launch time (ms) of each configuration on the synthetic (m, n, k) stack."""
    arr = (KernelCfg * len(cfgs))(*cfgs)
    out = np.zeros(len(cfgs))
    _check(lib().dbcsr_time_config(int(prec), int(m), int(n), int(k), int(stack_len), int(reps), arr, len(cfgs),
                                   _ptr(out)), "time_config")
    return out


def tune_set(prec: int, m: int, n: int, k: int, cfg):
    _check(lib().dbcsr_tune_set(int(prec), int(m), int(n), int(k), C.byref(cfg) if cfg is not None else None),
           "tune_set")


def tune_get(prec: int, m: int, n: int, k: int):
    """(config, found) of the tune table entry (the default configuration when absent)."""
    c, f = KernelCfg(), C.c_int()
    _check(lib().dbcsr_tune_get(int(prec), int(m), int(n), int(k), C.byref(c), C.byref(f)), "tune_get")
    return c, bool(f.value)


def tune_clear():
    _check(lib().dbcsr_tune_clear(), "tune_clear")


def tune_save(path: str):
    _check(lib().dbcsr_tune_save(path.encode()), "tune_save")


def tune_load(path: str):
    _check(lib().dbcsr_tune_load(path.encode()), "tune_load")


# ------------------------------------------------------------------ prediction model
def mlp_init(nfeat: int = MLP_FEATURES, seed: int = 1):
    p = np.zeros(lib().dbcsr_mlp_param_count(int(nfeat)), dtype=np.float32)
    _check(lib().dbcsr_mlp_init(int(nfeat), int(seed), _ptr(p)), "mlp_init")
    return p


def mlp_features(triples, cfgs, prec: int = DBCSR_FP64):
    """Feature rows of samples (m, n, k, cfg); ``triples`` [n, 3], ``cfgs`` a list of KernelCfg."""
    t = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
    arr = (KernelCfg * len(cfgs))(*cfgs)
    out = np.zeros((t.shape[0], MLP_FEATURES), dtype=np.float32)
    _check(lib().dbcsr_mlp_features(int(prec), _ptr(t), arr, int(t.shape[0]), _ptr(out)), "mlp_features")
    return out


def mlp_forward(params, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    p = np.ascontiguousarray(params, dtype=np.float32)
    y = np.zeros(X.shape[0], dtype=np.float32)
    _check(lib().dbcsr_mlp_forward(int(X.shape[1]), _ptr(p), _ptr(X), int(X.shape[0]), _ptr(y)), "mlp_forward")
    return y


def mlp_loss_grad(params, X, T):
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    p = np.ascontiguousarray(params, dtype=np.float32)
    g = np.zeros_like(p)
    loss = C.c_float()
    _check(lib().dbcsr_mlp_loss_grad(int(X.shape[1]), _ptr(p), _ptr(X), _ptr(T), int(X.shape[0]), C.byref(loss),
                                     _ptr(g)), "mlp_loss_grad")
    return float(loss.value), g


def mlp_train(params, X, T, epochs: int = 2000, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """Trains a copy of ``params`` on the GPU; returns (params, MlpReport)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    p = np.array(params, dtype=np.float32, copy=True)
    o = MlpOpts(int(epochs), 0, float(lr), float(beta1), float(beta2), float(eps))
    r = MlpReport()
    _check(lib().dbcsr_mlp_train(int(X.shape[1]), _ptr(p), _ptr(X), _ptr(T), int(X.shape[0]), C.byref(o),
                                 C.byref(r)), "mlp_train")
    return p, r


def tune_records_save(path: str, recs, append: bool = False):
    """Writes autotuner records (TuneRecord list) to a records file (dbcsr_tune_records_save)."""
    arr = (TuneRecord * len(recs))(*recs)
    _check(lib().dbcsr_tune_records_save(os.fsencode(path), arr, len(recs), 1 if append else 0), "tune_records_save")


def predictor_data(path: str, prec: int = DBCSR_FP64):
    """(X, T): the features and targets dbcsr_predictor_train builds from a records file."""
    n = C.c_int64()
    _check(lib().dbcsr_predictor_data(os.fsencode(path), int(prec), None, None, 0, C.byref(n)), "predictor_data")
    X = np.zeros((n.value, MLP_FEATURES), dtype=np.float32)
    T = np.zeros(n.value, dtype=np.float32)
    _check(lib().dbcsr_predictor_data(os.fsencode(path), int(prec), _ptr(X), _ptr(T), n.value, C.byref(n)),
           "predictor_data")
    return X, T


def predictor_train(path: str, prec: int = DBCSR_FP64, epochs: int = 3000, lr: float = 2e-3, seed: int = 3,
                    beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """Trains the library's prediction model on a records file (dbcsr_predictor_train); the
    library keeps the model for prec.  Returns (params, MlpReport)."""
    o = MlpOpts(int(epochs), 0, float(lr), float(beta1), float(beta2), float(eps))
    r = MlpReport()
    _check(lib().dbcsr_predictor_train(os.fsencode(path), int(prec), int(seed), C.byref(o), C.byref(r)),
           "predictor_train")
    p = np.zeros(lib().dbcsr_mlp_param_count(MLP_FEATURES), dtype=np.float32)
    _check(lib().dbcsr_predictor_params(int(prec), _ptr(p)), "predictor_params")
    return p, r


def train_predictor(recs, prec: int = DBCSR_FP64, epochs: int = 3000, lr: float = 2e-3, seed: int = 3):
    """Trains the prediction model on autotuner records (TuneRecord list) of one precision:
    the records go to a temporary records file and dbcsr_predictor_train builds the targets
    and trains there.  Returns (params, MlpReport)."""
    import tempfile
    fd, path = tempfile.mkstemp(suffix=".tune")
    os.close(fd)
    try:
        tune_records_save(path, recs)
        return predictor_train(path, prec, epochs=epochs, lr=lr, seed=seed)
    finally:
        os.unlink(path)


def tune_predicted(params, triples, prec: int = DBCSR_FP64, stack_len: int = 500000, reps: int = 3,
                   tolerance: float = 0.02):
    """Installs the MLP's configuration for each triple when its measured time is within
    tolerance of the default's, else the exhaustive best (dbcsr_tune_predicted).  Returns
    the per-triple fallback flags.  params=None takes the model the library keeps for prec
    (predictor_train)."""
    t = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    fb = np.zeros(t.shape[0], dtype=np.int32)
    _check(lib().dbcsr_tune_predicted(int(prec), _ptr(p), _ptr(t), int(t.shape[0]), int(stack_len), int(reps),
                                      float(tolerance), _ptr(fb)), "tune_predicted")
    return [bool(x) for x in fb]


def mlp_predict_best(params, triples, prec: int = DBCSR_FP64):
    """Predicted-fastest configuration of every triple (list of KernelCfg); params=None takes
    the model the library keeps for prec (predictor_train)."""
    t = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    best = (KernelCfg * t.shape[0])()
    _check(lib().dbcsr_mlp_predict_best(int(prec), _ptr(p), _ptr(t), int(t.shape[0]), best, None),
           "mlp_predict_best")
    return list(best)

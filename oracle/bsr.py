"""FP64 block-CSR operations of the oracle (TEST INFRASTRUCTURE ONLY).

Follows the paper's DBCSR section: matrices are stored as dense atom blocks in a
blocked CSR format ("DBCSR library"), a product is a sum of small dense block
products ("Local multiplication"), and after every product the blocks whose
magnitude is below eps_filter are flushed to zero (section "Sign-Method").
Readings taken where the paper is silent:

* the filter acts on whole blocks: a block is dropped when its Frobenius norm is
  strictly below eps_filter; diagonal blocks are never dropped;
* C = alpha*A*B + beta*C_in is formed on the union of the patterns of A*B and
  C_in, and filtered afterwards.

The arithmetic runs in ``bsr_oracle.c`` (plain loops, ascending K then k, no FMA);
this module only marshals arrays and does the index bookkeeping of the filter.
Only tests, the smoke check and the benchmark's CPU-baseline leg import it.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        p = C.c_void_p
        L.oracle_mm_count.argtypes = [C.c_int32, p, p, p, p, p, p, p]
        L.oracle_mm_pattern.argtypes = [C.c_int32, p, p, p, p, p, p, p, p]
        L.oracle_mm_numeric.argtypes = [C.c_int32, p, C.c_double] + [p] * 8 + [C.c_double] + [p] * 8 + [p]
        L.oracle_block_norms.argtypes = [C.c_int64, p, p, p, p, p, p, p]
        L.oracle_sum_dev2.argtypes = [C.c_int32, p, p, p, p]
        L.oracle_sum_dev2.restype = C.c_double
        L.oracle_trace.argtypes = [C.c_int32, p, p, p, p, p]
        L.oracle_trace.restype = C.c_double
        L.oracle_trace_product.argtypes = [C.c_int32, p] + [p] * 8
        L.oracle_trace_product.restype = C.c_double
        L.oracle_abs_row_sums.argtypes = [C.c_int32, p, p, p, p, p, p, C.c_double, p]
        L.oracle_num_threads.restype = C.c_int
        L.oracle_prescreen.argtypes = [C.c_int32, C.c_double, p, p, p, p, p, p, C.c_double, p, p, p, p, p,
                                       C.c_double, p]
        L.oracle_prescreen.restype = C.c_int
        L.oracle_set_num_threads.argtypes = [C.c_int]
        L.oracle_set_num_threads.restype = None
        L.oracle_mm_block.argtypes = [C.c_int32, C.c_int32, p, C.c_double] + [p] * 8 + [C.c_double, p, p]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


@dataclasses.dataclass
class Mat:
    """Square block matrix in block-CSR form (the oracle's own copy of the arrays)."""

    bs: np.ndarray      # int32 [nblk]
    rp: np.ndarray      # int64 [nblk + 1]
    col: np.ndarray     # int32 [nnzb]
    data: np.ndarray    # float64

    def __post_init__(self):
        self.bs = np.ascontiguousarray(self.bs, dtype=np.int32)
        self.rp = np.ascontiguousarray(self.rp, dtype=np.int64)
        self.col = np.ascontiguousarray(self.col, dtype=np.int32)
        self.data = np.ascontiguousarray(self.data, dtype=np.float64)
        self.roff = np.zeros(self.nblk + 1, dtype=np.int64)
        np.cumsum(self.bs, out=self.roff[1:])
        self.rows = np.repeat(np.arange(self.nblk, dtype=np.int32), np.diff(self.rp))
        area = self.bs[self.rows].astype(np.int64) * self.bs[self.col].astype(np.int64)
        self.boff = np.zeros(self.nnzb + 1, dtype=np.int64)
        np.cumsum(area, out=self.boff[1:])
        if self.data.shape[0] != int(self.boff[-1]):
            raise ValueError(f"data has {self.data.shape[0]} entries, pattern needs {int(self.boff[-1])}")

    @property
    def nblk(self) -> int:
        return int(self.bs.shape[0])

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])

    @property
    def n(self) -> int:
        return int(self.roff[-1])

    @classmethod
    def of(cls, m) -> "Mat":
        """Copy of any object with blk_size/row_ptr/col/data (the generator's format)."""
        return cls(np.array(m.blk_size), np.array(m.row_ptr), np.array(m.col), np.array(m.data))

    def copy(self) -> "Mat":
        return Mat(self.bs.copy(), self.rp.copy(), self.col.copy(), self.data.copy())

    def block(self, I: int, J: int):
        lo, hi = int(self.rp[I]), int(self.rp[I + 1])
        k = lo + int(np.searchsorted(self.col[lo:hi], J))
        if k < hi and self.col[k] == J:
            m, n = int(self.bs[I]), int(self.bs[J])
            return self.data[self.boff[k]:self.boff[k] + m * n].reshape(m, n)
        return None


def to_dense(M: Mat) -> np.ndarray:
    out = np.zeros((M.n, M.n))
    for b in range(M.nnzb):
        I, J = int(M.rows[b]), int(M.col[b])
        m, n = int(M.bs[I]), int(M.bs[J])
        out[M.roff[I]:M.roff[I] + m, M.roff[J]:M.roff[J] + n] = M.data[M.boff[b]:M.boff[b] + m * n].reshape(m, n)
    return out


def from_dense(D: np.ndarray, bs, pattern=None) -> Mat:
    """Block matrix holding D on ``pattern`` (list of (I, J)), or on every nonzero block."""
    bs = np.asarray(bs, dtype=np.int32)
    roff = np.concatenate([[0], np.cumsum(bs)])
    nblk = bs.shape[0]
    if pattern is None:
        pattern = [(I, J) for I in range(nblk) for J in range(nblk)
                   if np.any(D[roff[I]:roff[I + 1], roff[J]:roff[J + 1]] != 0) or I == J]
    pattern = sorted(pattern)
    rp = np.zeros(nblk + 1, dtype=np.int64)
    for I, _ in pattern:
        rp[I + 1] += 1
    rp = np.cumsum(rp)
    col = np.array([J for _, J in pattern], dtype=np.int32)
    data = np.concatenate([D[roff[I]:roff[I + 1], roff[J]:roff[J + 1]].ravel() for I, J in pattern]) \
        if pattern else np.zeros(0)
    return Mat(bs, rp, col, data)


@dataclasses.dataclass
class MultInfo:
    unfiltered: Mat         # alpha*A*B + beta*C_in on the full product pattern (prescreened: the formed blocks)
    norms: np.ndarray       # Frobenius norm of each unfiltered block
    keep: np.ndarray        # bool mask of the blocks that survive the filter
    dev2: float             # ||filtered - 1||_F^2 (the residual the sign iteration tests)
    dev2_unfiltered: float  # ||unfiltered - 1||_F^2
    n_products: int         # block products A_IK * B_KJ
    flops: int              # sum of 2*m*k*n over those products


def product_pattern(A: Mat, B: Mat, Cin: Mat | None = None):
    """Row pointers and sorted block columns of the pattern of A*B (union C_in)."""
    L = lib()
    cnt = np.zeros(A.nblk, dtype=np.int64)
    err = L.oracle_mm_count(A.nblk, _p(A.rp), _p(A.col), _p(B.rp), _p(B.col),
                            _p(Cin.rp) if Cin else None, _p(Cin.col) if Cin else None, _p(cnt))
    if err:
        raise MemoryError("oracle_mm_count")
    rp = np.zeros(A.nblk + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp[1:])
    col = np.zeros(int(rp[-1]), dtype=np.int32)
    err = L.oracle_mm_pattern(A.nblk, _p(A.rp), _p(A.col), _p(B.rp), _p(B.col),
                              _p(Cin.rp) if Cin else None, _p(Cin.col) if Cin else None, _p(rp), _p(col))
    if err:
        raise MemoryError("oracle_mm_pattern")
    return rp, col


def block_norms(M: Mat):
    norm = np.zeros(M.nnzb)
    dev2 = np.zeros(M.nnzb)
    lib().oracle_block_norms(M.nnzb, _p(M.rows), _p(M.col), _p(M.bs), _p(M.boff), _p(M.data), _p(norm), _p(dev2))
    return norm, dev2


def keep_mask(M: Mat, norms: np.ndarray, eps: float) -> np.ndarray:
    """Blocks kept by the filter: norm >= eps, and every diagonal block."""
    return (norms >= eps) | (M.rows == M.col)


def select_blocks(M: Mat, keep: np.ndarray) -> Mat:
    """The sub-matrix made of the blocks flagged in ``keep`` (order preserved)."""
    keep = np.asarray(keep, dtype=bool)
    cnt = np.bincount(M.rows[keep], minlength=M.nblk)
    rp = np.zeros(M.nblk + 1, dtype=np.int64)
    np.cumsum(cnt, out=rp[1:])
    area = M.boff[1:] - M.boff[:-1]
    idx = np.repeat(M.boff[:-1][keep], area[keep]) + (
        np.arange(int(area[keep].sum())) - np.repeat(np.cumsum(area[keep]) - area[keep], area[keep]))
    return Mat(M.bs, rp, M.col[keep], M.data[idx])


def filter_blocks(M: Mat, eps: float) -> Mat:
    """Drops the blocks with Frobenius norm < eps (diagonal blocks are kept)."""
    norms, _ = block_norms(M)
    return select_blocks(M, keep_mask(M, norms, eps))


# a candidate is kept when its bound reaches eps (1 - 1e-12): the margin covers the rounding of
# the bound's sum, so that no block whose computed norm reaches eps is left out
PRESCREEN_MARGIN = 1.0 - 1e-12


def prescreen_mask(alpha: float, A: Mat, B: Mat, beta: float, Cin: Mat | None, rp, col, eps: float):
    """keep[q] for the candidates (rp, col) of alpha*A*B + beta*C_in: I == J, or the norm bound
    |alpha| sum_K ||A_IK|| ||B_KJ|| (+ |beta| ||C_in,IJ||) at least eps (1 - 1e-12)."""
    na, _ = block_norms(A)
    nb, _ = block_norms(B)
    use_c = Cin is not None and beta != 0.0
    nc = block_norms(Cin)[0] if use_c else None
    keep = np.zeros(max(int(rp[-1]), 1), dtype=np.int32)
    err = lib().oracle_prescreen(A.nblk, abs(float(alpha)), _p(A.rp), _p(A.col), _p(na), _p(B.rp), _p(B.col),
                                 _p(nb), abs(float(beta)), _p(Cin.rp) if use_c else None,
                                 _p(Cin.col) if use_c else None, _p(nc) if use_c else None,
                                 _p(np.ascontiguousarray(rp, dtype=np.int64)),
                                 _p(np.ascontiguousarray(col, dtype=np.int32)), float(eps) * PRESCREEN_MARGIN, _p(keep))
    if err:
        raise MemoryError("oracle_prescreen")
    return keep[:int(rp[-1])].astype(bool)


def multiply(alpha: float, A: Mat, B: Mat, beta: float = 0.0, Cin: Mat | None = None,
             eps: float = 0.0, info: bool = False, prescreen: bool = False):
    """C = filter(alpha*A*B + beta*C_in, eps).  Returns C (and a MultInfo if ``info``).

    prescreen: form only the candidate blocks whose norm bound reaches eps (and the diagonal
    ones); the others would be filtered anyway, so C is the same, bit for bit, with fewer block
    products (``MultInfo.unfiltered`` then holds the formed blocks)."""
    if not (np.array_equal(A.bs, B.bs) and (Cin is None or np.array_equal(A.bs, Cin.bs))):
        raise ValueError("block sizes differ")
    rp, col = product_pattern(A, B, Cin if (Cin is not None and beta != 0.0) else None)
    if prescreen and eps > 0.0:
        keep0 = prescreen_mask(alpha, A, B, beta, Cin, rp, col, eps)
        cnt = np.bincount(np.repeat(np.arange(A.nblk), np.diff(rp))[keep0], minlength=A.nblk)
        rp = np.zeros(A.nblk + 1, dtype=np.int64)
        np.cumsum(cnt, out=rp[1:])
        col = np.ascontiguousarray(col[keep0])
    rows = np.repeat(np.arange(A.nblk, dtype=np.int32), np.diff(rp))
    area = A.bs[rows].astype(np.int64) * A.bs[col].astype(np.int64)
    data = np.zeros(int(area.sum()))
    Cu = Mat(A.bs, rp, col, data)
    stats = np.zeros(2, dtype=np.int64)
    use_c = Cin is not None and beta != 0.0
    err = lib().oracle_mm_numeric(
        A.nblk, _p(A.bs), float(alpha),
        _p(A.rp), _p(A.col), _p(A.boff), _p(A.data),
        _p(B.rp), _p(B.col), _p(B.boff), _p(B.data),
        float(beta),
        _p(Cin.rp) if use_c else None, _p(Cin.col) if use_c else None,
        _p(Cin.boff) if use_c else None, _p(Cin.data) if use_c else None,
        _p(Cu.rp), _p(Cu.col), _p(Cu.boff), _p(Cu.data), _p(stats))
    if err:
        raise MemoryError("oracle_mm_numeric")
    norms, dev2 = block_norms(Cu)
    keep = keep_mask(Cu, norms, eps)
    Cf = select_blocks(Cu, keep)
    if not info:
        return Cf
    d2u = lib().oracle_sum_dev2(Cu.nblk, _p(Cu.bs), _p(Cu.rp), _p(Cu.col), _p(dev2))
    dk = np.ascontiguousarray(dev2[keep])
    d2f = lib().oracle_sum_dev2(Cf.nblk, _p(Cf.bs), _p(Cf.rp), _p(Cf.col), _p(dk))
    return Cf, MultInfo(Cu, norms, keep, float(d2f), float(d2u), int(stats[0]), int(stats[1]))


def product_block(I: int, J: int, alpha: float, A: Mat, B: Mat, beta: float = 0.0, Cin: Mat | None = None):
    """Block (I, J) of alpha*A*B + beta*C_in, computed on its own (same loop order as multiply)."""
    out = np.zeros(int(A.bs[I]) * int(A.bs[J]))
    ci = Cin.block(I, J) if (Cin is not None and beta != 0.0) else None
    ci = None if ci is None else np.ascontiguousarray(ci).ravel()
    lib().oracle_mm_block(int(I), int(J), _p(A.bs), float(alpha), _p(A.rp), _p(A.col), _p(A.boff), _p(A.data),
                          _p(B.rp), _p(B.col), _p(B.boff), _p(B.data), float(beta), _p(ci), _p(out))
    return out.reshape(int(A.bs[I]), int(A.bs[J]))


def trace(M: Mat) -> float:
    return float(lib().oracle_trace(M.nblk, _p(M.bs), _p(M.rp), _p(M.col), _p(M.boff), _p(M.data)))


def trace_product(A: Mat, B: Mat) -> float:
    """Tr(A*B) without forming the product."""
    return float(lib().oracle_trace_product(A.nblk, _p(A.bs), _p(A.rp), _p(A.col), _p(A.boff), _p(A.data),
                                            _p(B.rp), _p(B.col), _p(B.boff), _p(B.data)))


def abs_row_sums(M: Mat, mu: float = 0.0) -> np.ndarray:
    out = np.zeros(M.n)
    lib().oracle_abs_row_sums(M.nblk, _p(M.bs), _p(M.roff), _p(M.rp), _p(M.col), _p(M.boff), _p(M.data),
                              float(mu), _p(out))
    return out


def add_identity(M: Mat, scale: float, shift: float) -> Mat:
    """scale*M + shift*1 (every diagonal block must be present)."""
    out = M.copy()
    out.data *= scale
    for I in range(M.nblk):
        blk = out.block(I, I)
        if blk is None:
            raise ValueError(f"diagonal block {I} missing")
        blk[np.diag_indices(int(M.bs[I]))] += shift
    return out


def add(alpha: float, A: Mat, beta: float, B: Mat) -> Mat:
    """alpha*A + beta*B on the union of the two patterns, unfiltered (DBCSR's add).

    A block present in one operand only is that operand's term alone; in a block of
    both, every element is alpha*a + beta*b (two rounded products, then their sum)."""
    if not np.array_equal(A.bs, B.bs):
        raise ValueError("block sizes differ")
    nblk = A.nblk
    ka = A.rows.astype(np.int64) * nblk + A.col
    kb = B.rows.astype(np.int64) * nblk + B.col
    keys = np.union1d(ka, kb)
    rows = (keys // nblk).astype(np.int32)
    rp = np.zeros(nblk + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=nblk), out=rp[1:])
    area = A.bs[rows].astype(np.int64) * A.bs[(keys % nblk)].astype(np.int64)
    out = Mat(A.bs, rp, (keys % nblk).astype(np.int32), np.zeros(int(area.sum())))

    def scatter(M: Mat, k: np.ndarray, scale: float):
        """M's elements times scale at their places in out, and where they land."""
        dst_blk = np.searchsorted(keys, k)
        areas = np.diff(M.boff)
        blk = np.repeat(np.arange(M.nnzb), areas)
        dst = out.boff[dst_blk[blk]] + (np.arange(M.data.shape[0]) - M.boff[blk])
        term = np.zeros(out.data.shape[0])
        term[dst] = scale * M.data
        has = np.zeros(out.data.shape[0], dtype=bool)
        has[dst] = True
        return term, has

    ta, ha = scatter(A, ka, alpha)
    tb, hb = scatter(B, kb, beta)
    out.data[:] = np.where(ha & hb, ta + tb, np.where(ha, ta, tb))
    return out


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (timing on fewer cores; no effect on
    the results, which do not depend on the thread count)."""
    lib().oracle_set_num_threads(int(n))


def os_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", "0")) or num_threads()

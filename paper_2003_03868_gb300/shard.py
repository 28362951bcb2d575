"""The sign iteration sharded over ranks by spatial domains of block rows (host side).

The paper's DBCSR distributes a matrix over a 2-D process grid and multiplies with Cannon's
algorithm and asynchronous point-to-point messages (section "DBCSR library").  For the
local, banded matrices of the sign iteration a 1-D split is enough: each rank owns a domain
of block rows (``dbcsr_partition_rows``: compact regions of the coupling graph), and a
product C = A B needs on each rank only the rows of B that its rows of A reference -- its
own rows and a halo of neighbouring rows (``dbcsr_halo_rows``).  So every product takes one
exchange of halo rows, every scalar one sum over the ranks, and each rank multiplies its
rows on its own GPU.

The data plane moves block rows as tensors through ``torch.distributed``: with NCCL they are
device tensors, with gloo host tensors; every round is one batched set of point-to-point
sends and receives.  A rank first tells each owner which rows it needs (its halo: the block
columns of its rows of X that other ranks own), then the owners send the rows' block counts,
columns and values.  The local arithmetic is a backend object: ``LibraryBackend`` runs every
product, shift and trace in the library on the rank's GPU; the tests run the same driver
with the oracle's CPU arithmetic.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math

import numpy as np

from . import _ffi


def _lib():
    return _ffi.load()


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _check(st, where):
    if st != _ffi.DBCSR_OK:
        raise RuntimeError(f"{where}: {_ffi.STATUS_NAMES.get(st, st)}: {_lib().dbcsr_last_error().decode()}")


def partition_rows(row_ptr, col, nparts: int) -> np.ndarray:
    """Owner rank of every block row (dbcsr_partition_rows)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    nblk = rp.shape[0] - 1
    owner = np.zeros(nblk, dtype=np.int32)
    _check(_lib().dbcsr_partition_rows(nblk, _p(rp), _p(cl), int(nparts), _p(owner)), "partition_rows")
    return owner


def halo_rows(row_ptr, col, owner, rank: int) -> np.ndarray:
    """Block rows that rank's rows reference but other ranks own, ascending (dbcsr_halo_rows)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    ow = np.ascontiguousarray(owner, dtype=np.int32)
    nblk = rp.shape[0] - 1
    n = C.c_int32()
    _check(_lib().dbcsr_halo_rows(nblk, _p(rp), _p(cl), _p(ow), int(rank), None, 0, C.byref(n)), "halo_rows")
    out = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(_lib().dbcsr_halo_rows(nblk, _p(rp), _p(cl), _p(ow), int(rank), _p(out), n.value, C.byref(n)),
           "halo_rows")
    return out[:n.value]


def _block_offsets(bs, rows_of_blocks, col):
    area = bs[rows_of_blocks].astype(np.int64) * bs[col].astype(np.int64) if len(col) else np.zeros(0, np.int64)
    return np.concatenate([[0], np.cumsum(area)]).astype(np.int64)


@dataclasses.dataclass
class Rows:
    """Some block rows of a square block matrix, on the host: rows (ascending block-row ids),
    rp[len(rows) + 1] local row pointers, col (block columns, ascending per row), data (the
    blocks row-major, packed in row order)."""

    bs: np.ndarray
    rows: np.ndarray
    rp: np.ndarray
    col: np.ndarray
    data: np.ndarray

    @classmethod
    def select(cls, bs, row_ptr, col, data, rows) -> "Rows":
        """The given rows of a full block-CSR matrix (blk_size, row_ptr, col, data)."""
        bs = np.asarray(bs, dtype=np.int32)
        row_ptr = np.asarray(row_ptr, dtype=np.int64)
        col = np.asarray(col, dtype=np.int32)
        rows = np.asarray(rows, dtype=np.int32)
        off = _block_offsets(bs, np.repeat(np.arange(bs.shape[0], dtype=np.int32), np.diff(row_ptr)), col)
        cnt = row_ptr[rows + 1] - row_ptr[rows]
        rp = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
        bidx = (np.concatenate([np.arange(row_ptr[r], row_ptr[r + 1]) for r in rows]).astype(np.int64)
                if len(rows) else np.zeros(0, np.int64))
        vals = (np.concatenate([np.asarray(data)[off[b]:off[b + 1]] for b in bidx]) if len(bidx) else np.zeros(0))
        return cls(bs, rows, rp, col[bidx], vals.astype(np.float64))

    @property
    def nblk(self) -> int:
        return int(self.bs.shape[0])

    def offsets(self):
        return _block_offsets(self.bs, self.rows[np.repeat(np.arange(len(self.rows)), np.diff(self.rp))], self.col)

    def full(self):
        """(row_ptr[nblk + 1], col, data) of the block matrix that holds only these rows."""
        cnt = np.zeros(self.nblk, dtype=np.int64)
        cnt[self.rows] = np.diff(self.rp)
        return np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64), self.col, self.data

    def merged(self, other: "Rows") -> "Rows":
        """The union of two disjoint row sets, rows ascending."""
        parts = []
        for R in (self, other):
            off = R.offsets()
            for i in range(len(R.rows)):
                b0, b1 = int(R.rp[i]), int(R.rp[i + 1])
                parts.append((int(R.rows[i]), R.col[b0:b1], R.data[off[b0]:off[b1]]))
        parts.sort(key=lambda p: p[0])
        rows = np.array([p[0] for p in parts], dtype=np.int32)
        rp = np.concatenate([[0], np.cumsum([len(p[1]) for p in parts])]).astype(np.int64)
        col = np.concatenate([p[1] for p in parts]).astype(np.int32) if parts else np.zeros(0, np.int32)
        data = np.concatenate([p[2] for p in parts]) if parts else np.zeros(0)
        return Rows(self.bs, rows, rp, col, data)


class Shard:
    """One rank's view: the owner of every block row (the same on all ranks) and its own rows."""

    def __init__(self, row_ptr, col, rank: int, world: int, owner=None):
        self.rank, self.world = int(rank), int(world)
        self.owner = partition_rows(row_ptr, col, world) if owner is None else np.asarray(owner, np.int32)
        self.own = np.nonzero(self.owner == self.rank)[0].astype(np.int32)

    def halo(self, A: Rows) -> np.ndarray:
        """The rows this rank needs for a product with A's rows on the left: the block columns
        of A's rows that other ranks own (dbcsr_halo_rows on the pattern of A's rows)."""
        rp, col, _ = A.full()
        return halo_rows(rp, col, self.owner, self.rank)


def _rows_payload(R: Rows, rows):
    """(block counts per row, block columns, values) of the given rows of R (a subset of R.rows)."""
    pos = np.searchsorted(R.rows, rows)
    cnt = (R.rp[pos + 1] - R.rp[pos]).astype(np.int64)
    off = R.offsets()
    cols, vals = [], []
    for p in pos:
        b0, b1 = int(R.rp[p]), int(R.rp[p + 1])
        cols.append(R.col[b0:b1])
        vals.append(R.data[off[b0]:off[b1]])
    col = np.concatenate(cols).astype(np.int64) if cols else np.zeros(0, np.int64)
    val = np.concatenate(vals) if vals else np.zeros(0)
    return cnt, col, val


def _p2p(dist, sends, recvs):
    """One batched round of point-to-point messages: sends and recvs map a peer to a tensor.
    Empty messages are left out (both ends know the size in advance)."""
    ops = [dist.P2POp(dist.isend, t, p) for p, t in sends.items() if t.numel()]
    ops += [dist.P2POp(dist.irecv, t, p) for p, t in recvs.items() if t.numel()]
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()


def exchange(sh: Shard, need, R: Rows, dist, device="cpu") -> Rows:
    """The rows ``need`` (owned by other ranks) of the matrix whose own rows this rank holds in
    R, received from their owners.  Four batched rounds: how many rows each rank asks of each
    peer, which rows, their block counts with the number of values, then columns and values."""
    import torch
    peers = [p for p in range(sh.world) if p != sh.rank]
    need = np.asarray(need, dtype=np.int32)
    need_from = {p: need[sh.owner[need] == p] for p in peers}

    def tens(a, dt=torch.int64):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt, device=device)

    n_give = {p: torch.zeros(1, dtype=torch.int64, device=device) for p in peers}
    _p2p(dist, {p: tens(np.array([len(need_from[p])])) for p in peers}, n_give)
    give = {p: torch.zeros(int(n_give[p].item()), dtype=torch.int64, device=device) for p in peers}
    _p2p(dist, {p: tens(need_from[p]) for p in peers}, give)
    payload = {p: _rows_payload(R, give[p].cpu().numpy().astype(np.int32)) for p in peers}
    sizes = {p: torch.zeros(len(need_from[p]) + 1, dtype=torch.int64, device=device) for p in peers}
    _p2p(dist, {p: tens(np.concatenate([payload[p][0], [payload[p][2].shape[0]]])) for p in peers}, sizes)
    got = {}
    for p in peers:
        c = sizes[p].cpu().numpy()
        got[p] = (c[:-1], torch.zeros(int(c[:-1].sum()), dtype=torch.int64, device=device),
                  torch.zeros(int(c[-1]), dtype=torch.float64, device=device))
    _p2p(dist, {p: tens(payload[p][1]) for p in peers}, {p: got[p][1] for p in peers})
    _p2p(dist, {p: tens(payload[p][2], torch.float64) for p in peers}, {p: got[p][2] for p in peers})
    parts = []
    for p in peers:
        cnt, cl, vl = got[p][0], got[p][1].cpu().numpy().astype(np.int32), got[p][2].cpu().numpy()
        b_start = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
        row_of = np.repeat(need_from[p], cnt)
        voff = _block_offsets(R.bs, row_of, cl)
        for i, r in enumerate(need_from[p]):
            b0, b1 = int(b_start[i]), int(b_start[i + 1])
            parts.append((int(r), cl[b0:b1], vl[voff[b0]:voff[b1]]))
    parts.sort(key=lambda x: x[0])
    rows = np.array([x[0] for x in parts], dtype=np.int32)
    rp = np.concatenate([[0], np.cumsum([len(x[1]) for x in parts])]).astype(np.int64)
    col = np.concatenate([x[1] for x in parts]).astype(np.int32) if parts else np.zeros(0, np.int32)
    data = np.concatenate([x[2] for x in parts]) if parts else np.zeros(0)
    return Rows(R.bs, rows, rp, col, data)


def _allreduce(x: float, dist, device, op="sum") -> float:
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX)
    return float(t.item())


def shift_diagonal(R: Rows, scale: float, shift: float) -> Rows:
    """scale R + shift on the diagonal of R's rows (each of them must hold its diagonal block)."""
    data = R.data * scale
    off = R.offsets()
    for i, I in enumerate(R.rows):
        seg = R.col[R.rp[i]:R.rp[i + 1]]
        q = int(R.rp[i]) + int(np.searchsorted(seg, I))
        if q >= R.rp[i + 1] or R.col[q] != I:
            raise ValueError(f"diagonal block {I} missing")
        m = int(R.bs[I])
        data[off[q]:off[q] + m * m].reshape(m, m)[np.diag_indices(m)] += shift
    return Rows(R.bs, R.rows, R.rp, R.col, data)


class LibraryBackend:
    """A rank's local arithmetic in the library, on its GPU: the products, the Gershgorin
    bound and the scaled shifts run in the library's kernels (rows move through host memory
    between products)."""

    def __init__(self, prec=None):
        from . import DBCSR_FP64
        self.prec = DBCSR_FP64 if prec is None else prec

    def _mat(self, R: Rows):
        from . import Matrix
        rp, col, data = R.full()
        return Matrix.from_blocks(R.bs, rp, col, data)

    def gershgorin(self, R: Rows, mu: float) -> float:
        from . import gershgorin
        return gershgorin(self._mat(R), mu)

    def add_identity(self, R: Rows, scale: float, shift: float) -> Rows:
        return shift_diagonal(R, scale, shift)

    def multiply(self, alpha: float, A: Rows, B: Rows, eps: float):
        from . import Matrix, multiply
        Am, Bm = self._mat(A), self._mat(B)
        Cm = Matrix(A.bs, Am.stream)
        st = multiply(alpha, Am, Bm, 0.0, Cm, eps, prec=self.prec)
        rp, col, data = Cm.export()
        return Rows.select(A.bs, rp, col, data, A.rows), float(st.dev2_filtered), float(st.flops)


@dataclasses.dataclass
class ShardedResult:
    P: Rows                 # this rank's rows of P = (1 - X) / 2
    iterations: int
    converged: bool
    stalled: bool
    residuals: list
    alpha: float
    trace_p: float
    e_band: float
    flops: float            # this rank's executed block-product flops
    halo_rows: int          # rows received in the last exchange


def sign_iterate(H: Rows, sh: Shard, mu: float, eps: float, tol: float, backend, dist, device="cpu",
                 max_iter: int = 100, stall_ratio: float = 0.5) -> ShardedResult:
    """Newton-Schulz sign iteration X <- X (3 - X^2) / 2 on the rank's rows (the paper's sign
    method, section "Sign-Method", with the filter after every product):
      X_0 = (H - mu) / alpha, alpha the Gershgorin bound (max over every rank's rows);
      per step: X2 = filter(X X) with X's halo rows received first; r = ||X2 - 1||_F / N with
      the squared norm summed over the ranks; stop at r < tol or on the stall rule; else
      T = 3 - X2 and X = filter(X T / 2) with T's halo rows received first.
    The halo of a step is the block columns of the rank's rows of X owned elsewhere (for X X
    and X T alike).  P = (1 - X) / 2 on the rank's rows; Tr P and Tr(P H) are sums over the
    ranks (H symmetric: Tr(P H) = sum over blocks of <P_IJ, H_IJ>, local to each rank)."""
    n = int(H.bs.sum())
    alpha = _allreduce(backend.gershgorin(H, mu), dist, device, op="max")
    X = backend.add_identity(H, 1.0 / alpha, -mu / alpha)
    res, flops = [], 0.0
    converged = stalled = False
    it, nh = 0, 0
    while it < max_iter:
        need = sh.halo(X)
        nh = len(need)
        X2, d2, fl = backend.multiply(1.0, X, X.merged(exchange(sh, need, X, dist, device)), eps)
        flops += fl
        it += 1
        r = math.sqrt(max(_allreduce(d2, dist, device), 0.0)) / n
        res.append(r)
        if r < tol:
            converged = True
            break
        if len(res) >= 3 and res[-2] < stall_ratio * res[-3] and r > stall_ratio * res[-2]:
            stalled = True
            break
        T = backend.add_identity(X2, -1.0, 3.0)
        X, _, fl = backend.multiply(0.5, X, T.merged(exchange(sh, need, T, dist, device)), eps)
        flops += fl
    P = backend.add_identity(X, -0.5, 0.5)
    tr = _allreduce(_diag_sum(P), dist, device)
    eb = _allreduce(_inner(P, H), dist, device)
    return ShardedResult(P, it, converged, stalled, res, alpha, tr, eb, flops, nh)


def _diag_sum(R: Rows) -> float:
    off = R.offsets()
    s = 0.0
    for i, I in enumerate(R.rows):
        for q in range(int(R.rp[i]), int(R.rp[i + 1])):
            if R.col[q] == I:
                m = int(R.bs[I])
                s += float(np.trace(R.data[off[q]:off[q] + m * m].reshape(m, m)))
    return s


def _inner(P: Rows, H: Rows) -> float:
    """sum over P's blocks (I, J) of <P_IJ, H_IJ>; H holds the same rows as P."""
    if not np.array_equal(P.rows, H.rows):
        raise ValueError("P and H must hold the same rows")
    op, oh = P.offsets(), H.offsets()
    s = 0.0
    for i in range(len(P.rows)):
        hseg = H.col[H.rp[i]:H.rp[i + 1]]
        for q in range(int(P.rp[i]), int(P.rp[i + 1])):
            k = int(np.searchsorted(hseg, P.col[q]))
            if k < len(hseg) and hseg[k] == P.col[q]:
                qh = int(H.rp[i]) + k
                s += float(np.dot(P.data[op[q]:op[q + 1]], H.data[oh[qh]:oh[qh + 1]]))
    return s

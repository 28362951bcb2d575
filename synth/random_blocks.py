"""Seeded random block-sparse matrices with arbitrary block sizes and patterns
(input generator for edge cases: ragged sizes, empty rows, non-symmetric data)."""
from __future__ import annotations

import numpy as np

from . import splitmix
from .waterbox import BlockMatrix


def random_block_matrix(blk_size, density: float, seed: int, scale: float = 1.0,
                        diag: bool = True, symmetric: bool = False, empty_rows=()) -> BlockMatrix:
    """Block (I, J) present with probability ``density`` (always when I == J and
    ``diag``); entries scale * U[-1, 1).  ``symmetric`` mirrors the upper triangle.
    Rows listed in ``empty_rows`` hold no block (and, if symmetric, no column either)."""
    bs = np.asarray(blk_size, dtype=np.int32)
    nb = bs.shape[0]
    u = splitmix.uniform01(splitmix.substream(seed, 11), np.arange(nb * nb, dtype=np.uint64)).reshape(nb, nb)
    present = u < density
    if diag:
        present |= np.eye(nb, dtype=bool)
    if symmetric:
        present = np.triu(present) | np.triu(present).T
    for r in empty_rows:
        present[r, :] = False
        if symmetric:
            present[:, r] = False
    rows, cols = np.nonzero(present)
    rp = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=nb), out=rp[1:])
    area = bs[rows].astype(np.int64) * bs[cols].astype(np.int64)
    off = np.concatenate([[0], np.cumsum(area)])
    vals = scale * splitmix.uniform_pm1(splitmix.substream(seed, 12), np.arange(int(off[-1]), dtype=np.uint64))
    if symmetric:
        pos = {(int(r), int(c)): i for i, (r, c) in enumerate(zip(rows, cols))}
        for i, (r, c) in enumerate(zip(rows, cols)):
            if r > c:
                j = pos[(int(c), int(r))]
                m, n = int(bs[r]), int(bs[c])
                vals[off[i]:off[i + 1]] = vals[off[j]:off[j + 1]].reshape(n, m).T.ravel()
            elif r == c:
                m = int(bs[r])
                blk = vals[off[i]:off[i + 1]].reshape(m, m)
                vals[off[i]:off[i + 1]] = (0.5 * (blk + blk.T)).ravel()
    return BlockMatrix(bs, rp, cols.astype(np.int32), vals)

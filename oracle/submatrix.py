"""Density matrix by the submatrix method, FP64 (TEST INFRASTRUCTURE ONLY).

Section "Submatrix Method": instead of the whole Kohn-Sham matrix, principal submatrices
are purified.  Each covers the atoms of one block of the DBCSR matrix together with the
atoms in its neighbourhood whose basis functions overlap it; the submatrices are small
and dense, and purification is done either with an iterative sign scheme or with a
direct eigendecomposition.

Readings taken where the paper is silent:

* one submatrix per block column j (one atom): its index set I_j is the pattern of
  column j of H (the blocks i with H_ij present, j included), and H^(j) = H[I_j, I_j]
  holds every block of H between two atoms of I_j (zero where H has no block);
* P^(j) = (1 - sign(H^(j) - mu 1)) / 2 from the eigendecomposition of H^(j) (the paper's
  direct variant; eigenvalues equal to mu do not occur on gapped inputs);
* block (i, j) of P, for i in I_j, is the block of P^(j) at the rows of i and the columns
  of j: P has the pattern of H and is not symmetrised (its blocks (i, j) and (j, i) come
  from different submatrices).
"""
from __future__ import annotations

import numpy as np

from . import bsr


def submatrix_index_sets(H: bsr.Mat):
    """I_j for every block column j (the column pattern; H's pattern is symmetric)."""
    return [H.col[H.rp[j]:H.rp[j + 1]].astype(np.int64) for j in range(H.nblk)]


def element_index(H: bsr.Mat, I) -> np.ndarray:
    """The matrix rows of the blocks in I, in the order of I."""
    return np.concatenate([np.arange(H.roff[i], H.roff[i] + H.bs[i]) for i in I]).astype(np.int64)


def submatrix_density(H: bsr.Mat, mu: float) -> bsr.Mat:
    """P by the submatrix method (see the module header), on the pattern of H."""
    Hd = bsr.to_dense(H)                                   # test sizes: the whole H fits
    out = H.copy()
    out.data[:] = 0.0
    for j, I in enumerate(submatrix_index_sets(H)):
        idx = element_index(H, I)
        w, Q = np.linalg.eigh(Hd[np.ix_(idx, idx)])        # H^(j) = H[I_j, I_j]
        occ = w < mu
        Pj = Q[:, occ] @ Q[:, occ].T
        off = np.concatenate([[0], np.cumsum(H.bs[I])]).astype(np.int64)
        pj = int(np.searchsorted(I, j))
        cols = slice(int(off[pj]), int(off[pj + 1]))
        for a, i in enumerate(I):
            blk = out.block(int(i), j)
            blk[:, :] = Pj[off[a]:off[a + 1], cols]
    return out

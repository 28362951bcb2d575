"""Dense reference of the sign and the density matrix (TEST INFRASTRUCTURE ONLY).

sign(A) = A (A^2)^(-1/2) (section "Sign-Method", Eq. signdef) is, for a
symmetric A = Q diag(lambda) Q^T, the matrix Q diag(sgn(lambda)) Q^T: the plain
definition, computed with a dense symmetric eigendecomposition (LAPACK through
numpy).  P = (1 - sign(H - mu 1)) / 2 (S = 1) then gives the exact, unfiltered
occupation and band energy: Tr(P) = number of eigenvalues below mu and
Tr(P H) = sum of those eigenvalues.
"""
from __future__ import annotations

import numpy as np

from . import bsr


def spectrum(H: bsr.Mat) -> np.ndarray:
    """Eigenvalues of the (symmetric) block matrix, ascending."""
    return np.linalg.eigvalsh(bsr.to_dense(H))


def band_energy_exact(H: bsr.Mat, mu: float):
    """(Tr(P), Tr(P H)) of the exact density matrix: count and sum of eigenvalues below mu."""
    w = spectrum(H)
    occ = w < mu
    return int(occ.sum()), float(np.sum(w[occ])), w


def sign_dense(H: bsr.Mat, mu: float) -> np.ndarray:
    """Dense sign(H - mu 1) = Q sgn(Lambda - mu) Q^T."""
    D = bsr.to_dense(H)
    w, Q = np.linalg.eigh(D - mu * np.eye(D.shape[0]))
    return (Q * np.sign(w)) @ Q.T

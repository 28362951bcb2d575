"""Pins of the oracle's submatrix method (no GPU): where the neighbourhoods cover the
coupling the method is exact (a box in which every atom overlaps every other, and a
Hamiltonian without inter-molecular blocks), the result keeps the pattern of H, and on a
larger box its band energy stays close to the exact one."""
import numpy as np
import pytest

import synth
from oracle import bsr, submatrix


def _exact(H: bsr.Mat, mu=0.0):
    w, Q = np.linalg.eigh(bsr.to_dense(H))
    return Q[:, w < mu] @ Q[:, w < mu].T


@pytest.mark.parametrize("basis", [(13, 5), (4, 1)])
def test_complete_neighbourhoods_give_the_exact_density_matrix(basis):
    # 4 waters at 1 g/cc: every atom pair lies within the 8 A cutoff, so I_j is every atom
    h = synth.build_hamiltonian(synth.small(4, basis=basis, seed=41))
    H = bsr.Mat.of(h.H)
    assert H.nnzb == H.nblk ** 2
    P = submatrix.submatrix_density(H, 0.0)
    assert np.linalg.norm(bsr.to_dense(P) - _exact(H)) < 1e-12


def test_decoupled_molecules_are_exact():
    h = synth.build_hamiltonian(synth.small(12, basis=(4, 1), seed=42))
    H = bsr.Mat.of(h.H)
    keep = (H.rows // 3) == (H.col // 3)
    Hm = bsr.select_blocks(H, keep)                 # intra-molecular blocks only
    P = submatrix.submatrix_density(Hm, 0.0)
    assert np.linalg.norm(bsr.to_dense(P) - _exact(Hm)) < 1e-12
    assert np.array_equal(P.col, Hm.col)


def test_pattern_and_energy_on_a_larger_box():
    # 48 waters: neighbourhoods of 134 to 144 of the 144 atoms
    h = synth.build_hamiltonian(synth.small(48, basis=(4, 1), seed=43))
    H = bsr.Mat.of(h.H)
    assert min(len(I) for I in submatrix.submatrix_index_sets(H)) < H.nblk
    P = submatrix.submatrix_density(H, 0.0)
    assert np.array_equal(P.rp, H.rp) and np.array_equal(P.col, H.col)
    Pe = _exact(H)
    Hd = bsr.to_dense(H)
    e_sub = float(np.sum(bsr.to_dense(P) * Hd.T))
    e_ex = float(np.sum(Pe * Hd.T))
    # an approximation, but a close one on these weakly coupled molecules
    assert 0 < abs(e_sub - e_ex) / h.n_atoms < 1e-8
    assert abs(np.trace(bsr.to_dense(P)) - h.n_occ) < 1e-2 * h.n_occ

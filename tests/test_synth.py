"""Seeded input generator: determinism, geometry, symmetry, the guaranteed gap."""
import hashlib

import numpy as np
import pytest

import synth
from synth import splitmix, waterbox


def test_splitmix_reference_values():
    # SplitMix64 seeded with 0: first outputs as published with the algorithm
    # (Steele, Lea & Flood 2014; the same sequence seeds xoshiro generators).
    got = splitmix.raw(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range_and_counter_independence():
    u = splitmix.uniform_pm1(123, np.arange(100000, dtype=np.uint64))
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 0.01
    # any element can be drawn on its own
    v = splitmix.uniform_pm1(123, np.array([99999, 5], dtype=np.uint64))
    assert v[0] == u[99999] and v[1] == u[5]


def test_water_geometry():
    wb = waterbox.place_waters(64, 77)
    assert wb.box == pytest.approx(9.86 * 2 ** (1 / 3))
    pos = wb.pos.reshape(64, 3, 3)
    for a in (1, 2):
        d = pos[:, a] - pos[:, 0]
        d -= wb.box * np.round(d / wb.box)
        assert np.allclose(np.linalg.norm(d, axis=1), waterbox.R_OH, atol=1e-9)
    o = pos[:, 0]
    d = o[:, None, :] - o[None, :, :]
    d -= wb.box * np.round(d / wb.box)
    r = np.linalg.norm(d, axis=2) + np.eye(64) * 100
    assert r.min() >= waterbox.MIN_OO


def test_decay_matrix_structure():
    A = synth.build_decay(synth.DECAY_32)
    assert A.nblk == 96 and A.n == 736
    # 32 waters in a 9.86 A box: almost every atom pair is within 8 A (min image)
    assert 0.99 < A.nnzb / 96 ** 2 <= 1.0
    from oracle.bsr import Mat, to_dense
    D = to_dense(Mat.of(A))
    assert np.array_equal(D, D.T)
    # diagonal blocks carry the +2 shift, entries of off-diagonal blocks are below exp(0)
    assert np.all(np.diag(D) > 1.0)


def test_generator_is_deterministic():
    a = synth.build_decay(synth.DECAY_32)
    b = synth.build_decay(synth.DECAY_32)
    assert np.array_equal(a.data, b.data) and np.array_equal(a.col, b.col)
    h = hashlib.sha256(a.col.tobytes()).hexdigest()
    assert h == hashlib.sha256(b.col.tobytes()).hexdigest()


@pytest.mark.parametrize("basis", [(13, 5), (23, 7)])
def test_gapped_hamiltonian_spectrum(basis):
    w = synth.small(24, basis=basis, seed=4242)
    h = synth.build_hamiltonian(w)
    from oracle.bsr import Mat, to_dense
    D = to_dense(Mat.of(h.H))
    assert np.array_equal(D, D.T)
    ev = np.linalg.eigvalsh(D)
    assert (ev < 0).sum() == h.n_occ == 4 * 24
    assert np.all(np.abs(ev) >= 0.25 - 1e-12) and np.all(np.abs(ev) <= 1.75 + 1e-12)
    assert 0 < h.gamma < 1


def test_workload_sizes():
    assert synth.SIGN_1024.n == 23552
    assert synth.SIGN_4096.n == 151552
    assert synth.SIGN_20736.n == 767232
    sys_ = synth.batch_systems()
    assert len(sys_) == 64
    assert all(100 <= s.n_mol <= 2000 for s in sys_)
    assert {s.basis[0] for s in sys_} == {13, 23} and {s.basis[1] for s in sys_} == {5, 7}


def test_overlap_is_deterministic_and_on_the_hamiltonian_pattern():
    w = synth.small(12, seed=31337)
    a, b = synth.build_overlap(w), synth.build_overlap(w)
    h = synth.build_hamiltonian(w)
    assert np.array_equal(a.data, b.data)
    assert np.array_equal(a.row_ptr, h.H.row_ptr) and np.array_equal(a.col, h.H.col)
    assert np.all(a.data >= 0)                             # 1 + sigma |D|
    assert not np.array_equal(synth.build_overlap(synth.small(12, seed=31338)).data[:50], a.data[:50])

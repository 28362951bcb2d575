"""GPU parity of the BF16 tensor-core product and the mixed-precision sign iteration.

BF16 product: the oracle multiplies the operands rounded to bfloat16 (nearest,
ties to even) in FP64; the GPU accumulates the same exact bf16 x bf16 products
in FP32, so the difference is bounded by FP32 summation: |d_ij| <= K_ij u32 (|A||B|)_ij.
Mixed sign iteration: the converged P must give the FP64 oracle's band energy
within 1e-6 Ha/atom."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import bsr, sign
from oracle.lowprec import round_bf16

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
U32 = 2.0 ** -24
DE_ATOM = 1e-6


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2003_03868_gb300 as m
    m.lib()
    return m


def _bf16_reference(Ao, Bo, alpha=1.0, beta=0.0, Co=None):
    Ar, Br = Ao.copy(), Bo.copy()
    Ar.data = round_bf16(Ar.data)
    Br.data = round_bf16(Br.data)
    ref = bsr.multiply(alpha, Ar, Br, beta, Co)
    Aa, Ba = Ar.copy(), Br.copy()
    Aa.data = np.abs(Aa.data)
    Ba.data = np.abs(Ba.data)
    mag = bsr.multiply(abs(alpha), Aa, Ba)
    return ref, mag


SIZES = [[13, 5, 5] * 6, [23, 7, 7] * 5, list(range(1, 33)), [16, 8, 17, 9, 32, 31]]


@pytest.mark.parametrize("si", range(len(SIZES)))
@pytest.mark.parametrize("density", [0.1, 0.6])
def test_bf16_product_matches_rounded_oracle(gb, si, density):
    bs = SIZES[si]
    a = synth.random_block_matrix(bs, density, 300 + si)
    b = synth.random_block_matrix(bs, density, 400 + si)
    A, B = gb.Matrix.of(a), gb.Matrix.of(b)
    Ao, Bo = bsr.Mat.of(a), bsr.Mat.of(b)
    C = gb.Matrix(A.blk_size, A.stream)
    st = gb.multiply(1.0, A, B, 0.0, C, 0.0, prec=gb.DBCSR_BF16)
    ref, mag = _bf16_reference(Ao, Bo)
    rp, col, data = C.export()
    assert np.array_equal(rp, ref.rp) and np.array_equal(col, ref.col)
    kmax = int(np.max(bs)) * len(bs)
    assert np.all(np.abs(data - ref.data) <= 2 * kmax * U32 * mag.data + 1e-300)
    # the low precision did happen: the FP64 product differs at the bf16 level
    exact = bsr.multiply(1.0, Ao, Bo)
    assert np.abs(data - exact.data).max() > 1e-6 * np.abs(exact.data).max()
    assert st.flops == bsr.multiply(1.0, Ao, Bo, info=True)[1].flops


def test_bf16_alpha_beta_and_aliasing(gb):
    bs = SIZES[0]
    x = synth.random_block_matrix(bs, 0.4, 501, symmetric=True)
    y = synth.random_block_matrix(bs, 0.4, 502, symmetric=True)
    X, Y = gb.Matrix.of(x), gb.Matrix.of(y)
    Xo, Yo = bsr.Mat.of(x), bsr.Mat.of(y)
    gb.multiply(-0.5, X, Y, 1.5, X, 0.0, prec=gb.DBCSR_BF16)
    ref, mag = _bf16_reference(Xo, Yo, -0.5, 1.5, Xo)
    rp, col, data = X.export()
    assert np.array_equal(col, ref.col)
    # beta * C_in is added in FP64 to the unrounded C_in
    assert np.all(np.abs(data - ref.data) <= 2 * 13 * 18 * U32 * mag.data + 1e-15)


def test_bf16_long_products_span_several_panels(gb):
    # 40 block rows of 23: a C block sums up to 40 products (920 > 128 columns per panel)
    bs = [23] * 40
    a = synth.random_block_matrix(bs, 1.0, 601)
    A, Ao = gb.Matrix.of(a), bsr.Mat.of(a)
    C = gb.Matrix(A.blk_size, A.stream)
    gb.multiply(1.0, A, A, 0.0, C, 0.0, prec=gb.DBCSR_BF16)
    ref, mag = _bf16_reference(Ao, Ao)
    _, _, data = C.export()
    assert np.all(np.abs(data - ref.data) <= 2 * 920 * U32 * mag.data + 1e-300)


@pytest.mark.parametrize("n_mol,basis,eps", [(24, (13, 5), 1e-7), (16, (23, 7), 1e-6)])
def test_mixed_sign_matches_fp64_oracle(gb, n_mol, basis, eps):
    h = synth.build_hamiltonian(synth.small(n_mol, basis=basis, seed=990 + n_mol))
    H = gb.Matrix.of(h.H)
    g = gb.sign_iterate(H, 0.0, eps, 1e-8, prec=gb.DBCSR_MIXED, switch_tol=1e-4)
    o = sign.sign_iterate(bsr.Mat.of(h.H), 0.0, eps, 1e-8)
    assert g.report.fp64_from > 1                     # some steps ran in BF16
    assert g.converged or g.report.stalled
    assert abs(g.report.e_band - o.e_band) / h.n_atoms < DE_ATOM
    assert g.report.trace_p == pytest.approx(h.n_occ, abs=1e-4)


@pytest.mark.slow
def test_mixed_sign_1024_waters(gb):
    w = synth.SIGN_1024
    h = synth.build_hamiltonian(w)
    g = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, w.eps_filter, w.tol, prec=gb.DBCSR_MIXED, switch_tol=1e-4)
    ref = json.load(open(os.path.join(HERE, "golden", "sign_1024h2o.json")))
    assert g.report.fp64_from > 1
    assert abs(g.report.e_band - ref["e_band"]) / h.n_atoms < DE_ATOM
    assert g.report.trace_p == pytest.approx(4096, abs=1e-4)


def test_mixed_density_matrix_is_symmetric(gb):
    h = synth.build_hamiltonian(synth.small(24, seed=990 + 24))
    g = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, 1e-7, 1e-8, prec=gb.DBCSR_MIXED)
    rp, col, data = g.P.export()
    D = bsr.to_dense(bsr.Mat(h.H.blk_size, rp, col, data))
    assert np.linalg.norm(D - D.T) <= 1e-14 * np.linalg.norm(D)
    # the default FP64 iteration mirrors its off-diagonal blocks; its diagonal blocks
    # are computed, so they are symmetric to rounding
    f = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, 1e-7, 1e-8)
    rp, col, data = f.P.export()
    D = bsr.to_dense(bsr.Mat(h.H.blk_size, rp, col, data))
    assert np.linalg.norm(D - D.T) <= 1e-14 * np.linalg.norm(D)

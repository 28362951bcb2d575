"""GPU parity of the BF16 tensor-core product and the mixed-precision sign iteration.

BF16 product: the oracle multiplies the operands rounded to bfloat16 (nearest,
ties to even) in FP64; the GPU accumulates the same exact bf16 x bf16 products
in FP32, so the difference is bounded by FP32 summation: |d_ij| <= K_ij u32 (|A||B|)_ij.
Split BF16 product (BF16X3): the oracle forms Ah Bh + Ah Bl + Al Bh in FP64 from
hi = bf16(x), lo = bf16(x - hi); the GPU accumulates the same exact products in FP32.
Mixed sign iteration: the converged P must give the FP64 oracle's band energy
within 1e-6 Ha/atom."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import bsr, sign
from oracle.lowprec import round_bf16, split_bf16

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
    assert st.flops_tensor >= st.flops


def _split_reference(Ao, Bo):
    parts = []
    for M in (Ao, Bo):
        h, l = M.copy(), M.copy()
        h.data, l.data = split_bf16(M.data)
        parts.append((h, l))
    (Ah, Al), (Bh, Bl) = parts
    ref = bsr.multiply(1.0, Ah, Bh)
    for X, Y in ((Ah, Bl), (Al, Bh)):
        t = bsr.multiply(1.0, X, Y)
        assert np.array_equal(t.col, ref.col)
        ref.data = ref.data + t.data
    Aa, Ba = Ao.copy(), Bo.copy()
    Aa.data = np.abs(Aa.data)
    Ba.data = np.abs(Ba.data)
    return ref, bsr.multiply(1.0, Aa, Ba)


@pytest.mark.parametrize("si", range(len(SIZES)))
@pytest.mark.parametrize("density", [0.1, 0.6])
def test_bf16x3_product_matches_split_oracle(gb, si, density):
    bs = SIZES[si]
    a = synth.random_block_matrix(bs, density, 700 + si)
    b = synth.random_block_matrix(bs, density, 800 + si)
    A, B = gb.Matrix.of(a), gb.Matrix.of(b)
    Ao, Bo = bsr.Mat.of(a), bsr.Mat.of(b)
    C = gb.Matrix(A.blk_size, A.stream)
    st = gb.multiply(1.0, A, B, 0.0, C, 0.0, prec=gb.DBCSR_BF16X3)
    ref, mag = _split_reference(Ao, Bo)
    rp, col, data = C.export()
    assert np.array_equal(rp, ref.rp) and np.array_equal(col, ref.col)
    # three FP32 sums of exact products, each term at most (1 + 2^-8)^2 |a||b|
    kmax = int(np.max(bs)) * len(bs)
    assert np.all(np.abs(data - ref.data) <= 2 * kmax * U32 * 1.1 * mag.data + 1e-300)
    # about 16 significant bits: far closer to the FP64 product than plain BF16
    exact = bsr.multiply(1.0, Ao, Bo)
    assert np.all(np.abs(data - exact.data) <= (3 * 2.0 ** -16 + 2 * kmax * U32) * mag.data + 1e-300)
    assert st.flops == bsr.multiply(1.0, Ao, Bo, info=True)[1].flops
    # three MMAs per K step; group tiles and the 128-row MMA only add padded work
    assert st.flops_tensor >= 3 * st.flops


def test_bf16x3_filtered_product_keeps_the_split_oracle_pattern(gb):
    # norms far from eps: the filtered patterns agree
    bs = SIZES[1]
    a = synth.random_block_matrix(bs, 0.5, 901, symmetric=True)
    A, Ao = gb.Matrix.of(a), bsr.Mat.of(a)
    C = gb.Matrix(A.blk_size, A.stream)
    gb.multiply(1.0, A, A, 0.0, C, 1e-3, prec=gb.DBCSR_BF16X3)
    ref, _ = _split_reference(Ao, Ao)
    keep = bsr.keep_mask(ref, bsr.block_norms(ref)[0], 1e-3)
    rp, col, data = C.export()
    sel = bsr.select_blocks(ref, keep)
    assert np.array_equal(col, sel.col)
    assert np.allclose(data, sel.data, rtol=0, atol=1e-5 * np.abs(sel.data).max())


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


@pytest.mark.parametrize("low", ["bf16x3", "bf16", "bf16x3+correction"])
@pytest.mark.parametrize("n_mol,basis,eps", [(24, (13, 5), 1e-7), (16, (23, 7), 1e-6)])
def test_mixed_sign_matches_fp64_oracle(gb, n_mol, basis, eps, low):
    h = synth.build_hamiltonian(synth.small(n_mol, basis=basis, seed=990 + n_mol))
    lo = gb.DBCSR_BF16 if low == "bf16" else gb.DBCSR_BF16X3
    g = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, eps, 1e-8, prec=gb.DBCSR_MIXED, switch_tol=1e-4, low=lo,
                        low_correction=low.endswith("correction"))
    o = sign.sign_iterate(bsr.Mat.of(h.H), 0.0, eps, 1e-8)
    assert g.report.fp64_from > 1                     # some steps ran in the low tier
    assert g.converged or g.report.stalled
    assert abs(g.report.e_band - o.e_band) / h.n_atoms < DE_ATOM
    assert g.report.trace_p == pytest.approx(h.n_occ, abs=1e-4)
    assert g.report.ms_low > 0 and g.report.ms_low < g.report.ms_multiply


@pytest.mark.slow
def test_mixed_sign_1024_waters(gb):
    w = synth.SIGN_1024
    h = synth.build_hamiltonian(w)
    g = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, w.eps_filter, w.tol, prec=gb.DBCSR_MIXED, switch_tol=1e-4)
    ref = json.load(open(os.path.join(HERE, "golden", "sign_1024h2o.json")))
    assert g.report.fp64_from > 1
    assert abs(g.report.e_band - ref["e_band"]) / h.n_atoms < DE_ATOM
    assert g.report.trace_p == pytest.approx(4096, abs=1e-4)


@pytest.mark.parametrize("low", ["bf16x3", "bf16"])
def test_mixed_density_matrix_is_symmetric(gb, low):
    h = synth.build_hamiltonian(synth.small(24, seed=990 + 24))
    lo = gb.DBCSR_BF16X3 if low == "bf16x3" else gb.DBCSR_BF16
    g = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, 1e-7, 1e-8, prec=gb.DBCSR_MIXED, low=lo)
    rp, col, data = g.P.export()
    D = bsr.to_dense(bsr.Mat(h.H.blk_size, rp, col, data))
    assert np.array_equal(D, D.T)                     # the final X is replaced by its symmetric part


def test_fp64_density_matrix_is_exactly_symmetric(gb):
    # the default FP64 iteration mirrors its off-diagonal blocks and takes the symmetric part
    # of its diagonal blocks (a diagonal block of X X2 is symmetric only as far as X and the
    # filtered X2 commute, and under mirroring that antisymmetric part would grow)
    h = synth.build_hamiltonian(synth.small(24, seed=990 + 24))
    f = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, 1e-7, 1e-8)
    rp, col, data = f.P.export()
    D = bsr.to_dense(bsr.Mat(h.H.blk_size, rp, col, data))
    assert np.array_equal(D, D.T)


@pytest.mark.parametrize("order", [2, 3])
def test_mixed_fp64_tail_stays_converged(gb, order):
    # the split-BF16 tier leaves X near the FP64 filter floor; the FP64 tail must then hold
    # the residual there (max_iter well past convergence, tol below the floor)
    h = synth.build_hamiltonian(synth.small(24, seed=990 + 24))
    g = gb.sign_iterate(gb.Matrix.of(h.H), 0.0, 1e-7, 1e-14, prec=gb.DBCSR_MIXED, switch_tol=1e-4, order=order,
                        max_iter=30)
    r = [g.report.residual_history[i] for i in range(g.report.iterations)]
    tail = r[g.report.fp64_from - 1:]
    assert max(tail[2:] or [0.0]) < 1e-8
    assert all(np.isfinite(r))

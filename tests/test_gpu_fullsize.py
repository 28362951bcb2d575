"""Full-size products of the benchmark workloads, in the launch configuration the
benchmark times (empty tune table), checked on outputs the oracle computes one block
at a time: whole sampled block rows (pattern after the eps_filter truncation, and
values) of H*H on 1,024 waters, and sampled blocks of H*H on 4,096 waters with 23/7
blocks in FP64 and in split BF16."""
import numpy as np
import pytest

import synth
from oracle import bsr
from oracle.lowprec import split_bf16

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2003_03868_gb300 as m
    m.lib()
    m.tune_clear()
    return m


def _gpu_blocks(C):
    rp, col, data = C.export()
    M = bsr.Mat(C.blk_size, rp, col, data)
    return M


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_sign1024_product_sampled_rows_and_blocks(gb):
    w = synth.SIGN_1024
    h = synth.build_hamiltonian(w)
    Ho = bsr.Mat.of(h.H)
    H = gb.Matrix.of(h.H)
    C = gb.Matrix(H.blk_size, H.stream)
    eps = w.eps_filter
    st = gb.multiply(1.0, H, H, 0.0, C, eps)
    G = _gpu_blocks(C)
    assert st.n_kept == G.nnzb
    rp_o, col_o = bsr.product_pattern(Ho, Ho)
    assert st.n_candidates == int(rp_o[-1])
    rng = np.random.default_rng(1024)
    # whole rows: every candidate block by the oracle, the kept set, and the values
    for I in rng.choice(Ho.nblk, 3, replace=False):
        cand = col_o[rp_o[I]:rp_o[I + 1]]
        ref = {int(J): bsr.product_block(int(I), int(J), 1.0, Ho, Ho) for J in cand}
        norms = {J: np.linalg.norm(b) for J, b in ref.items()}
        kept = {J for J in ref if J == I or norms[J] >= eps}
        got = set(int(J) for J in G.col[G.rp[I]:G.rp[I + 1]])
        # a block whose norm is within rounding of eps may land on either side
        ties = {J for J in ref if abs(norms[J] - eps) <= 1e-12 * eps}
        assert (got ^ kept) <= ties
        for J in got & kept:
            assert _rel(G.block(int(I), J), ref[J]) <= 1e-12
    # random kept blocks anywhere
    for b in rng.choice(G.nnzb, 300, replace=False):
        I, J = int(G.rows[b]), int(G.col[b])
        assert _rel(G.block(I, J), bsr.product_block(I, J, 1.0, Ho, Ho)) <= 1e-12


def _split_block(Ho, I, J):
    """Block (I, J) of the split-BF16 product Ah Bh + Ah Bl + Al Bh (H symmetric: B_KJ = H_JK^T),
    and of |H| |H| for the rounding bound, in FP64."""
    m, n = int(Ho.bs[I]), int(Ho.bs[J])
    ref = np.zeros((m, n))
    mag = np.zeros((m, n))
    ksum = 0
    for q in range(int(Ho.rp[I]), int(Ho.rp[I + 1])):
        K = int(Ho.col[q])
        B = Ho.block(K, J)
        if B is None:
            continue
        A = Ho.block(I, K)
        ah, al = split_bf16(A)
        bh, bl = split_bf16(B)
        ref += ah @ bh + ah @ bl + al @ bh
        mag += np.abs(A) @ np.abs(B)
        ksum += int(Ho.bs[K])
    return ref, mag, ksum


def test_sign4096_23_7_products_sampled(gb):
    w = synth.SIGN_4096
    h = synth.build_hamiltonian(w)
    Ho = bsr.Mat.of(h.H)
    H = gb.Matrix.of(h.H)
    rng = np.random.default_rng(4096)
    C = gb.Matrix(H.blk_size, H.stream)
    gb.multiply(1.0, H, H, 0.0, C, w.eps_filter)
    G = _gpu_blocks(C)
    for b in rng.choice(G.nnzb, 120, replace=False):
        I, J = int(G.rows[b]), int(G.col[b])
        assert _rel(G.block(I, J), bsr.product_block(I, J, 1.0, Ho, Ho)) <= 1e-12
    del C, G
    C3 = gb.Matrix(H.blk_size, H.stream)
    gb.multiply(1.0, H, H, 0.0, C3, w.eps_filter, prec=gb.DBCSR_BF16X3)
    G3 = _gpu_blocks(C3)
    for b in rng.choice(G3.nnzb, 60, replace=False):
        I, J = int(G3.rows[b]), int(G3.col[b])
        ref, mag, ksum = _split_block(Ho, I, J)
        assert np.all(np.abs(G3.block(I, J) - ref) <= 2 * ksum * U32 * 1.1 * mag + 1e-300)

"""GPU parity of the submatrix method (dbcsr_submatrix_sign: batched dense sign of every
block column's neighbourhood) against the oracle's per-submatrix eigendecomposition."""
import numpy as np
import pytest

import synth
from oracle import bsr, submatrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2003_03868_gb300 as m
    m.lib()
    return m


def _mat(M):
    rp, col, data = M.export()
    return bsr.Mat(M.blk_size, rp, col, data)


@pytest.mark.parametrize("n_mol,basis", [(4, (13, 5)), (48, (4, 1)), (40, (13, 5)), (24, (23, 7))])
def test_submatrix_matches_oracle(gb, n_mol, basis):
    h = synth.build_hamiltonian(synth.small(n_mol, basis=basis, seed=6000 + n_mol))
    Ho = bsr.Mat.of(h.H)
    o = submatrix.submatrix_density(Ho, 0.0)
    g = gb.submatrix_sign(gb.Matrix.of(h.H), 0.0, 1e-12)
    assert g.converged
    P = _mat(g.P)
    assert np.array_equal(P.rp, o.rp) and np.array_equal(P.col, o.col)
    assert np.linalg.norm(P.data - o.data) / np.linalg.norm(o.data) < 1e-10
    assert g.report.n_products == Ho.nblk                      # one submatrix per block column
    assert g.report.e_band == pytest.approx(bsr.trace_product(o, Ho), abs=1e-9 * h.n_atoms)


def test_complete_neighbourhoods_give_the_exact_projector(gb):
    h = synth.build_hamiltonian(synth.small(4, seed=77))
    Hd = bsr.to_dense(bsr.Mat.of(h.H))
    w, Q = np.linalg.eigh(Hd)
    g = gb.submatrix_sign(gb.Matrix.of(h.H), 0.0, 1e-13)
    assert np.linalg.norm(bsr.to_dense(_mat(g.P)) - Q[:, w < 0] @ Q[:, w < 0].T) < 1e-11


def test_submatrix_fp32_tf32(gb):
    h = synth.build_hamiltonian(synth.small(48, basis=(4, 1), seed=6100))
    H = gb.Matrix.of(h.H)
    f = gb.submatrix_sign(H, 0.0, 1e-12)
    m = gb.submatrix_sign(H, 0.0, 1e-5, prec=gb.DBCSR_MIXED)
    assert m.converged and m.report.fp64_from > 1             # some steps on the TF32 tensor cores
    # FP32 floor: elements of X to about 1e-5 on these ~300-dimensional submatrices
    assert abs(m.report.e_band - f.report.e_band) / h.n_atoms < 1e-5
    assert m.report.trace_p == pytest.approx(h.n_occ, abs=1e-3)


def test_submatrix_arguments_are_checked(gb):
    h = synth.build_hamiltonian(synth.small(4, seed=1))
    H = gb.Matrix.of(h.H)
    with pytest.raises(gb.DbcsrError) as e:
        gb.submatrix_sign(H, 0.0, 1e-9, P=H)
    assert e.value.status == gb._ffi.DBCSR_EINVAL
    with pytest.raises(gb.DbcsrError) as e:
        gb.submatrix_sign(H, 0.0, 0.0)
    assert e.value.status == gb._ffi.DBCSR_EINVAL


@pytest.mark.parametrize("n,nb", [(16, 1), (100, 3), (130, 2), (132, 2), (257, 1), (260, 1), (400, 2)])
def test_dense_products_match_fp64_reference(gb, n, nb):
    # the submatrix method's dense kernels against FP64 products: FP64 to rounding; TF32 and
    # split TF32 within the truncation of their operands to TF32 (as the tensor cores read FP32:
    # below 2^-10 relative per operand; split: hi*lo, lo*hi and the dropped lo*lo, each below
    # 2^-20 |a||b|) plus FP32 summation over n terms
    import torch
    rng = np.random.default_rng(n + nb)
    A = rng.uniform(-1, 1, (nb, n, n))
    B = rng.uniform(-1, 1, (nb, n, n))
    C0 = rng.uniform(-1, 1, (nb, n, n))
    ref = -0.5 * np.einsum("bij,bjk->bik", A, B) + 1.5 * C0
    mag = 0.5 * np.einsum("bij,bjk->bik", np.abs(A), np.abs(B)) + 1.5 * np.abs(C0)
    for prec, dt, tol in ((gb.DBCSR_FP64, torch.float64, 4 * n * 2.0 ** -53),
                          (gb.DBCSR_TF32, torch.float32, 2.0 ** -9 + n * 2.0 ** -24),
                          (gb.DBCSR_TF32X3, torch.float32, 2.0 ** -18 + n * 2.0 ** -24)):
        a = torch.tensor(A, dtype=dt, device="cuda")
        b = torch.tensor(B, dtype=dt, device="cuda")
        c = torch.tensor(C0, dtype=dt, device="cuda")
        gb.dense_multiply(prec, nb, n, -0.5, a.data_ptr(), b.data_ptr(), 1.5, c.data_ptr())
        torch.cuda.synchronize()
        got = c.double().cpu().numpy()
        # the inputs as the kernel saw them (FP32 data carries its own rounding)
        inp_err = 0 if dt == torch.float64 else 2.0 ** -23 * 3
        assert np.all(np.abs(got - ref) <= (tol + inp_err) * mag + 1e-300), prec
    if n >= 100:     # plain TF32 really rounds: its error is far above split TF32's
        a = torch.tensor(A, dtype=torch.float32, device="cuda")
        b = torch.tensor(B, dtype=torch.float32, device="cuda")
        errs = []
        for prec in (gb.DBCSR_TF32, gb.DBCSR_TF32X3):
            c = torch.zeros((nb, n, n), dtype=torch.float32, device="cuda")
            gb.dense_multiply(prec, nb, n, 1.0, a.data_ptr(), b.data_ptr(), 0.0, c.data_ptr())
            errs.append(np.abs(c.double().cpu().numpy() - np.einsum("bij,bjk->bik", A, B)).max())
        assert errs[0] > 30 * errs[1]


@pytest.mark.parametrize("n,nb", [(4, 3), (8, 1), (20, 5), (252, 1), (256, 2), (268, 1)])
def test_dense_tf32_edge_sizes(gb, n, nb):
    # sizes at the edges of the tensor-map path (n a multiple of 4): a single 16-column stage
    # partly past n, one or two 256-row tiles of B^T, N tiles of 16 rows; products against
    # float64 with the truncation bound (2^-9 plain, 2^-18 split) plus FP32 summation
    import torch
    rng = np.random.default_rng(1000 + n)
    A = rng.uniform(-1, 1, (nb, n, n))
    B = rng.uniform(-1, 1, (nb, n, n))
    a = torch.tensor(A, dtype=torch.float32, device="cuda")
    b = torch.tensor(B, dtype=torch.float32, device="cuda")
    A32, B32 = a.double().cpu().numpy(), b.double().cpu().numpy()
    ref = np.einsum("bij,bjk->bik", A32, B32)
    mag = np.einsum("bij,bjk->bik", np.abs(A32), np.abs(B32))
    for prec, tol in ((gb.DBCSR_TF32, 2.0 ** -9), (gb.DBCSR_TF32X3, 2.0 ** -18)):
        c = torch.full((nb, n, n), float("nan"), dtype=torch.float32, device="cuda")
        gb.dense_multiply(prec, nb, n, 1.0, a.data_ptr(), b.data_ptr(), 0.0, c.data_ptr())
        torch.cuda.synchronize()
        got = c.double().cpu().numpy()
        assert np.all(np.isfinite(got)), prec
        assert np.all(np.abs(got - ref) <= (tol + n * 2.0 ** -24) * mag + 1e-30), prec

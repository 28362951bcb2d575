"""The tune table's host-side logic (set, get, save, load, validation) without a GPU."""
import os

import numpy as np

import pytest


@pytest.fixture(scope="module")
def gb():
    from paper_2003_03868_gb300 import build
    build.build()
    import paper_2003_03868_gb300 as m
    return m


def test_table_round_trip(gb, tmp_path):
    gb.tune_clear()
    c = gb.KernelCfg(128, 8, 1, 1, 1)
    gb.tune_set(gb.DBCSR_FP64, 13, 5, 13, c)
    gb.tune_set(gb.DBCSR_FP64, 23, 7, 23, gb.KernelCfg(64, 16, 0, 0, 2))      # 161 = 5 * 32 + 1: K-split
    got, found = gb.tune_get(gb.DBCSR_FP64, 13, 5, 13)
    assert found and (got.tpb, got.ctas_per_sm, got.colmajor, got.prefetch2, got.split) == (128, 8, 1, 1, 1)
    path = str(tmp_path / "tune.txt")
    gb.tune_save(path)
    gb.tune_clear()
    assert not gb.tune_get(gb.DBCSR_FP64, 13, 5, 13)[1]
    gb.tune_load(path)
    got, found = gb.tune_get(gb.DBCSR_FP64, 23, 7, 23)
    assert found and (got.tpb, got.ctas_per_sm, got.split) == (64, 16, 2)
    gb.tune_set(gb.DBCSR_FP64, 13, 5, 13, None)
    assert not gb.tune_get(gb.DBCSR_FP64, 13, 5, 13)[1]
    gb.tune_clear()


def test_default_when_absent_and_validation(gb, tmp_path):
    gb.tune_clear()
    c, found = gb.tune_get(gb.DBCSR_FP64, 4, 4, 4)
    assert not found and c.tpb == 256 and c.split == -1
    with pytest.raises(gb.DbcsrError):
        gb.tune_set(gb.DBCSR_FP64, 0, 5, 5, gb.KernelCfg(128, 8, 0, 0, 0))
    with pytest.raises(gb.DbcsrError):                           # a warp pair for 16 elements
        gb.tune_set(gb.DBCSR_FP64, 4, 4, 4, gb.KernelCfg(128, 8, 0, 0, 1))
    with pytest.raises(gb.DbcsrError):                           # K-split: 169 = 5 * 32 + 9 elements
        gb.tune_set(gb.DBCSR_FP64, 13, 13, 13, gb.KernelCfg(128, 8, 0, 0, 2))
    bad = tmp_path / "bad.txt"
    bad.write_text("0 13 5 13 100 8 0 0 0\n")     # 100 threads: not a multiple of 32
    with pytest.raises(gb.DbcsrError):
        gb.tune_load(str(bad))
    bad.write_text("0 13 5 13 128 8 0 0\n")       # the split field missing
    with pytest.raises(gb.DbcsrError):
        gb.tune_load(str(bad))
    # work splits x threads x CTAs per SM x lane order x prefetch; no per-shape BF16 kernels
    space = gb.tune_space(gb.DBCSR_FP64)
    assert len(space) == 96 and {c.split for c in space} == {0, 1, 2}
    with pytest.raises(gb.DbcsrError):
        gb.tune_space(gb.DBCSR_BF16)


def test_mlp_host_side_init_and_features(gb):
    import numpy as np
    from oracle import mlp as omlp
    p = gb.mlp_init(10, seed=1)
    assert p.size == omlp.n_params(10)
    W1, b1, W2, b2, W3, b3 = omlp.unpack(p, 10)
    assert gb.MLP_FEATURES == 12
    assert np.all(b1 == 0) and np.all(b2 == 0) and b3 == 0
    assert np.abs(W1).max() <= np.sqrt(6 / 74) and np.abs(W2).max() <= np.sqrt(6 / 128)
    # 13 x 5 = 65 elements: one warp uses 3 slots per lane (96 lane slots); a pair 2 per lane;
    # the K-split 2 per lane plus the remainder element
    f = gb.mlp_features([(13, 5, 13)] * 3, [gb.KernelCfg(128, 8, 1, 0, s) for s in (0, 1, 2)])
    base = [13 / 32, 5 / 32, 13 / 32, np.log2(845) / 15]
    np.testing.assert_allclose(f[0], base + [65 / 96, 0.0, 0.5, 0.5, 1.0, 0.0, 0.0, 3 / 32], rtol=1e-6)
    np.testing.assert_allclose(f[1], base + [65 / 96, 0.0, 0.5, 0.5, 1.0, 0.0, 1.0, 2 / 32], rtol=1e-6)
    np.testing.assert_allclose(f[2], base + [65 / 96, 1.0, 0.5, 0.5, 1.0, 0.0, 0.0, 2 / 32], rtol=1e-6)


def _records(gb, rng, prec, triples):
    recs = []
    for (m, n, k) in triples:
        for c in gb.tune_space(gb.DBCSR_FP64)[::7]:
            mn = m * n
            if (c.split == 1 and mn <= 32) or (c.split == 2 and not (mn > 32 and mn % 32 == 1)):
                continue
            r = gb.TuneRecord()
            r.m, r.n, r.k, r.prec = m, n, k, prec
            r.cfg = c
            r.ms = float(np.exp(rng.normal(0.0, 0.5)) * m * n * k / 1e3)
            r.gflops = 1.0
            recs.append(r)
    return recs


def test_predictor_training_data_from_records_file(gb, tmp_path):
    # the targets dbcsr_predictor_train regresses: log time, centred per (m, n, k) triple,
    # divided by the population standard deviation of the centred values
    rng = np.random.default_rng(21)
    rf = _records(gb, rng, gb.DBCSR_FP64, [(13, 5, 13), (23, 7, 23), (4, 4, 4)])
    rb = _records(gb, rng, 99, [(13, 13, 13)])       # records of another precision are skipped
    path = str(tmp_path / "recs.tune")
    gb.tune_records_save(path, rf[:5])
    gb.tune_records_save(path, rf[5:] + rb, append=True)
    X, T = gb.predictor_data(path, gb.DBCSR_FP64)
    assert X.shape == (len(rf), gb.MLP_FEATURES) and T.shape == (len(rf),)
    tri = [(r.m, r.n, r.k) for r in rf]
    np.testing.assert_array_equal(X, gb.mlp_features(tri, [r.cfg for r in rf]))
    y = np.log(np.array([r.ms for r in rf]))
    mean = {t: np.mean([yy for tt, yy in zip(tri, y) if tt == t]) for t in set(tri)}
    t = np.array([yy - mean[tt] for tt, yy in zip(tri, y)])
    np.testing.assert_allclose(T, t / t.std(), rtol=1e-6, atol=1e-6)
    for tt in set(tri):                           # centred per triple
        assert abs(np.mean([v for v, u in zip(T, tri) if u == tt])) < 1e-5
    assert abs(float(np.std(T.astype(np.float64))) - 1.0) < 1e-5
    Xb, Tb = gb.predictor_data(path, 99)
    assert Xb.shape[0] == len(rb)


def test_predictor_records_are_checked(gb, tmp_path):
    bad = tmp_path / "bad.tune"
    bad.write_text("0 13 5 13 128 8 0 0 0 -1.0\n")     # a non-positive time
    with pytest.raises(gb.DbcsrError):
        gb.predictor_data(str(bad))
    bad.write_text("0 13 5 13 128 8 0 0 -1.0\n")       # a field missing
    with pytest.raises(gb.DbcsrError):
        gb.predictor_data(str(bad))
    bad.write_text("# nothing\n")
    with pytest.raises(gb.DbcsrError):
        gb.predictor_data(str(bad))
    with pytest.raises(gb.DbcsrError):
        gb.predictor_data(str(tmp_path / "missing.tune"))
    # no model trained yet for the plain BF16 precision (params == NULL is refused)
    p = np.zeros(gb.lib().dbcsr_mlp_param_count(gb.MLP_FEATURES), dtype=np.float32)
    assert gb.lib().dbcsr_predictor_params(99, gb._ptr(p)) == gb._ffi.DBCSR_ESTATE

"""The tune table's host-side logic (set, get, save, load, validation) without a GPU."""
import os

import pytest


@pytest.fixture(scope="module")
def gb():
    from paper_2003_03868_gb300 import build
    build.build()
    import paper_2003_03868_gb300 as m
    return m


def test_table_round_trip(gb, tmp_path):
    gb.tune_clear()
    c = gb.KernelCfg(128, 8, 1, 1)
    gb.tune_set(gb.DBCSR_FP64, 13, 5, 13, c)
    gb.tune_set(gb.DBCSR_BF16, 23, 7, 23, gb.KernelCfg(64, 16, 0, 0))
    got, found = gb.tune_get(gb.DBCSR_FP64, 13, 5, 13)
    assert found and (got.tpb, got.ctas_per_sm, got.colmajor, got.prefetch2) == (128, 8, 1, 1)
    path = str(tmp_path / "tune.txt")
    gb.tune_save(path)
    gb.tune_clear()
    assert not gb.tune_get(gb.DBCSR_FP64, 13, 5, 13)[1]
    gb.tune_load(path)
    got, found = gb.tune_get(gb.DBCSR_BF16, 23, 7, 23)
    assert found and (got.tpb, got.ctas_per_sm) == (64, 16)
    gb.tune_set(gb.DBCSR_FP64, 13, 5, 13, None)
    assert not gb.tune_get(gb.DBCSR_FP64, 13, 5, 13)[1]
    gb.tune_clear()


def test_default_when_absent_and_validation(gb, tmp_path):
    gb.tune_clear()
    c, found = gb.tune_get(gb.DBCSR_FP64, 4, 4, 4)
    assert not found and c.tpb == 256
    with pytest.raises(gb.DbcsrError):
        gb.tune_set(gb.DBCSR_FP64, 0, 5, 5, gb.KernelCfg(128, 8, 0, 0))
    bad = tmp_path / "bad.txt"
    bad.write_text("0 13 5 13 100 8 0 0\n")       # 100 threads: not a multiple of 32
    with pytest.raises(gb.DbcsrError):
        gb.tune_load(str(bad))
    assert len(gb.tune_space(gb.DBCSR_FP64)) == 60 and len(gb.tune_space(gb.DBCSR_BF16)) == 15


def test_mlp_host_side_init_and_features(gb):
    import numpy as np
    from oracle import mlp as omlp
    p = gb.mlp_init(10, seed=1)
    assert p.size == omlp.n_params(10)
    W1, b1, W2, b2, W3, b3 = omlp.unpack(p, 10)
    assert np.all(b1 == 0) and np.all(b2 == 0) and b3 == 0
    assert np.abs(W1).max() <= np.sqrt(6 / 74) and np.abs(W2).max() <= np.sqrt(6 / 128)
    f = gb.mlp_features([(13, 5, 13)], [gb.KernelCfg(128, 8, 1, 0)])[0]
    expect = [13 / 32, 5 / 32, 13 / 32, np.log2(845) / 15, 65 / 96, 1.0, 0.5, 0.5, 1.0, 0.0]
    np.testing.assert_allclose(f, expect, rtol=1e-6)

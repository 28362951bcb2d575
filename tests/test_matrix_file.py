"""The matrix file format, checked on the host without a GPU (dbcsr_file_info), and the
save / load round trip on the GPU."""
import zlib

import numpy as np
import pytest

import synth


def _write(path, bs, rp, col, data, magic=b"DBCSRGB1", zero=0, extra=b"", crc_delta=0):
    body = b"".join([magic, np.int32(len(bs)).tobytes(), np.int32(zero).tobytes(), np.int64(len(col)).tobytes(),
                     np.int64(len(data)).tobytes(), np.asarray(bs, np.int32).tobytes(),
                     np.asarray(rp, np.int64).tobytes(), np.asarray(col, np.int32).tobytes(),
                     np.asarray(data, np.float64).tobytes()])
    crc = (zlib.crc32(body) + crc_delta) & 0xFFFFFFFF
    with open(path, "wb") as f:
        f.write(body + np.uint32(crc).tobytes() + extra)


@pytest.fixture(scope="module")
def gb():
    import paper_2003_03868_gb300 as m
    m.lib()
    return m


@pytest.fixture
def good(tmp_path):
    a = synth.random_block_matrix([13, 5, 5, 23, 7, 1] * 3, 0.4, 5, empty_rows=(4,))
    p = tmp_path / "m.bin"
    _write(p, a.blk_size, a.row_ptr, a.col, a.data)
    return a, p


def test_file_info_reads_a_valid_file(gb, good):
    a, p = good
    assert gb.file_info(str(p)) == (18, a.col.shape[0], a.data.shape[0])


@pytest.mark.parametrize("breakage", ["magic", "short", "trailing", "reserved", "col_order", "col_range",
                                      "row_ptr", "row_ptr_past_end", "data_size", "block_edge", "checksum", "flipped_bit"])
def test_file_info_rejects_broken_files(gb, good, tmp_path, breakage):
    a, _ = good
    bs, rp, col, data = a.blk_size.copy(), a.row_ptr.copy(), a.col.copy(), a.data.copy()
    kw = {}
    if breakage == "magic":
        kw["magic"] = b"DBCSRGB2"
    elif breakage == "trailing":
        kw["extra"] = b"\0"
    elif breakage == "reserved":
        kw["zero"] = 1
    elif breakage == "col_order":
        i = int(np.argmax(np.diff(rp) >= 2))
        col[rp[i]], col[rp[i] + 1] = col[rp[i] + 1], col[rp[i]]
    elif breakage == "col_range":
        col[0] = len(bs)
    elif breakage == "row_ptr":
        rp[-1] -= 1
    elif breakage == "row_ptr_past_end":
        # an inner pointer beyond the column count, the last one still right (the file's
        # CRC is recomputed, so only the layout check can catch it)
        rp[1] = len(col) + 50
    elif breakage == "data_size":
        data = data[:-1]
    elif breakage == "block_edge":
        bs[0] = 33
    elif breakage == "checksum":
        kw["crc_delta"] = 1
    p = tmp_path / "bad.bin"
    _write(p, bs, rp, col, data, **kw)
    if breakage == "short":
        raw = open(p, "rb").read()
        open(p, "wb").write(raw[:-5])
    elif breakage == "flipped_bit":                         # one bit of the data, CRC unchanged
        raw = bytearray(open(p, "rb").read())
        raw[-20] ^= 0x04
        open(p, "wb").write(bytes(raw))
    with pytest.raises(gb.DbcsrError) as e:
        gb.file_info(str(p))
    assert e.value.status == gb._ffi.DBCSR_EINVAL
    with pytest.raises(gb.DbcsrError):
        gb.file_info(str(tmp_path / "missing.bin"))


@pytest.mark.gpu
def test_save_load_round_trip(gb, good, tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    a, p = good
    M = gb.Matrix.of(a)
    out = tmp_path / "saved.bin"
    M.save(str(out))
    assert open(out, "rb").read() == open(p, "rb").read()     # the same bytes as the layout above
    L = gb.Matrix.load(str(out))
    assert np.array_equal(L.blk_size, a.blk_size)
    for x, y in zip(L.export(), (a.row_ptr, a.col, a.data)):
        assert np.array_equal(x, y)
    E = gb.Matrix.of(synth.random_block_matrix([5] * 4, 0.0, 1, diag=False))   # no blocks
    E.save(str(tmp_path / "empty.bin"))
    assert gb.file_info(str(tmp_path / "empty.bin")) == (4, 0, 0)
    assert gb.Matrix.load(str(tmp_path / "empty.bin")).nnzb == 0
